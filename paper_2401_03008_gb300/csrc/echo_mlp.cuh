// Device side of the learned Newton starting guess, shared by the inversion
// kernel (fused inference) and the training/inference entry points.
//
// Network 5 -> 64 -> 64 -> 1 (tanh, tanh, linear) on five rotation-invariant,
// dimensionless features of a cell's conserved state; output y = W/U, guess
// W0 = U y.  Parameters: one flat float vector of 4609 values,
// W1[64][5], b1[64], W2[64][64], b2[64], w3[64], b3.  The 64x64 hidden layer runs
// as BF16 mma.sync.m16n8k16 with FP32 accumulation.
#pragma once

#include <cuda_bf16.h>

#include "echo_device.cuh"

namespace echo {

constexpr int NH = 64, NIN = 5;
constexpr int NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1;  // 4609
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH;

// device form of the parameters used by the kernels
struct MlpDev {
    float W1[NH * NIN];
    float b1[NH];
    float b2[NH];
    float w3[NH];
    float b3;
    float pad[3];
    __nv_bfloat16 W2[NH * NH];   // [out][in]
    __nv_bfloat16 W2T[NH * NH];  // [in][out]
};

__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// hardware tanh approximation (one SFU instruction); its error (about 2^-11) is
// below the bfloat16 rounding the hidden activations go through anyway
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

// features of one cell: D/U, S^2/U^2, B^2/U, (S.B)^2/(S^2 B^2), ln(U/D)
__device__ __forceinline__ void mlp_features(const double *u, const double *B, float *x)
{
    float D = (float)u[0], U = (float)u[4];
    float sx = (float)u[1], sy = (float)u[2], sz = (float)u[3];
    float bx = (float)B[0], by = (float)B[1], bz = (float)B[2];
    float S2 = sx * sx + sy * sy + sz * sz;
    float B2 = bx * bx + by * by + bz * bz;
    float SB = sx * bx + sy * by + sz * bz;
    float den = S2 * B2;
    x[0] = D / U;
    x[1] = S2 / (U * U);
    x[2] = B2 / U;
    x[3] = den > 0.f ? SB * SB / den : 0.f;
    x[4] = logf(U / D);
}

// Forward pass of the 32 samples of a warp (lane = sample; x of inactive lanes is
// ignored).  Returns y of the lane's own sample.  Layout of the m16n8k16
// fragments: lane = 4 g + t; A rows g, g+8, cols 2t(+1), 2t+8(+1); B col g,
// rows 2t(+1), 2t+8(+1); C rows g, g+8, cols 2t, 2t+1.  The tanh outputs of the
// first layer land in exactly the A layout of the second product.
__device__ __forceinline__ float mlp_warp_forward(const MlpDev &w, const float *x, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const int g = lane >> 2, t = lane & 3;
    float ysel[2][2];
    // not unrolled: keeps the compiler from holding the first-layer weights of both
    // m-tiles in registers at once
#pragma unroll 1
    for (int mt = 0; mt < 2; mt++) {
        float xa[NIN], xb[NIN];
#pragma unroll
        for (int f = 0; f < NIN; f++) {
            xa[f] = __shfl_sync(FULL, x[f], 16 * mt + g);
            xb[f] = __shfl_sync(FULL, x[f], 16 * mt + g + 8);
        }
        unsigned A[4][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float ha[2], hb[2];
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const int col = 8 * j + 2 * t + e;
                float za = w.b1[col], zb = w.b1[col];
#pragma unroll
                for (int f = 0; f < NIN; f++) {
                    za = fmaf(w.W1[col * NIN + f], xa[f], za);
                    zb = fmaf(w.W1[col * NIN + f], xb[f], zb);
                }
                ha[e] = tanh_fast(za);
                hb[e] = tanh_fast(zb);
            }
            const int kk = j >> 1, hi = j & 1;
            A[kk][2 * hi + 0] = pack_bf16(ha[0], ha[1]);
            A[kk][2 * hi + 1] = pack_bf16(hb[0], hb[1]);
        }
        // hidden layer in two halves of four n-tiles (fewer live accumulators)
        float pa = 0.f, pb = 0.f;
#pragma unroll
        for (int jh = 0; jh < 2; jh++) {
            float acc[4][4];
#pragma unroll
            for (int jj = 0; jj < 4; jj++) {
                const int j = 4 * jh + jj;
                acc[jj][0] = acc[jj][2] = w.b2[8 * j + 2 * t];
                acc[jj][1] = acc[jj][3] = w.b2[8 * j + 2 * t + 1];
            }
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
#pragma unroll
                for (int jj = 0; jj < 4; jj++) {
                    const int j = 4 * jh + jj;
                    const __nv_bfloat16 *row = w.W2 + (8 * j + g) * NH + 16 * kk + 2 * t;
                    unsigned b0 = *reinterpret_cast<const unsigned *>(row);
                    unsigned b1 = *reinterpret_cast<const unsigned *>(row + 8);
                    mma_bf16(acc[jj], A[kk], b0, b1);
                }
            }
#pragma unroll
            for (int jj = 0; jj < 4; jj++) {
                const int j = 4 * jh + jj;
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const float w3 = w.w3[8 * j + 2 * t + e];
                    pa = fmaf(w3, tanh_fast(acc[jj][e]), pa);
                    pb = fmaf(w3, tanh_fast(acc[jj][2 + e]), pb);
                }
            }
        }
        pa += __shfl_xor_sync(FULL, pa, 1);
        pa += __shfl_xor_sync(FULL, pa, 2);
        pb += __shfl_xor_sync(FULL, pb, 1);
        pb += __shfl_xor_sync(FULL, pb, 2);
        ysel[mt][0] = pa + w.b3;
        ysel[mt][1] = pb + w.b3;
    }
    // sample s = lane: m-tile s/16, row r = s%16 -> quad 4 (r%8), half r/8
    const int r = lane & 15, src = 4 * (r & 7);
    float v00 = __shfl_sync(FULL, ysel[0][0], src), v01 = __shfl_sync(FULL, ysel[0][1], src);
    float v10 = __shfl_sync(FULL, ysel[1][0], src), v11 = __shfl_sync(FULL, ysel[1][1], src);
    const bool upper = lane >= 16, half = r >= 8;
    return upper ? (half ? v11 : v10) : (half ? v01 : v00);
}

__device__ __forceinline__ void load_mlp_shared(MlpDev &sw, const MlpDev *w)
{
    const int4 *src = reinterpret_cast<const int4 *>(w);
    int4 *dst = reinterpret_cast<int4 *>(&sw);
    for (int q = threadIdx.x; q < (int)(sizeof(MlpDev) / 16); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
}

}  // namespace echo
