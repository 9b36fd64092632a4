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
#include <stddef.h>

#include "echo_device.cuh"

namespace echo {

constexpr int NH = 64, NIN = 5;
constexpr int NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1;  // 4609
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH;

// device form of the parameters used by the kernels.  The inference kernels copy
// the prefix up to W2 (MLP_INFER_BYTES) to shared memory; W2 and W2T serve training.
struct MlpDev {
    float W1[NH * NIN];
    float b1[NH];
    float b2[NH];
    float w3[NH];
    float b3;
    float pad[3];
    // B fragments of the hidden-layer product, [n-tile][k-tile][lane]: for lane
    // 4 g + t, (W2[8 nt + g][16 kk + 2t .. +1], W2[8 nt + g][16 kk + 2t + 8 .. +9])
    // as bf16 pairs, so that a warp reads one n-tile / k-tile in one 8-byte load
    uint2 W2F[NH / 8][NH / 16][32];
    __nv_bfloat16 W2[NH * NH];   // [out][in]
    __nv_bfloat16 W2T[NH * NH];  // [in][out]
};
constexpr int MLP_INFER_BYTES = (int)offsetof(MlpDev, W2);
static_assert(MLP_INFER_BYTES % 16 == 0, "inference prefix is copied in 16-byte words");
static_assert(offsetof(MlpDev, b1) % 8 == 0 && offsetof(MlpDev, b2) % 8 == 0 &&
                  offsetof(MlpDev, w3) % 8 == 0 && offsetof(MlpDev, W2F) % 8 == 0,
              "pairs are read as float2 / uint2");

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
    float D = to_f32(u[0]), U = to_f32(u[4]);
    float sx = to_f32(u[1]), sy = to_f32(u[2]), sz = to_f32(u[3]);
    float bx = to_f32(B[0]), by = to_f32(B[1]), bz = to_f32(B[2]);
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
// ignored).  Returns y of the lane's own sample.  The warp's 32 samples form two
// m-tiles of the m16n8k16 product; lane 4 g + t holds rows g and g + 8 of both,
// that is samples g, g + 8, g + 16, g + 24.  Fragment layouts: A rows g, g+8,
// cols 2t(+1), 2t+8(+1); B col g, rows 2t(+1), 2t+8(+1); C rows g, g+8, cols 2t,
// 2t+1.  The first layer computes exactly the hidden values of the lane's A
// fragments; each B fragment of W2 is read once and serves both m-tiles; the
// second layer's tanh and the output dot product run on the C fragments of one
// n-tile at a time, so only the A fragments stay live across the product.
__device__ __forceinline__ float mlp_warp_forward(const MlpDev &w, const float *x, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const int g = lane >> 2, t = lane & 3;
    unsigned A[2][4][4];
    {
        float xs[4][NIN];
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int f = 0; f < NIN; f++) xs[r][f] = __shfl_sync(FULL, x[f], g + 8 * r);
#pragma unroll
        for (int j = 0; j < 8; j++) {  // hidden columns 8 j + 2 t, 8 j + 2 t + 1
            const int col = 8 * j + 2 * t;
            const float2 bb = *reinterpret_cast<const float2 *>(&w.b1[col]);
            float wv[2 * NIN];  // rows col and col + 1 of W1: ten consecutive floats
            const float2 *wp = reinterpret_cast<const float2 *>(&w.W1[col * NIN]);
#pragma unroll
            for (int q = 0; q < NIN; q++) {
                const float2 v = wp[q];
                wv[2 * q] = v.x;
                wv[2 * q + 1] = v.y;
            }
            float h[4][2];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                float za = bb.x, zb = bb.y;
#pragma unroll
                for (int f = 0; f < NIN; f++) {
                    za = fmaf(wv[f], xs[r][f], za);
                    zb = fmaf(wv[NIN + f], xs[r][f], zb);
                }
                h[r][0] = tanh_fast(za);
                h[r][1] = tanh_fast(zb);
            }
            const int kk = j >> 1, hi = j & 1;
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                A[mt][kk][2 * hi + 0] = pack_bf16(h[2 * mt][0], h[2 * mt][1]);          // row g
                A[mt][kk][2 * hi + 1] = pack_bf16(h[2 * mt + 1][0], h[2 * mt + 1][1]);  // row g + 8
            }
        }
    }
    float p[4] = {0.f, 0.f, 0.f, 0.f};  // partial y of samples g, g + 8, g + 16, g + 24
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int col = 8 * nt + 2 * t;
        const float2 b2 = *reinterpret_cast<const float2 *>(&w.b2[col]);
        const float2 w3 = *reinterpret_cast<const float2 *>(&w.w3[col]);
        float acc[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            acc[mt][0] = acc[mt][2] = b2.x;
            acc[mt][1] = acc[mt][3] = b2.y;
        }
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            const uint2 b = w.W2F[nt][kk][lane];
            mma_bf16(acc[0], A[0][kk], b.x, b.y);
            mma_bf16(acc[1], A[1][kk], b.x, b.y);
        }
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            p[2 * mt] = fmaf(w3.x, tanh_fast(acc[mt][0]), p[2 * mt]);
            p[2 * mt] = fmaf(w3.y, tanh_fast(acc[mt][1]), p[2 * mt]);
            p[2 * mt + 1] = fmaf(w3.x, tanh_fast(acc[mt][2]), p[2 * mt + 1]);
            p[2 * mt + 1] = fmaf(w3.y, tanh_fast(acc[mt][3]), p[2 * mt + 1]);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        p[r] += __shfl_xor_sync(FULL, p[r], 1);
        p[r] += __shfl_xor_sync(FULL, p[r], 2);
    }
    // sample s = lane sits in row s & 7 of quad s >> 3, held by lane 4 (s & 7)
    const int src = 4 * (lane & 7), q = lane >> 3;
    float v[4];
#pragma unroll
    for (int r = 0; r < 4; r++) v[r] = __shfl_sync(FULL, p[r], src);
    return (q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? v[2] : v[3]) + w.b3;
}

// Learned starting guess of the lane's cell, W0 = U y, rounded through float (the
// precision of the network's output).  Every lane of the warp calls it together
// (the product is warp-wide); a lane without a cell passes any finite state and
// ignores the result.  w: the parameters in shared or global memory.
__device__ __forceinline__ double mlp_guess_warp(const MlpDev &w, const double *u,
                                                 const double *B, int lane)
{
    float x[NIN];
    mlp_features(u, B, x);
    const float y = mlp_warp_forward(w, x, lane);
    return to_f64(to_f32(u[4] * to_f64(y)));
}

// the inference prefix of the parameters into shared memory (sw: MLP_INFER_BYTES,
// 16-byte aligned); the block synchronises before returning
__device__ __forceinline__ const MlpDev &load_mlp_shared(unsigned char *sw, const MlpDev *w)
{
    const int4 *src = reinterpret_cast<const int4 *>(w);
    int4 *dst = reinterpret_cast<int4 *>(sw);
    for (int q = threadIdx.x; q < MLP_INFER_BYTES / 16; q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    return *reinterpret_cast<const MlpDev *>(sw);
}

}  // namespace echo
