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
#include <cuda_fp16.h>
#include <stddef.h>

#include "echo_device.cuh"

namespace echo {

constexpr int NH = 64, NIN = 5;
constexpr int NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1;  // 4609
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH;

// Device form of the parameters.  The inference part comes first (the prefix of
// MLP_INFER_BYTES that the inference kernels may copy to shared memory): every
// product runs on tensor cores with f16 operands, each weight matrix stored as
// the per-lane B fragments of mma.m16n8k16 (lane 4 g + t holds rows 2t, 2t+1 and
// 2t+8, 2t+9 of column g of the n-tile), so a warp reads a fragment with one
// 4- or 8-byte load.  Training reads the fp32 W1, w3 and the bf16 W2 copies.
struct MlpDev {
    uint2 W1H[NH / 8][32];           // layer 1, [n-tile][lane]: rows 2t, 2t+1, 2t+8, 2t+9 of
                                     // column g of (W1hi, W1hi, W1lo, 0) stacked along k
                                     // (k 0-4, 5-9, 10-14, 15), the f16 split W1 = hi + lo
    uint2 W2H[NH / 8][NH / 16][32];  // layer 2, [n-tile][k-tile][lane]: W2[8nt+g][16kk+2t..+1],
                                     // W2[8nt+g][16kk+2t+8..+9]
    uint2 W3H[NH / 16][32];          // output layer, [k-tile][lane]: w3 = hi + lo split over
                                     // columns 0 (hi) and 1 (lo), zero in the other six
    float b1[NH];
    float b2[NH];
    float b3;
    float pad[3];
    // training
    float W1[NH * NIN];
    float w3[NH];
    __nv_bfloat16 W2[NH * NH];   // [out][in]
    __nv_bfloat16 W2T[NH * NH];  // [in][out]
};
constexpr int MLP_INFER_BYTES = (int)offsetof(MlpDev, W1);
static_assert(MLP_INFER_BYTES % 16 == 0, "inference prefix is copied in 16-byte words");
static_assert(offsetof(MlpDev, b1) % 8 == 0 && offsetof(MlpDev, b2) % 8 == 0 &&
                  offsetof(MlpDev, W2H) % 8 == 0 && offsetof(MlpDev, W3H) % 8 == 0 &&
                  offsetof(MlpDev, w3) % 8 == 0,
              "pairs are read as float2 / uint2");

__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16(float *c, unsigned a0, unsigned a1, unsigned a2,
                                        unsigned a3, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
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

__device__ __forceinline__ unsigned pack_f16(float lo, float hi)
{
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

// tanh of two values rounded to f16, as a packed f16 pair (one SFU instruction for
// both): the A fragment of the next product comes out of it directly
__device__ __forceinline__ unsigned tanh_h2(float lo, float hi)
{
    unsigned r;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(r) : "r"(pack_f16(lo, hi)));
    return r;
}

// Features of one cell from its FP64 invariants D, S^2, B^2, S.B, U (the ones the
// inversion forms anyway): D/U, S^2/U^2, B^2/U, (S.B)^2/(S^2 B^2) (0 when S or B
// vanish), ln(U/D).  FP32 with the approximate reciprocal and logarithm: the
// features are rounded to f16 for the network.
__device__ __forceinline__ void mlp_features_inv(double D, double S2, double B2, double SB,
                                                 double U, float *x)
{
    const float d = to_f32(D), s2 = to_f32(S2), b2 = to_f32(B2), sb = to_f32(SB),
                u = to_f32(U);
    const float iu = __frcp_rn(u);
    const float den = s2 * b2;
    x[0] = d * iu;
    x[1] = s2 * iu * iu;
    x[2] = b2 * iu;
    x[3] = den > 0.f ? sb * sb * __frcp_rn(den) : 0.f;
    x[4] = __logf(u * __frcp_rn(d));
}

// features of one cell from its conserved variables u[5] and cell-centred field B[3]
__device__ __forceinline__ void mlp_features(const double *u, const double *B, float *x)
{
    mlp_features_inv(u[0], u[1] * u[1] + u[2] * u[2] + u[3] * u[3],
                     B[0] * B[0] + B[1] * B[1] + B[2] * B[2],
                     u[1] * B[0] + u[2] * B[1] + u[3] * B[2], u[4], x);
}

// Forward pass of the 32 samples of a warp (lane = sample; x of lanes without a
// sample is ignored); returns y of the lane's own sample.  The warp's samples form
// two m-tiles of 16 rows for mma.m16n8k16 (f16 operands, FP32 accumulation); lane
// 4 g + t holds rows g and g + 8 of a tile.  Layer 1 multiplies the features
// (columns 0..4 of k, the rest zero) by W1 with the bias as the accumulator's
// start; the accumulator of n-tiles 2 kk and 2 kk + 1, rows g and g + 8, columns
// 2t and 2t + 1, is exactly the A fragment of k-tile kk of the next product, so
// tanh of each packed f16 pair feeds it without any data movement.  Layer 2 runs
// two n-tiles at a time and its tanh pairs feed the output product, whose B has
// w3 in column 0: y of samples g, g + 8 of each m-tile lands in lane 4 g.
__device__ __forceinline__ float mlp_warp_forward(const MlpDev &w, const float *x, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const int g = lane >> 2, t = lane & 3;
    // Layer 1 as one product with k = 15: the features split as x = hi + lo in f16
    // times W1 = Whi + Wlo, keeping x_hi Whi + x_lo Whi + x_hi Wlo, so the first
    // layer is as accurate as FP32 (the dropped x_lo Wlo is below 2^-22 relative).
    // k columns: 0-4 x_hi, 5-9 x_lo, 10-14 x_hi, 15 zero; a lane's pair t of a row
    // is columns (2t, 2t+1) for a0/a1 and (2t+8, 2t+9) for a2/a3.
    float hi[NIN], lo[NIN];
#pragma unroll
    for (int f = 0; f < NIN; f++) {
        hi[f] = __half2float(__float2half_rn(x[f]));
        lo[f] = x[f] - hi[f];
    }
    const unsigned Q0 = pack_f16(hi[0], hi[1]), Q1 = pack_f16(hi[2], hi[3]),
                   Q2 = pack_f16(hi[4], lo[0]), Q3 = pack_f16(lo[1], lo[2]),
                   Q4 = pack_f16(lo[3], lo[4]), Q7 = pack_f16(hi[4], 0.f);
    // pair indices of this lane: (t) for columns 2t.., (4 + t) for 2t+8..:
    // 0:(Q0,Q4) 1:(Q1,Q0) 2:(Q2,Q1) 3:(Q3,Q7)
    unsigned a1[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int src = 16 * mt + 8 * h + g;
            const unsigned v0 = __shfl_sync(FULL, Q0, src), v1 = __shfl_sync(FULL, Q1, src),
                           v2 = __shfl_sync(FULL, Q2, src), v3 = __shfl_sync(FULL, Q3, src),
                           v4 = __shfl_sync(FULL, Q4, src), v7 = __shfl_sync(FULL, Q7, src);
            a1[mt][h] = t == 0 ? v0 : (t == 1 ? v1 : (t == 2 ? v2 : v3));
            a1[mt][2 + h] = t == 0 ? v4 : (t == 1 ? v0 : (t == 2 ? v1 : v7));
        }
    unsigned A[2][4][4];  // layer-2 A fragments [m-tile][k-tile]
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float2 bb = *reinterpret_cast<const float2 *>(&w.b1[8 * j + 2 * t]);
        const uint2 wb = w.W1H[j][lane];
        const int kk = j >> 1, hj = j & 1;
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            float c[4] = {bb.x, bb.y, bb.x, bb.y};
            mma_f16(c, a1[mt][0], a1[mt][1], a1[mt][2], a1[mt][3], wb.x, wb.y);
            A[mt][kk][2 * hj + 0] = tanh_h2(c[0], c[1]);  // row g
            A[mt][kk][2 * hj + 1] = tanh_h2(c[2], c[3]);  // row g + 8
        }
    }
    float yacc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int k3 = 0; k3 < 4; k3++) {  // layer-2 n-tiles 2 k3, 2 k3 + 1 = output k-tile k3
        unsigned A3[2][4];
#pragma unroll
        for (int hj = 0; hj < 2; hj++) {
            const int nt = 2 * k3 + hj;
            const float2 b2 = *reinterpret_cast<const float2 *>(&w.b2[8 * nt + 2 * t]);
            float acc[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                acc[mt][0] = acc[mt][2] = b2.x;
                acc[mt][1] = acc[mt][3] = b2.y;
            }
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
                const uint2 b = w.W2H[nt][kk][lane];
#pragma unroll
                for (int mt = 0; mt < 2; mt++)
                    mma_f16(acc[mt], A[mt][kk][0], A[mt][kk][1], A[mt][kk][2], A[mt][kk][3],
                            b.x, b.y);
            }
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                A3[mt][2 * hj + 0] = tanh_h2(acc[mt][0], acc[mt][1]);
                A3[mt][2 * hj + 1] = tanh_h2(acc[mt][2], acc[mt][3]);
            }
        }
        const uint2 b3 = w.W3H[k3][lane];
#pragma unroll
        for (int mt = 0; mt < 2; mt++)
            mma_f16(yacc[mt], A3[mt][0], A3[mt][1], A3[mt][2], A3[mt][3], b3.x, b3.y);
    }
    // sample s sits in m-tile s >> 4, row s & 15, held by lane 4 (s & 7): columns 0
    // (w3 hi) and 1 (w3 lo) are elements 0, 1 (row < 8) or 2, 3 (row >= 8)
    const int src = 4 * (lane & 7), q = lane >> 3;
    const float v0 = __shfl_sync(FULL, yacc[0][0] + yacc[0][1], src),
                v1 = __shfl_sync(FULL, yacc[0][2] + yacc[0][3], src),
                v2 = __shfl_sync(FULL, yacc[1][0] + yacc[1][1], src),
                v3 = __shfl_sync(FULL, yacc[1][2] + yacc[1][3], src);
    return (q == 0 ? v0 : q == 1 ? v1 : q == 2 ? v2 : v3) + w.b3;
}

// Learned starting guess of the lane's cell, W0 = U y, from the cell's invariants.  Every lane of
// the warp calls it together (the product is warp-wide); a lane without a cell
// passes any finite state and ignores the result.  w: the parameters in shared or
// global memory.
__device__ __forceinline__ double mlp_guess_warp(const MlpDev &w, const C2PInv &q, int lane)
{
    float x[NIN];
    mlp_features_inv(q.D, q.S2, q.B2, q.SB, q.U, x);
    const float y = mlp_warp_forward(w, x, lane);
    return q.U * to_f64(y);
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
