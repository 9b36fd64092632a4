// The learned Newton starting guess: inference inside the time step, training on
// states the solver itself produced, and the entry points that expose both.
//
// Network 5 -> 64 -> 64 -> 1 (tanh, tanh, linear) on five rotation-invariant,
// dimensionless features of a cell's conserved state; output y = W/U, guess
// W0 = U y.  Parameters: one flat float vector of 4609 values,
// W1[64][5], b1[64], W2[64][64], b2[64], w3[64], b3.
//
// Tensor cores: the 64x64 hidden layer (and, in training, the two 64x64 products
// of back-propagation) run as BF16 mma.sync.m16n8k16 with FP32 accumulation; the
// 5-input layer, the output dot product and all activations are FP32 on the CUDA
// cores.  The Newton iteration that follows always runs to tolerance, so the
// guess only changes the iteration count.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "echo_internal.h"
#include "echo_mlp.cuh"

namespace echo {

constexpr int MLP_BS = 128;

// y for caller-given features [n][5] (the inference kernel on its own)
__global__ void __launch_bounds__(MLP_BS)
k_mlp_forward(long n, const float *__restrict__ feats, const MlpDev *__restrict__ w,
              float *__restrict__ y)
{
    __shared__ __align__(16) unsigned char smem[MLP_INFER_BYTES];
    const MlpDev &sw = load_mlp_shared(smem, w);
    const long s = blockIdx.x * (long)MLP_BS + threadIdx.x;
    float x[NIN] = {0.5f, 0.f, 0.f, 0.f, 1.f};
    if (s < n)
        for (int f = 0; f < NIN; f++) x[f] = feats[s * NIN + f];
    float v = mlp_warp_forward(sw, x, threadIdx.x & 31);
    if (s < n) y[s] = v;
}

// build the device form from the flat FP32 parameters
__device__ __forceinline__ unsigned h2pair(float lo, float hi)
{
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

__global__ void k_mlp_build(const float *__restrict__ p, MlpDev *w)
{
    for (int q = threadIdx.x; q < NH * NH; q += blockDim.x) {
        int o = q / NH, i = q % NH;
        w->W2[q] = __float2bfloat16_rn(p[O_W2 + q]);
        w->W2T[i * NH + o] = __float2bfloat16_rn(p[O_W2 + q]);
    }
    for (int q = threadIdx.x; q < (NH / 8) * (NH / 16) * 32; q += blockDim.x) {
        const int nt = q / 128, kk = (q / 32) % 4, lane = q % 32, g = lane >> 2, t = lane & 3;
        const float *row = p + O_W2 + (8 * nt + g) * NH + 16 * kk + 2 * t;
        w->W2H[nt][kk][lane] = make_uint2(h2pair(row[0], row[1]), h2pair(row[8], row[9]));
    }
    // f16 split v = hi + lo of a weight
    auto hi16 = [](float v) { return __half2float(__float2half_rn(v)); };
    for (int q = threadIdx.x; q < (NH / 8) * 32; q += blockDim.x) {
        const int j = q / 32, lane = q % 32, g = lane >> 2, t = lane & 3;
        const float *row = p + O_W1 + (8 * j + g) * NIN;
        // k column c of the stacked (Whi, Whi, Wlo, 0)
        auto colv = [&](int c) -> float {
            if (c < NIN) return hi16(row[c]);
            if (c < 2 * NIN) return hi16(row[c - NIN]);
            if (c < 3 * NIN) return row[c - 2 * NIN] - hi16(row[c - 2 * NIN]);
            return 0.f;
        };
        w->W1H[j][lane] = make_uint2(h2pair(colv(2 * t), colv(2 * t + 1)),
                                     h2pair(colv(2 * t + 8), colv(2 * t + 9)));
    }
    for (int q = threadIdx.x; q < (NH / 16) * 32; q += blockDim.x) {
        const int kk = q / 32, lane = q % 32, g = lane >> 2, t = lane & 3;
        const float *v = p + O_W3 + 16 * kk + 2 * t;
        uint2 f = make_uint2(0u, 0u);
        if (g == 0) f = make_uint2(h2pair(hi16(v[0]), hi16(v[1])), h2pair(hi16(v[8]), hi16(v[9])));
        if (g == 1)
            f = make_uint2(h2pair(v[0] - hi16(v[0]), v[1] - hi16(v[1])),
                           h2pair(v[8] - hi16(v[8]), v[9] - hi16(v[9])));
        w->W3H[kk][lane] = f;
    }
    for (int q = threadIdx.x; q < NH * NIN; q += blockDim.x) w->W1[q] = p[O_W1 + q];
    for (int q = threadIdx.x; q < NH; q += blockDim.x) {
        w->b1[q] = p[O_B1 + q];
        w->b2[q] = p[O_B2 + q];
        w->w3[q] = p[O_W3 + q];
    }
    if (threadIdx.x == 0) {
        w->b3 = p[O_B3];
        w->pad[0] = w->pad[1] = w->pad[2] = 0.f;
    }
}

// features and the converged W/U of a strided subset of cells, written to a caller
// buffer (harvest of training states from the solver's own inversions).  Cell
// q stride + offset goes to slot base + q, so the buffer holds the states in cell
// order within each inversion and in inversion order across calls.
__global__ void __launch_bounds__(256)
k_mlp_harvest(Grid g, const double *__restrict__ U, const double *__restrict__ Bf,
              const double *__restrict__ W, long stride, long offset, float *feats,
              float *target, long base, long capacity)
{
    const long q = blockIdx.x * 256L + threadIdx.x;
    const long c = q * stride + offset;
    const long n = g.n;
    const long slot = base + q;
    if (c >= n || slot >= capacity) return;
    int i, j, k;
    coords(g, c, i, j, k);
    double B[3];
    for (int d = 0; d < 3; d++) B[d] = cell_field(g, Bf, c, i, j, k, d);
    double u[5];
    for (int v = 0; v < 5; v++) u[v] = U[v * n + c];
    float x[NIN];
    mlp_features(u, B, x);
    for (int f = 0; f < NIN; f++) feats[slot * NIN + f] = x[f];
    target[slot] = (float)(W[c] / u[4]);
}

// ---------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------

// C[M][64] (FP32) = A[M][K] (bf16, row-major) x Bt[64][K]^T (bf16, row-major);
// a block of 4 warps covers 64 rows, each warp 16 rows x 64 columns; M % 64 == 0,
// K % 16 == 0.  With kchunk < K, block y takes the K range [y kchunk, (y+1) kchunk)
// and adds its partial product into C (which the caller zeroes): the
// back-propagation product dW2 = dZ2^T H1 has only 64 rows but the batch as K.
__global__ void __launch_bounds__(128)
k_gemm_bf16(int M, int K, const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ Bt,
            float *__restrict__ C, int kchunk = 0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const long m0 = (long)blockIdx.x * 64 + warp * 16;
    if (m0 >= M) return;
    const bool split = kchunk > 0;
    const int kbeg = split ? blockIdx.y * kchunk : 0;
    const int kend = split ? min(K, kbeg + kchunk) : K;
    float acc[8][4];
    for (int j = 0; j < 8; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += 16) {
        unsigned a[4];
        a[0] = *reinterpret_cast<const unsigned *>(A + (m0 + g) * K + k0 + 2 * t);
        a[1] = *reinterpret_cast<const unsigned *>(A + (m0 + g + 8) * K + k0 + 2 * t);
        a[2] = *reinterpret_cast<const unsigned *>(A + (m0 + g) * K + k0 + 8 + 2 * t);
        a[3] = *reinterpret_cast<const unsigned *>(A + (m0 + g + 8) * K + k0 + 8 + 2 * t);
        for (int j = 0; j < 8; j++) {
            const __nv_bfloat16 *row = Bt + (long)(8 * j + g) * K + k0 + 2 * t;
            mma_bf16(acc[j], a, *reinterpret_cast<const unsigned *>(row),
                     *reinterpret_cast<const unsigned *>(row + 8));
        }
    }
    for (int j = 0; j < 8; j++) {
        float *c0 = C + (m0 + g) * NH + 8 * j + 2 * t;
        float *c1 = C + (m0 + g + 8) * NH + 8 * j + 2 * t;
        if (split) {
            atomicAdd(c0, acc[j][0]);
            atomicAdd(c0 + 1, acc[j][1]);
            atomicAdd(c1, acc[j][2]);
            atomicAdd(c1 + 1, acc[j][3]);
        } else {
            c0[0] = acc[j][0];
            c0[1] = acc[j][1];
            c1[0] = acc[j][2];
            c1[1] = acc[j][3];
        }
    }
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct TrainBufs {
    float *X, *T;             // batch features [B][5], targets [B]
    float *H1f;               // [B][64] tanh(z1)
    __nv_bfloat16 *H1, *H1T;  // [B][64], [64][B]
    float *Z2;                // [B][64]
    __nv_bfloat16 *DZ2, *DZ2T;
    float *DH1;               // [B][64]
    float *grad;              // [NPARAM]
    float *loss;              // [1]
};

// gather a batch (index permutation idx = (b*B + r) * P + off mod n) and layer 1
__global__ void __launch_bounds__(256)
k_train_l1(int B, long n, long first, long P, long off, const float *__restrict__ feats,
           const float *__restrict__ target, const MlpDev *__restrict__ w, TrainBufs tb)
{
    const int s = blockIdx.x * 256 + threadIdx.x;
    if (s >= B) return;
    const long idx = (long)(((unsigned long long)(first + s) * (unsigned long long)P + off) % n);
    float x[NIN];
    for (int f = 0; f < NIN; f++) {
        x[f] = feats[idx * NIN + f];
        tb.X[s * NIN + f] = x[f];
    }
    tb.T[s] = target[idx];
    for (int o = 0; o < NH; o++) {
        float z = w->b1[o];
        for (int f = 0; f < NIN; f++) z = fmaf(w->W1[o * NIN + f], x[f], z);
        float h = tanhf(z);
        tb.H1f[s * NH + o] = h;
        __nv_bfloat16 hb = __float2bfloat16_rn(h);
        tb.H1[s * NH + o] = hb;
        tb.H1T[(long)o * B + s] = hb;
    }
}

// output layer, loss and the gradients of w3, b3, b2; dz2 for the products.  The
// per-sample contributions are summed over each warp with shuffles first, so the
// block's shared accumulators take one atomic per warp instead of one per sample.
__global__ void __launch_bounds__(256)
k_train_out(int B, const MlpDev *__restrict__ w, TrainBufs tb)
{
    __shared__ float red[NH + NH + 2];
    for (int q = threadIdx.x; q < 2 * NH + 2; q += blockDim.x) red[q] = 0.f;
    __syncthreads();
    const int s = blockIdx.x * 256 + threadIdx.x;
    const bool act = s < B;
    const bool lead = (threadIdx.x & 31) == 0;
    float h2[NH];
    float y = w->b3;
    for (int o = 0; o < NH; o++) {
        h2[o] = act ? tanhf(tb.Z2[s * NH + o] + w->b2[o]) : 0.f;
        y = fmaf(w->w3[o], h2[o], y);
    }
    const float e = act ? y - tb.T[s] : 0.f;
    const float dy = 2.f * e / (float)B;
    const float se = warp_sum_f(e * e), sdy = warp_sum_f(dy);
    if (lead) {
        atomicAdd(&red[2 * NH], se);
        atomicAdd(&red[2 * NH + 1], sdy);
    }
    for (int o = 0; o < NH; o++) {
        const float dz = dy * w->w3[o] * (1.f - h2[o] * h2[o]);
        const float a = warp_sum_f(dy * h2[o]), b = warp_sum_f(dz);
        if (lead) {
            atomicAdd(&red[o], a);
            atomicAdd(&red[NH + o], b);
        }
        if (act) {
            __nv_bfloat16 db = __float2bfloat16_rn(dz);
            tb.DZ2[s * NH + o] = db;
            tb.DZ2T[(long)o * B + s] = db;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NH; q += blockDim.x) {
        atomicAdd(&tb.grad[O_W3 + q], red[q]);
        atomicAdd(&tb.grad[O_B2 + q], red[NH + q]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(tb.loss, red[2 * NH]);
        atomicAdd(&tb.grad[O_B3], red[2 * NH + 1]);
    }
}

// layer-1 gradients from dh1
__global__ void __launch_bounds__(256) k_train_back1(int B, TrainBufs tb)
{
    __shared__ float red[NH * NIN + NH];
    for (int q = threadIdx.x; q < NH * NIN + NH; q += blockDim.x) red[q] = 0.f;
    __syncthreads();
    const int s = blockIdx.x * 256 + threadIdx.x;
    const bool act = s < B;
    const bool lead = (threadIdx.x & 31) == 0;
    float x[NIN];
    for (int f = 0; f < NIN; f++) x[f] = act ? tb.X[s * NIN + f] : 0.f;
    for (int o = 0; o < NH; o++) {
        float dz = 0.f;
        if (act) {
            const float h = tb.H1f[s * NH + o];
            dz = tb.DH1[s * NH + o] * (1.f - h * h);
        }
        const float sb = warp_sum_f(dz);
        if (lead) atomicAdd(&red[NH * NIN + o], sb);
        for (int f = 0; f < NIN; f++) {
            const float sw = warp_sum_f(dz * x[f]);
            if (lead) atomicAdd(&red[o * NIN + f], sw);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NH * NIN; q += blockDim.x) atomicAdd(&tb.grad[O_W1 + q], red[q]);
    for (int q = threadIdx.x; q < NH; q += blockDim.x)
        atomicAdd(&tb.grad[O_B1 + q], red[NH * NIN + q]);
}

__global__ void k_adam(float *p, float *m, float *v, const float *gr, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    const float gq = gr[q];
    m[q] = b1 * m[q] + (1.f - b1) * gq;
    v[q] = b2 * v[q] + (1.f - b2) * gq * gq;
    p[q] -= lr * (m[q] / c1) / (sqrtf(v[q] / c2) + eps);
}

__global__ void k_accumulate(float *dst, const float *src) { *dst += *src; }

struct Trainer {
    int B;
    TrainBufs tb;
    MlpDev *w;
    float *p, *m, *v;
    std::vector<void *> allocs;
    cudaStream_t s;

    bool alloc(void **ptr, size_t bytes)
    {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        allocs.push_back(*ptr);
        return true;
    }
    bool init(int batch, cudaStream_t st)
    {
        B = batch;
        s = st;
        bool ok = alloc((void **)&tb.X, (size_t)B * NIN * 4) && alloc((void **)&tb.T, (size_t)B * 4) &&
                  alloc((void **)&tb.H1f, (size_t)B * NH * 4) && alloc((void **)&tb.H1, (size_t)B * NH * 2) &&
                  alloc((void **)&tb.H1T, (size_t)B * NH * 2) && alloc((void **)&tb.Z2, (size_t)B * NH * 4) &&
                  alloc((void **)&tb.DZ2, (size_t)B * NH * 2) && alloc((void **)&tb.DZ2T, (size_t)B * NH * 2) &&
                  alloc((void **)&tb.DH1, (size_t)B * NH * 4) && alloc((void **)&tb.grad, NPARAM * 4) &&
                  alloc((void **)&tb.loss, 4) && alloc((void **)&w, sizeof(MlpDev)) &&
                  alloc((void **)&p, NPARAM * 4) && alloc((void **)&m, NPARAM * 4) &&
                  alloc((void **)&v, NPARAM * 4);
        return ok;
    }
    ~Trainer()
    {
        for (void *q : allocs) cudaFree(q);
    }
    // one forward/backward pass over the batch starting at permuted index 'first'
    void grad(long n, long first, long P, long off, const float *feats, const float *target)
    {
        cudaMemsetAsync(tb.grad, 0, NPARAM * 4, s);
        cudaMemsetAsync(tb.loss, 0, 4, s);
        k_mlp_build<<<1, 256, 0, s>>>(p, w);
        const int nb = (B + 255) / 256;
        k_train_l1<<<nb, 256, 0, s>>>(B, n, first, P, off, feats, target, w, tb);
        k_gemm_bf16<<<B / 64, 128, 0, s>>>(B, NH, tb.H1, w->W2, tb.Z2);
        k_train_out<<<nb, 256, 0, s>>>(B, w, tb);
        const int kchunk = 256;
        k_gemm_bf16<<<dim3(1, (B + kchunk - 1) / kchunk), 128, 0, s>>>(NH, B, tb.DZ2T, tb.H1T,
                                                                      tb.grad + O_W2, kchunk);
        k_gemm_bf16<<<B / 64, 128, 0, s>>>(B, NH, tb.DZ2, w->W2T, tb.DH1);
        k_train_back1<<<nb, 256, 0, s>>>(B, tb);
    }
};

}  // namespace echo

using echo::MlpDev;
using echo::NPARAM;
using echo::Trainer;

namespace {
long coprime_step(long n)
{
    // a large odd step coprime to n, for the batch permutation
    long P = 2654435761L % n;
    if (P < 1) P = 1;
    auto gcd = [](long a, long b) {
        while (b) {
            long t = a % b;
            a = b;
            b = t;
        }
        return a;
    };
    while (gcd(P, n) != 1) P++;
    return P;
}
}  // namespace

extern "C" {

echo_status echo_mlp_load(echo_ctx *c, const float *weights, long n)
{
    if (!c || !weights) return ECHO_ERR_ARG;
    if (n != NPARAM) {
        echo::set_global_error("echo_mlp_load: expected 4609 parameters");
        return ECHO_ERR_ARG;
    }
    if (cudaSetDevice(c->cfg.device) != cudaSuccess) return ECHO_ERR_CUDA;
    if (!c->mlp_w && cudaMalloc(&c->mlp_w, sizeof(MlpDev)) != cudaSuccess) {
        c->mlp_w = nullptr;
        cudaGetLastError();
        return ECHO_ERR_OOM;
    }
    float *dp = nullptr;
    if (cudaMalloc((void **)&dp, NPARAM * sizeof(float)) != cudaSuccess) return ECHO_ERR_OOM;
    cudaMemcpyAsync(dp, weights, NPARAM * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    echo::k_mlp_build<<<1, 256, 0, c->stream>>>(dp, (MlpDev *)c->mlp_w);
    c->launches++;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(dp);
    // the persistent grid of the guess kernel of echo_mlp_guess; a captured step
    // graph holds the inversion kernel without the network and no longer matches
    c->mlp_blocks = c->mixed ? echo::Path<float>::mlp_grid(c) : echo::Path<double>::mlp_grid(c);
    echo::drop_step_graph(c);
    return e == cudaSuccess ? ECHO_OK : ECHO_ERR_CUDA;
}

echo_status echo_mlp_forward(const float *weights, const float *feats, long n, float *y,
                             void *stream)
{
    if (!weights || !feats || !y || n < 1) return ECHO_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float *dp = nullptr;
    MlpDev *w = nullptr;
    if (cudaMalloc((void **)&dp, NPARAM * 4) != cudaSuccess ||
        cudaMalloc((void **)&w, sizeof(MlpDev)) != cudaSuccess) {
        cudaGetLastError();
        if (dp) cudaFree(dp);
        return ECHO_ERR_OOM;
    }
    cudaMemcpyAsync(dp, weights, NPARAM * 4, cudaMemcpyHostToDevice, s);
    echo::k_mlp_build<<<1, 256, 0, s>>>(dp, w);
    echo::k_mlp_forward<<<(unsigned)((n + echo::MLP_BS - 1) / echo::MLP_BS), echo::MLP_BS, 0, s>>>(
        n, feats, w, y);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(dp);
    cudaFree(w);
    return e == cudaSuccess ? ECHO_OK : ECHO_ERR_CUDA;
}

echo_status echo_mlp_grad(const float *weights, const float *feats, const float *target, long n,
                          float *grad, float *loss, void *stream)
{
    if (!weights || !feats || !target || !grad || n < 64 || n % 64 || n > (1L << 24))
        return ECHO_ERR_ARG;
    Trainer tr;
    if (!tr.init((int)n, (cudaStream_t)stream)) return ECHO_ERR_OOM;
    cudaMemcpyAsync(tr.p, weights, NPARAM * 4, cudaMemcpyHostToDevice, tr.s);
    tr.grad(n, 0, 1, 0, feats, target);
    float l = 0.f;
    cudaMemcpyAsync(grad, tr.tb.grad, NPARAM * 4, cudaMemcpyDeviceToHost, tr.s);
    cudaMemcpyAsync(&l, tr.tb.loss, 4, cudaMemcpyDeviceToHost, tr.s);
    cudaError_t e = cudaStreamSynchronize(tr.s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (loss) *loss = l / (float)n;
    return e == cudaSuccess ? ECHO_OK : ECHO_ERR_CUDA;
}

echo_status echo_mlp_train(const float *feats, const float *target, long n,
                           const echo_train_cfg *cfg, float *weights, float *loss_hist,
                           void *stream)
{
    if (!feats || !target || !cfg || !weights || cfg->batch < 64 || cfg->batch % 64 ||
        cfg->epochs < 1 || n < cfg->batch)
        return ECHO_ERR_ARG;
    Trainer tr;
    if (!tr.init(cfg->batch, (cudaStream_t)stream)) return ECHO_ERR_OOM;
    cudaMemcpyAsync(tr.p, weights, NPARAM * 4, cudaMemcpyHostToDevice, tr.s);
    cudaMemsetAsync(tr.m, 0, NPARAM * 4, tr.s);
    cudaMemsetAsync(tr.v, 0, NPARAM * 4, tr.s);
    float *lsum = nullptr;
    if (cudaMalloc((void **)&lsum, sizeof(float) * cfg->epochs) != cudaSuccess) return ECHO_ERR_OOM;
    cudaMemsetAsync(lsum, 0, sizeof(float) * cfg->epochs, tr.s);
    const long P = coprime_step(n);
    const long nbatch = n / cfg->batch;
    long it = 0;
    for (int ep = 0; ep < cfg->epochs; ep++) {
        const long off = (long)(((unsigned long long)ep * 7919ULL + (unsigned long long)cfg->seed) % (unsigned long long)n);
        const float lr = (float)(cfg->lr * pow(cfg->lr_decay, ep));
        for (long b = 0; b < nbatch; b++) {
            tr.grad(n, b * cfg->batch, P, off, feats, target);
            it++;
            const float c1 = 1.f - powf((float)cfg->beta1, (float)it);
            const float c2 = 1.f - powf((float)cfg->beta2, (float)it);
            echo::k_adam<<<(NPARAM + 255) / 256, 256, 0, tr.s>>>(tr.p, tr.m, tr.v, tr.tb.grad, lr,
                                                                (float)cfg->beta1, (float)cfg->beta2,
                                                                (float)cfg->eps, c1, c2);
            // running loss sum of the epoch (device side)
            echo::k_accumulate<<<1, 1, 0, tr.s>>>(lsum + ep, tr.tb.loss);
        }
    }
    std::vector<float> hl(cfg->epochs);
    cudaMemcpyAsync(weights, tr.p, NPARAM * 4, cudaMemcpyDeviceToHost, tr.s);
    cudaMemcpyAsync(hl.data(), lsum, sizeof(float) * cfg->epochs, cudaMemcpyDeviceToHost, tr.s);
    cudaError_t e = cudaStreamSynchronize(tr.s);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(lsum);
    if (loss_hist)
        for (int ep = 0; ep < cfg->epochs; ep++)
            loss_hist[ep] = hl[ep] / (float)(nbatch * cfg->batch);
    return e == cudaSuccess ? ECHO_OK : ECHO_ERR_CUDA;
}

}  // extern "C"

namespace echo {

long launch_mlp_harvest(echo_ctx *c, long stride, long offset, float *feats, float *target,
                        long base, long capacity)
{
    const long m = (c->g.n - offset + stride - 1) / stride;
    if (m <= 0) return 0;
    if (base < capacity)
        launch(c, K_MISC, k_mlp_harvest, nblocks(m, 256), 256, 0, c->g, (const double *)c->U,
               (const double *)c->Bf, (const double *)c->W, stride, offset, feats, target, base,
               capacity);
    return m;
}

}  // namespace echo
