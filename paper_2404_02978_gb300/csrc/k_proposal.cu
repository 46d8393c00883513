// k_proposal.cu -- the learned frequency-sampling proposal (include/qrs_proposal.h):
// training targets from plain draws, the 6 -> 128 -> 128 -> C network's
// forward / backward passes, Adam, and the integer sampling CDF.  All FP32
// except where stated; every sum has a fixed order (deterministic) except the
// per-cell target histograms (shared-memory atomics).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/qrs_proposal.h"
#include "qrs_internal.h"

namespace qrs {

QRS_CHECK_HOOK(check_hook_proposal)

constexpr int kHid = 128;
constexpr uint32_t kStreamInit = 3u;  // Philox stream of the initial weights

__host__ __device__ inline int64_t mlp_params(int C) { return 6 * kHid + kHid + kHid * kHid + kHid + (int64_t)kHid * C + C; }

struct MlpView {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};

__host__ __device__ inline MlpView mlp_view(float* P, int C)
{
    MlpView v;
    v.W1 = P;
    v.b1 = v.W1 + 6 * kHid;
    v.W2 = v.b1 + kHid;
    v.b2 = v.W2 + kHid * kHid;
    v.W3 = v.b2 + kHid;
    v.b3 = v.W3 + (int64_t)kHid * C;
    return v;
}

// ------------------------------------------------------------------ init
__global__ void k_mlp_init(int C, uint64_t seed, float out_scale, float* __restrict__ P)
{
    const int64_t n = mlp_params(C);
    const int64_t e1 = 6 * kHid, e2 = e1 + kHid, e3 = e2 + kHid * kHid, e4 = e3 + kHid, e5 = e4 + (int64_t)kHid * C;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int fan = 0;
        if (i < e1) fan = 6;
        else if (i >= e2 && i < e3) fan = kHid;
        else if (i >= e4 && i < e5) fan = kHid;
        float v = 0.0f;
        if (fan) {
            const Words w = philox4x32_10((uint32_t)i, (uint32_t)((uint64_t)i >> 32), kStreamInit, 0u, (uint32_t)seed,
                                          (uint32_t)(seed >> 32));
            const float U1 = (float)((w.w0 >> 8) + 1u) * 0x1p-24f;
            const float U2 = (float)(w.w1 >> 8) * 0x1p-24f;
            v = sqrtf(-2.0f * logf(U1)) * cospif(2.0f * U2) * sqrtf(2.0f / (float)fan);
            if (i >= e4) v *= out_scale;  // the output layer's weights
        }
        *chk(P, i, n) = v;
    }
}

// -------------------------------------------------------------- features
__global__ void k_features(const double* __restrict__ geom, int64_t n, float* __restrict__ X)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double* g = chk(geom, 5 * i, 5 * n);
        const double B = hypot(g[3], g[4]);
        float* x = chk(X, 6 * i, 6 * n);
        x[0] = (float)((log(g[0]) - log(0.12)) / 0.6);
        x[1] = (float)((log(g[1]) - log(30.0)) / 0.8);
        x[2] = (float)((log(g[2]) - log(3.0)) / 0.6);
        x[3] = (float)((log(B) - log(15.0)) / 1.5);
        x[4] = (float)(g[3] / B);
        x[5] = (float)(g[4] / B);
    }
}

// ------------------------------------------------------------------ SGEMM
// C[M][N] = op(A) op(B) with op(A) [M][K] (A stored [M][K], or [K][M] if TA),
// op(B) [K][N] (B stored [K][N], or [N][K] if TB); epilogue: + bias[n],
// relu, multiply by (mask[m][n] > 0).  64 x 64 tiles, 16-deep K steps,
// 256 threads with 4 x 4 outputs each; ragged edges bounds-checked.
// epilogue: + bias[n], relu, multiply by (mask[m][n] > 0), + add[m][n] (the
// `mask` pointer carries the addend for kEpiAdd)
enum { kEpiNone = 0, kEpiBias = 1, kEpiRelu = 2, kEpiMask = 4, kEpiAdd = 8 };

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ Cm, int ldc,
                                               const float* __restrict__ bias, const float* __restrict__ mask, int ldm)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t nA = (int64_t)(TA ? K : M) * lda, nB = (int64_t)(TB ? N : K) * ldb;
    const int64_t nC = (int64_t)gridDim.z * M * ldc, nMask = (int64_t)M * ldm;
    float* const C0 = Cm;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float2 acc[4][2];  // acc[i][jp] = outputs (i, 2 jp), (i, 2 jp + 1): one FFMA2 updates both
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = make_float2(0.0f, 0.0f);
    const int kz0 = (int)(((int64_t)K * blockIdx.z) / gridDim.z), kz1 = (int)(((int64_t)K * (blockIdx.z + 1)) / gridDim.z);
    for (int k0 = kz0; k0 < kz1; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int mm, kk;
            if (TA) { kk = e >> 6; mm = e & 63; } else { mm = e >> 4; kk = e & 15; }
            const int gm = m0 + mm, gk = k0 + kk;
            el(As, kk, mm) = (gm < M && gk < kz1) ? *chk(A, TA ? (int64_t)gk * lda + gm : (int64_t)gm * lda + gk, nA) : 0.0f;
            int nn, kb;
            if (TB) { nn = e >> 4; kb = e & 15; } else { kb = e >> 6; nn = e & 63; }
            const int gn = n0 + nn, gkb = k0 + kb;
            el(Bs, kb, nn) = (gn < N && gkb < kz1) ? *chk(B, TB ? (int64_t)gn * ldb + gkb : (int64_t)gkb * ldb + gn, nB) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
            const float2 b01 = make_float2(Bs[kk][tx * 4 + 0], Bs[kk][tx * 4 + 1]);
            const float2 b23 = make_float2(Bs[kk][tx * 4 + 2], Bs[kk][tx * 4 + 3]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 ai = make_float2(a[i], a[i]);
                acc[i][0] = __ffma2_rn(ai, b01, acc[i][0]);
                acc[i][1] = __ffma2_rn(ai, b23, acc[i][1]);
            }
        }
        __syncthreads();
    }
    // split K (gridDim.z > 1): raw partial sums into slice z of Cm, [z][M][ldc]; the
    // epilogue then runs in k_sgemm_reduce
    if (gridDim.z > 1) Cm += (int64_t)blockIdx.z * M * ldc;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
            if (gridDim.z > 1) {
                *chk(C0, (Cm - C0) + (int64_t)m * ldc + n, nC) = v;
                continue;
            }
            if (EPI & kEpiBias) v += *chk(bias, n, N);
            if (EPI & kEpiRelu) v = fmaxf(v, 0.0f);
            if (EPI & kEpiMask) v = *chk(mask, (int64_t)m * ldm + n, nMask) > 0.0f ? v : 0.0f;
            if (EPI & kEpiAdd) v += *chk(mask, (int64_t)m * ldm + n, nMask);
            *chk(C0, (int64_t)m * ldc + n, nC) = v;
        }
    }
}

// Sum of the S split-K slices [S][M][ldc] in slice order (deterministic), then
// the epilogue (mask only: the split products have no bias or relu).
template <int EPI>
__global__ void k_sgemm_reduce(int M, int N, int S, const float* __restrict__ part, float* __restrict__ Cm, int ldc,
                               const float* __restrict__ mask, int ldm)
{
    const int64_t total = (int64_t)M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / N), n = (int)(e - (int64_t)m * N);
        const int64_t n_part = (int64_t)S * M * ldc;
        float v = *chk(part, (int64_t)m * ldc + n, n_part);
        for (int z = 1; z < S; ++z) v += *chk(part, ((int64_t)z * M + m) * ldc + n, n_part);
        if (EPI & kEpiMask) v = *chk(mask, (int64_t)m * ldm + n, (int64_t)M * ldm) > 0.0f ? v : 0.0f;
        *chk(Cm, (int64_t)m * ldc + n, (int64_t)M * ldc) = v;
    }
}

// split > 1: K in `split` slices, partials in `work` (split M ldc floats), then
// reduced in fixed order; for long K (the weight and input gradients: K = the
// sample count or the cell count) on small outputs, whose 64 x 64 tiles alone
// would not fill the GPU.
template <bool TA, bool TB, int EPI>
static cudaError_t sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                         const float* bias, const float* mask, int ldm, cudaStream_t s, int split = 1,
                         float* work = nullptr)
{
    if (split > 1 && work && !(EPI & (kEpiBias | kEpiRelu))) {  // split products carry no bias or relu
        dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), (unsigned)split);
        k_sgemm<TA, TB, kEpiNone><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, work, ldc, nullptr, nullptr, 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t total = (int64_t)M * N;
        k_sgemm_reduce<EPI><<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(M, N, split, work, C,
                                                                                                   ldc, mask, ldm);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    k_sgemm<TA, TB, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, ldm);
    return cudaGetLastError();
}

// Column sums out[c] = sum_r A[r][c] (the bias gradients), deterministic: thread
// (g, c) of a 8 x 32 block sums rows g, g + 8, ... of column c in order, then
// the 8 partials are added in order.
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ A, int rows, int cols, float* __restrict__ out)
{
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31), g = threadIdx.x >> 5;
    float v = 0.0f;
    if (c < cols)
        for (int r = g; r < rows; r += 8) v += *chk(A, (int64_t)r * cols + c, (int64_t)rows * cols);
    el(red, g, threadIdx.x & 31) = v;
    __syncthreads();
    if (g == 0 && c < cols) {
        float t = el(red, 0, threadIdx.x);
        for (int q = 1; q < 8; ++q) t += el(red, q, threadIdx.x);
        *chk(out, c, cols) = t;
    }
}

// ----------------------------------------------------- softmax cross entropy
__device__ __forceinline__ float block_reduce(float v, float* red, bool is_max)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmaxf(v, w) : v + w;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = lane < nw ? red[lane] : (is_max ? -INFINITY : 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmaxf(v, w) : v + w;
    }
    return v;
}

// One CTA per sample: dZ = (softmax(z) - t) / n, loss_row = sum_c t_c (lse - z_c).
__global__ void __launch_bounds__(256) k_softmax_ce(const float* __restrict__ Z, const float* __restrict__ T, int C,
                                                    int64_t n, float* __restrict__ dZ, float* __restrict__ loss_row)
{
    __shared__ float red[32];
    const int64_t i = blockIdx.x;
    const float* z = chk(Z, i * C, n * C);
    const float* t = chk(T, i * C, n * C);
    float mx = -INFINITY;
    for (int c = threadIdx.x; c < C; c += blockDim.x) mx = fmaxf(mx, z[c]);
    mx = block_reduce(mx, red, true);
    float se = 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) se += expf(z[c] - mx);
    se = block_reduce(se, red, false);
    const float lse = mx + logf(se);
    const float inv_n = 1.0f / (float)n;
    float l = 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const float q = expf(z[c] - lse);
        *chk(dZ, i * C + c, n * C) = (q - t[c]) * inv_n;
        l += t[c] * (lse - z[c]);
    }
    l = block_reduce(l, red, false);
    if (threadIdx.x == 0) *chk(loss_row, i, n) = l;
}

// Mean of loss_row in a fixed order (one CTA).
__global__ void k_loss_mean(const float* __restrict__ loss_row, int64_t n, float* __restrict__ loss)
{
    __shared__ float red[32];
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += *chk(loss_row, i, n);
    s = block_reduce(s, red, false);
    if (threadIdx.x == 0) *loss = s / (float)n;
}

// ------------------------------------------------------------------- Adam
__global__ void k_adam(int64_t n, float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = *chk(g, i, n);
        const float mi = 0.9f * *chk(m, i, n) + 0.1f * gi;
        const float vi = 0.999f * *chk(v, i, n) + 0.001f * gi * gi;
        *chk(m, i, n) = mi;
        *chk(v, i, n) = vi;
        *chk(P, i, n) -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
    }
}

// --------------------------------------------------------- training targets
// Plain log-polar draws: records (fx, fy, J, cell bits) of n_draws x n_f terms.
__global__ void k_prop_draws(DrawParams p, int n_draws, float4* __restrict__ rec)
{
    const int64_t total = (int64_t)n_draws * p.n_f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i % p.n_f;
        const Term t = draw_term(p, (uint64_t)i, k);
        *chk(rec, i, total) = make_float4(t.fx, t.fy, t.J, __int_as_float(t.cell));
    }
}

// One CTA per geometry: shared histogram of w A^2 2 (1 - cos 2 pi f.B) over the cells.
// fold_sh < 0: the draw's own cells (record .w).  fold_sh = 0, 1, 2: cells of the
// geometry's baseline frame over 2^fold_sh mirrored sectors: record k is stream
// point n = k, its R2 y coordinate Y = s0y + k step (0.64 turns); W = Y - frame
// with the baseline direction atan2(By, Bx) / 2 pi as a 0.64 fixed-point turn
// (FP64 x in (-1/2, 1/2], times 2^63, truncated, doubled mod 2^64); the top
// fold_sh bits of W are the sector, the rest (complemented in odd sectors)
// W' gives the angular cell ((W' >> 32) n_theta) >> 32; the radial band is
// the draw's own.
__global__ void __launch_bounds__(512) k_prop_targets(const float4* __restrict__ rec, int64_t n_rec, float inv_nf,
                                                      const double* __restrict__ geom, int psd_kind, double c_vk, int C,
                                                      int kind, int n_theta, int fold_sh, uint64_t s0y,
                                                      float* __restrict__ out)
{
    extern __shared__ float hist[];
    __shared__ float red[32];
    __shared__ float s_pc, s_pa, s_D, s_Bx, s_By;
    __shared__ unsigned long long s_frame;
    const int64_t i = blockIdx.x;
    if (threadIdx.x == 0) {
        const double* g = chk(geom, 5 * i, 5 * (int64_t)gridDim.x);
        s_pc = (float)(c_vk * pow(g[0], -5.0 / 3.0));
        s_pa = psd_kind == QRS_PSD_KOLMOGOROV ? 0.0f : (float)(1.0 / (g[1] * g[1]));
        s_D = (float)g[2];
        s_Bx = (float)g[3];
        s_By = (float)g[4];
        const double x = __ddiv_rn(atan2(g[4], g[3]), kTwoPi);
        s_frame = (unsigned long long)(long long)__dmul_rn(x, 0x1p63) * 2ull;
    }
    for (int c = threadIdx.x; c < C; c += blockDim.x) *chk(hist, c, C) = 0.0f;
    __syncthreads();
    const float pc = s_pc, pa = s_pa, D = s_D, Bx = s_Bx, By = s_By;
    for (int64_t k = threadIdx.x; k < n_rec; k += blockDim.x) {
        const float4 r = *chk(rec, k, n_rec);
        const float f2 = r.x * r.x + r.y * r.y;
        const float w = psd_w(pc, pa, f2) * r.z * inv_nf;
        const float A = airy_filter(sqrtf(f2), D, 0.0f);
        float s, c;
        sincos_turns(phase_df(r.x, r.y, Bx, By), s, c);
        const float v = w * A * A * 2.0f * (1.0f - c);
        int cell = __float_as_int(r.w);
        if (fold_sh >= 0) {
            uint64_t W = s0y + (uint64_t)k * kR2StepY - (uint64_t)s_frame;
            const uint64_t sec = fold_sh ? (W >> (64 - fold_sh)) : 0ull;
            W <<= fold_sh;
            if (sec & 1ull) W = ~W;
            cell = (cell / n_theta) * n_theta + (int)(((W >> 32) * (uint64_t)n_theta) >> 32);
        }
        atomicAdd(chk(hist, cell, C), kind == QRS_TARGET_RMS ? v * v : v);
    }
    __syncthreads();
    if (kind == QRS_TARGET_RMS)
        for (int c = threadIdx.x; c < C; c += blockDim.x) hist[c] = sqrtf(hist[c]);
    __syncthreads();
    float tot = 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) tot += hist[c];
    tot = block_reduce(tot, red, false);
    const float inv = tot > 0.0f ? 1.0f / tot : 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) *chk(out, i * C + c, (int64_t)gridDim.x * C) = hist[c] * inv;
}

// ------------------------------------------------------------ sampling CDF
// Integer widths floor(p (2^32 - n)) + 1 of a probability vector x[0..n) (FP64,
// stride `stride`), remainder to the largest (first on ties), exclusive scan
// into out[0..n).  Serial: n is a band count or a band's cell count.
__device__ void quantise_scan(const double* x, int n, int stride, double total, uint32_t* out)
{
    const double scale = 4294967296.0 - (double)n;
    unsigned long long sum = 0, best = 0;
    int arg = 0;
    for (int j = 0; j < n; ++j) {
        const unsigned long long w = (unsigned long long)floor(x[j * stride] / total * scale) + 1ull;
        sum += w;
        if (w > best) { best = w; arg = j; }
    }
    const unsigned long long rem = (1ull << 32) - sum;
    unsigned long long run = 0;
    for (int j = 0; j < n; ++j) {
        out[j] = (uint32_t)run;
        run += (unsigned long long)floor(x[j * stride] / total * scale) + 1ull + (j == arg ? rem : 0ull);
    }
}

// One CTA: p = (1 - eps) softmax(z) + eps / C in FP64 (FP32 exponentials),
// band sums, the marginal CDF (thread 0), the conditional CDFs (one thread
// per band).  pbuf: C + n_rho doubles of workspace.
__global__ void __launch_bounds__(1024) k_prop_cdf(const float* __restrict__ z, int n_rho, int n_theta, float eps,
                                                   float beta, uint32_t* __restrict__ cdf, double* __restrict__ pbuf)
{
    __shared__ float redf[32];
    __shared__ double redd[32];
    const int C = n_rho * n_theta;
    float mx = -INFINITY;
    for (int c = threadIdx.x; c < C; c += blockDim.x) mx = fmaxf(mx, z[c]);
    mx = block_reduce(mx, redf, true);
    double se = 0.0;
    for (int c = threadIdx.x; c < C; c += blockDim.x) se += (double)expf(beta * (z[c] - mx));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) redd[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += redd[q];
        redd[0] = t;
    }
    __syncthreads();
    const double sum = redd[0];
    for (int c = threadIdx.x; c < C; c += blockDim.x)
        *chk(pbuf, c, (int64_t)C + n_rho) = (1.0 - (double)eps) * ((double)expf(beta * (z[c] - mx)) / sum) + (double)eps / (double)C;
    __syncthreads();
    double* band = pbuf + C;
    for (int i = threadIdx.x; i < n_rho; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n_theta; ++j) s += *chk(pbuf, (int64_t)i * n_theta + j, (int64_t)C);
        *chk(band, i, n_rho) = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n_rho; ++i) t += band[i];
        if (chk_ok(0, n_rho, (int64_t)n_rho + C)) quantise_scan(band, n_rho, 1, t, cdf);
    }
    for (int i = threadIdx.x; i < n_rho; i += blockDim.x)
        if (chk_ok(n_rho + (int64_t)i * n_theta, n_theta, (int64_t)n_rho + C))
            quantise_scan(pbuf + i * n_theta, n_theta, 1, band[i], cdf + n_rho + (int64_t)i * n_theta);
}

static double vk_c()
{
    const double pi = 3.14159265358979323846;
    return std::tgamma(11.0 / 6.0) * std::tgamma(11.0 / 6.0) / (2.0 * std::pow(pi, 11.0 / 3.0)) *
           std::pow(24.0 / 5.0 * std::tgamma(6.0 / 5.0), 5.0 / 6.0);
}

// ------------------------------------------------------------------ prior
// One CTA per geometry: per importance cell the mean over kPriorNodes points
// of g = W(rho) A(pi D rho)^2 (1 - cos(2 pi rho |B| cos phi)) rho^2, the cell's
// share of the differential-piston structure function at B up to a constant
// (Sec. 4.4 with the Eq. 7 filter); then log(v / max v), floored at kPriorFloor.
// Node m sits at (u, t) = ((i_rho + s_x) / n_rho, (i_theta + s_y) / n_theta),
// (s_x, s_y) point m of the R2 sequence of Eq. 6 from (1/2, 1/2) (0.64 fixed
// point, top 24 bits); rho = fmin (fmax/fmin)^u; phi = 2 pi t / fold (the
// sector of the baseline frame; mirror images hold the same values) or
// 2 pi t - atan2(By, Bx) for fold 0.  The phase rho |B| cos phi is reduced to
// [-1/2, 1/2] turn, and 1 - cos is taken as 2 sin^2 (no cancellation where the
// phase is small).
constexpr int kPriorNodes = 64;
constexpr float kPriorFloor = -60.0f;

__global__ void __launch_bounds__(256) k_prop_prior(const double* __restrict__ geom, int psd_kind, double c_vk,
                                                    float fmin, float l2, int n_rho, int n_theta, int fold,
                                                    float* __restrict__ out)
{
    __shared__ float s_node[kPriorNodes][2];
    __shared__ float red[32];
    __shared__ float s_pc, s_pa, s_D, s_B, s_phiB;
    if (threadIdx.x < kPriorNodes) {
        const uint64_t m = threadIdx.x;
        el(s_node, m, 0) = (float)((0x8000000000000000ULL + m * kR2StepX) >> 40) * 0x1p-24f;
        el(s_node, m, 1) = (float)((0x8000000000000000ULL + m * kR2StepY) >> 40) * 0x1p-24f;
    }
    if (threadIdx.x == 0) {
        const double* g = chk(geom, 5 * (int64_t)blockIdx.x, 5 * (int64_t)gridDim.x);
        s_pc = (float)(c_vk * pow(g[0], -5.0 / 3.0));
        s_pa = psd_kind == kPsdKolmogorov ? 0.0f : (float)(1.0 / (g[1] * g[1]));
        s_D = (float)g[2];
        s_B = (float)hypot(g[3], g[4]);
        s_phiB = (float)atan2(g[4], g[3]);
    }
    __syncthreads();
    const int C = n_rho * n_theta;
    const int64_t o0 = (int64_t)blockIdx.x * C, n_out = (int64_t)gridDim.x * C;
    const float pc = s_pc, pa = s_pa, D = s_D, B = s_B, phiB = s_phiB;
    const float dphi = fold ? 6.28318530717958648f / (float)fold : 6.28318530717958648f;
    float vmax = 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const int ir = c / n_theta, it = c - ir * n_theta;
        float v = 0.0f;
        for (int m = 0; m < kPriorNodes; ++m) {
            const float u = ((float)ir + s_node[m][0]) / (float)n_rho;
            const float t = ((float)it + s_node[m][1]) / (float)n_theta;
            const float rho = fmin * exp2f(u * l2);
            const float phi = fold ? t * dphi : t * dphi - phiB;
            const float A = airy_g(3.14159265358979f * D * rho);
            const float ph = rho * B * __cosf(phi);
            const float sn = sinpif(ph - rintf(ph));  // 1 - cos 2 pi ph = 2 sin^2 pi ph, without cancellation
            v += psd_w(pc, pa, rho * rho) * A * A * (2.0f * sn * sn) * rho * rho;
        }
        v *= 1.0f / (float)kPriorNodes;
        *chk(out, o0 + c, n_out) = v;
        vmax = fmaxf(vmax, v);
    }
    vmax = block_reduce(vmax, red, true);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const float v = *chk(out, o0 + c, n_out);
        *chk(out, o0 + c, n_out) = v > 0.0f && vmax > 0.0f ? fmaxf(logf(v / vmax), kPriorFloor) : kPriorFloor;
    }
}

// Forward pass into workspace (X, H1, H2) and Z (+ prior [n][C] when non-NULL).
static cudaError_t mlp_forward(int C, const float* P, const double* geom, int64_t n, float* X, float* H1, float* H2,
                               float* Z, cudaStream_t s, const float* prior = nullptr)
{
    MlpView w = mlp_view(const_cast<float*>(P), C);
    const int N = (int)n;
    k_features<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(geom, n, X);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = sgemm<false, false, kEpiBias | kEpiRelu>(N, kHid, 6, X, 6, w.W1, kHid, H1, kHid, w.b1, nullptr, 0, s);
    if (e == cudaSuccess) e = sgemm<false, false, kEpiBias | kEpiRelu>(N, kHid, kHid, H1, kHid, w.W2, kHid, H2, kHid, w.b2, nullptr, 0, s);
    if (e == cudaSuccess) {
        if (prior) e = sgemm<false, false, kEpiBias | kEpiAdd>(N, C, kHid, H2, kHid, w.W3, C, Z, C, w.b3, prior, C, s);
        else e = sgemm<false, false, kEpiBias>(N, C, kHid, H2, kHid, w.W3, C, Z, C, w.b3, nullptr, 0, s);
    }
    return e;
}

constexpr int kMaxSplit = 8;  // K slices of the long-K gradient products

// Slices for a long-K product: enough 64 x 64 tiles for about two per SM on a
// 152-SM part, at most kMaxSplit, each slice at least 128 deep.
static int split_for(int M, int N, int K)
{
    const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
    int sp = (304 + tiles - 1) / tiles;
    sp = std::min(sp, kMaxSplit);
    sp = std::min(sp, std::max(1, K / 128));
    return std::max(sp, 1);
}

static size_t mlp_ws_floats(int C, int64_t n)
{
    return (size_t)n * (8 + 4 * kHid + 2 * (size_t)C + 2) + 64 +
           (size_t)kMaxSplit * std::max((size_t)kHid * (size_t)C, (size_t)n * kHid) + 64;
}

// The loss and its gradient (the launches of qrs_mlp_loss_grad) with the
// workspace at ws (mlp_ws_floats(C, n) floats); *launches counts the kernels.
static cudaError_t mlp_loss_grad(int C, const float* params, const double* geom, const float* targets, int64_t n,
                                 float* grad, float* loss, float* ws, cudaStream_t s, int* launches_out,
                                 const float* prior)
{
    float* X = ws;
    float* H1 = X + 8 * n;
    float* H2 = H1 + kHid * n;
    float* dA2 = H2 + kHid * n;
    float* dA1 = dA2 + kHid * n;
    float* Z = dA1 + kHid * n;
    float* dZ = Z + (int64_t)C * n;
    float* lrow = dZ + (int64_t)C * n + n;  // (n floats after dZ unused)
    float* part = reinterpret_cast<float*>(((uintptr_t)(lrow + n) + 255) & ~(uintptr_t)255);  // split-K slices
    MlpView w = mlp_view(const_cast<float*>(params), C);
    MlpView g = mlp_view(grad, C);
    const int N = (int)n;
    cudaError_t e = mlp_forward(C, params, geom, n, X, H1, H2, Z, s, prior);
    if (e == cudaSuccess) {
        k_softmax_ce<<<(unsigned)n, 256, 0, s>>>(Z, targets, C, n, dZ, lrow);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_loss_mean<<<1, 1024, 0, s>>>(lrow, n, loss);
        e = cudaGetLastError();
    }
    int launches = 4 + 2;
    auto colsum = [&](const float* A, int cols, float* out) {
        k_colsum<<<(unsigned)((cols + 31) / 32), 256, 0, s>>>(A, N, cols, out);
        ++launches;
        return cudaGetLastError();
    };
    auto gemm_launches = [&](int sp) { launches += sp > 1 ? 2 : 1; };
    // layer 3: dW3 = H2^T dZ, db3 = column sums of dZ, dA2 = (dZ W3^T) * (H2 > 0)
    int sp = split_for(kHid, C, N);
    if (e == cudaSuccess) e = sgemm<true, false, kEpiNone>(kHid, C, N, H2, kHid, dZ, C, g.W3, C, nullptr, nullptr, 0, s, sp, part);
    gemm_launches(sp);
    if (e == cudaSuccess) e = colsum(dZ, C, g.b3);
    sp = split_for(N, kHid, C);
    if (e == cudaSuccess) e = sgemm<false, true, kEpiMask>(N, kHid, C, dZ, C, w.W3, C, dA2, kHid, nullptr, H2, kHid, s, sp, part);
    gemm_launches(sp);
    // layer 2
    sp = split_for(kHid, kHid, N);
    if (e == cudaSuccess) e = sgemm<true, false, kEpiNone>(kHid, kHid, N, H1, kHid, dA2, kHid, g.W2, kHid, nullptr, nullptr, 0, s, sp, part);
    gemm_launches(sp);
    if (e == cudaSuccess) e = colsum(dA2, kHid, g.b2);
    if (e == cudaSuccess) e = sgemm<false, true, kEpiMask>(N, kHid, kHid, dA2, kHid, w.W2, kHid, dA1, kHid, nullptr, H1, kHid, s);
    gemm_launches(1);
    // layer 1
    sp = split_for(6, kHid, N);
    if (e == cudaSuccess) e = sgemm<true, false, kEpiNone>(6, kHid, N, X, 6, dA1, kHid, g.W1, kHid, nullptr, nullptr, 0, s, sp, part);
    gemm_launches(sp);
    if (e == cudaSuccess) e = colsum(dA1, kHid, g.b1);
    *launches_out = launches;
    return e;
}

// Adam's bias corrections 1 / (1 - beta^t) for step t.
static void adam_corrections(int64_t step, float* c1, float* c2)
{
    *c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)step)));
    *c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)step)));
}

static cudaError_t launch_adam(int C, float* params, float* m, float* v, const float* grad, float lr, int64_t step,
                               cudaStream_t s)
{
    const int64_t n = mlp_params(C);
    float c1, c2;
    adam_corrections(step, &c1, &c2);
    k_adam<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(n, params, m, v, grad, lr, c1, c2);
    return cudaGetLastError();
}

}  // namespace qrs

using namespace qrs;

extern "C" {

int64_t qrs_mlp_param_count(int32_t n_cells) { return n_cells >= 1 ? mlp_params(n_cells) : 0; }

// Cell counts the proposal kernels take: the targets kernel holds one FP32
// histogram bin per cell in shared memory (128 KB at the limit).
constexpr int64_t kMaxCells = 32768;
static bool cells_ok(int64_t C) { return C >= 1 && C <= kMaxCells; }

qrs_status qrs_mlp_init(qrs_handle* h, int32_t n_cells, uint64_t seed, float out_scale, float* params, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_mlp_init");
    if (qrs::injected_launch_fault(h, "qrs_mlp_init") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (!cells_ok(n_cells) || !params) return fail(h, QRS_ERR_ARG, "n_cells must be in [1, 32768] and params non-NULL");
    if (!(std::isfinite(out_scale) && out_scale >= 0.0f)) return fail(h, QRS_ERR_ARG, "out_scale must be finite and >= 0");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) {
        k_mlp_init<<<256, 256, 0, (cudaStream_t)stream>>>(n_cells, seed, out_scale, params);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_mlp_init");
    ++h->launches;
    return QRS_OK;
}

qrs_status qrs_proposal_targets(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, int32_t n_rho,
                                int32_t n_theta, uint64_t seed, int64_t n_f, int32_t n_draws, int32_t kind,
                                int32_t fold, const double* geom, int64_t n, float* targets, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_proposal_targets");
    if (qrs::injected_launch_fault(h, "qrs_proposal_targets") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (kind != QRS_TARGET_MEAN && kind != QRS_TARGET_RMS) return fail(h, QRS_ERR_ARG, "unknown target kind %d", kind);
    if (fold != 0 && fold != 1 && fold != 2 && fold != 4) return fail(h, QRS_ERR_ARG, "fold must be 0, 1, 2 or 4");
    if (!dom || dom->kind != QRS_DOMAIN_LOGPOLAR) return fail(h, QRS_ERR_ARG, "targets need a LOGPOLAR domain");
    if (n_draws < 1 || n < 0) return fail(h, QRS_ERR_ARG, "n_draws >= 1, n >= 0");
    const int64_t C = (int64_t)n_rho * n_theta;
    if (n_rho < 1 || n_theta < 1 || !cells_ok(C)) return fail(h, QRS_ERR_ARG, "n_rho x n_theta in [1, 32768]");
    qrs_sampler smp;
    memset(&smp, 0, sizeof(smp));
    smp.seed = seed;
    smp.kind = QRS_SAMPLER_R2;
    smp.coef_kind = QRS_COEF_GAUSS;
    smp.n_rho = n_rho;
    smp.n_theta = n_theta;
    DrawParams p;
    if (psd && psd->ap_D_m > 0.0)
        return fail(h, QRS_ERR_ARG, "targets apply each geometry's aperture filter: the PSD's filter must be off");
    qrs_status st = make_draw_params(h, psd, dom, &smp, n_f, 0, &p);
    if (st != QRS_OK) return st;
    if (n == 0) return QRS_OK;
    if (!geom || !targets) return fail(h, QRS_ERR_ARG, "geom and targets must be non-NULL");
    const int64_t n_rec = (int64_t)n_draws * n_f;
    st = ensure_work(h, (size_t)n_rec * sizeof(float4) + 256);
    if (st != QRS_OK) return st;
    float4* rec = reinterpret_cast<float4*>(((uintptr_t)h->d_work + 255) & ~(uintptr_t)255);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) {
        k_prop_draws<<<(unsigned)std::min<int64_t>((n_rec + 255) / 256, 8192), 256, 0, s>>>(p, n_draws, rec);
        e = cudaGetLastError();
    }
    // the histogram is dynamic shared memory beside the kernel's static arrays: the opt-in
    // limit is raised whatever C is (the default 48 KB covers the sum only for small C)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prop_targets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(C * sizeof(float)));
    if (e == cudaSuccess) {
        k_prop_targets<<<(unsigned)n, 512, (size_t)C * sizeof(float), s>>>(rec, n_rec, p.inv_nf, geom, psd->kind, vk_c(),
                                                                          (int)C, kind, n_theta,
                                                                          fold == 0 ? -1 : fold == 4 ? 2 : fold - 1,
                                                                          p.s0y, targets);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_proposal_targets");
    h->launches += 2;
    return QRS_OK;
}

qrs_status qrs_proposal_prior(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, int32_t n_rho,
                              int32_t n_theta, int32_t fold, const double* geom, int64_t n, float* prior, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_proposal_prior");
    if (qrs::injected_launch_fault(h, "qrs_proposal_prior") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (fold != 0 && fold != 1 && fold != 2 && fold != 4) return fail(h, QRS_ERR_ARG, "fold must be 0, 1, 2 or 4");
    if (!psd || (psd->kind != QRS_PSD_VON_KARMAN && psd->kind != QRS_PSD_KOLMOGOROV))
        return fail(h, QRS_ERR_ARG, "psd must be non-NULL with a known kind");
    if (!dom || dom->kind != QRS_DOMAIN_LOGPOLAR || !(dom->fmin > 0.0 && dom->fmax > dom->fmin && std::isfinite(dom->fmax)))
        return fail(h, QRS_ERR_ARG, "the prior needs a LOGPOLAR domain with 0 < fmin < fmax");
    const int64_t C = (int64_t)n_rho * n_theta;
    if (n_rho < 1 || n_theta < 1 || !cells_ok(C) || n < 0 || n > (1 << 24))
        return fail(h, QRS_ERR_ARG, "n_rho x n_theta in [1, 32768], n in [0, 2^24]");
    if (n == 0) return QRS_OK;
    if (!geom || !prior) return fail(h, QRS_ERR_ARG, "geom and prior must be non-NULL");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) {
        k_prop_prior<<<(unsigned)n, 256, 0, (cudaStream_t)stream>>>(geom, psd->kind, vk_c(), (float)dom->fmin,
                                                                    (float)std::log2(dom->fmax / dom->fmin), n_rho,
                                                                    n_theta, fold, prior);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_proposal_prior");
    ++h->launches;
    return QRS_OK;
}

qrs_status qrs_mlp_forward(qrs_handle* h, int32_t n_cells, const float* params, const double* geom,
                           const float* prior, int64_t n, float* logits, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_mlp_forward");
    if (qrs::injected_launch_fault(h, "qrs_mlp_forward") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (!cells_ok(n_cells) || n < 0 || n > (1 << 24)) return fail(h, QRS_ERR_ARG, "n_cells in [1, 32768], n in [0, 2^24]");
    if (n == 0) return QRS_OK;
    if (!params || !geom || !logits) return fail(h, QRS_ERR_ARG, "params, geom and logits must be non-NULL");
    qrs_status st = ensure_work(h, mlp_ws_floats(n_cells, n) * sizeof(float));
    if (st != QRS_OK) return st;
    float* X = static_cast<float*>(h->d_work);
    float* H1 = X + 8 * n;
    float* H2 = H1 + kHid * n;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = mlp_forward(n_cells, params, geom, n, X, H1, H2, logits, (cudaStream_t)stream, prior);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_mlp_forward");
    h->launches += 4;
    return QRS_OK;
}

qrs_status qrs_mlp_loss_grad(qrs_handle* h, int32_t n_cells, const float* params, const double* geom,
                             const float* prior, const float* targets, int64_t n, float* grad, float* loss,
                             void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_mlp_loss_grad");
    if (qrs::injected_launch_fault(h, "qrs_mlp_loss_grad") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (!cells_ok(n_cells) || n < 1 || n > (1 << 24)) return fail(h, QRS_ERR_ARG, "n_cells in [1, 32768], n in [1, 2^24]");
    if (!params || !geom || !targets || !grad || !loss) return fail(h, QRS_ERR_ARG, "null pointer argument");
    qrs_status st = ensure_work(h, mlp_ws_floats(n_cells, n) * sizeof(float));
    if (st != QRS_OK) return st;
    int launches = 0;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess)
        e = mlp_loss_grad(n_cells, params, geom, targets, n, grad, loss, static_cast<float*>(h->d_work),
                          (cudaStream_t)stream, &launches, prior);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_mlp_loss_grad");
    h->launches += launches;
    return QRS_OK;
}

qrs_status qrs_mlp_adam(qrs_handle* h, int32_t n_cells, float* params, float* m, float* v, const float* grad, float lr,
                        int64_t step, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_mlp_adam");
    if (qrs::injected_launch_fault(h, "qrs_mlp_adam") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (!cells_ok(n_cells) || step < 1 || !(lr > 0.0f)) return fail(h, QRS_ERR_ARG, "n_cells, step >= 1, lr > 0");
    if (!params || !m || !v || !grad) return fail(h, QRS_ERR_ARG, "null pointer argument");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = launch_adam(n_cells, params, m, v, grad, lr, step, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_mlp_adam");
    ++h->launches;
    return QRS_OK;
}

qrs_status qrs_proposal_train(qrs_handle* h, qrs_mlp_state* state, const double* geom, const float* prior,
                              const float* targets, int64_t n, int64_t steps, double lr, int32_t schedule,
                              int64_t total_steps, float* loss_trace, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_proposal_train");
    if (qrs::injected_launch_fault(h, "qrs_proposal_train") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (!state) return fail(h, QRS_ERR_ARG, "state must be non-NULL");
    const int C = state->n_cells;
    if (!cells_ok(C) || n < 1 || n > (1 << 24)) return fail(h, QRS_ERR_ARG, "n_cells in [1, 32768], n in [1, 2^24]");
    if (!state->params || !state->m || !state->v || !geom || !targets)
        return fail(h, QRS_ERR_ARG, "state vectors, geom and targets must be non-NULL");
    if (state->step < 0 || steps < 0 || steps > ((int64_t)1 << 40))
        return fail(h, QRS_ERR_ARG, "state->step >= 0 and steps in [0, 2^40]");
    if (!(std::isfinite(lr) && lr > 0.0)) return fail(h, QRS_ERR_ARG, "lr must be finite and > 0");
    if (schedule != QRS_LR_CONSTANT && schedule != QRS_LR_COSINE) return fail(h, QRS_ERR_ARG, "unknown schedule %d", schedule);
    const int64_t last = state->step + steps;
    if (schedule == QRS_LR_COSINE && total_steps < last)
        return fail(h, QRS_ERR_ARG, "the cosine schedule needs total_steps >= state->step + steps");
    if (steps == 0) return QRS_OK;
    // workspace: the loss-gradient buffers, the gradient, one loss slot
    const size_t ws = (mlp_ws_floats(C, n) * sizeof(float) + 255) & ~(size_t)255;
    const size_t gb = ((size_t)mlp_params(C) * sizeof(float) + 255) & ~(size_t)255;
    qrs_status st = ensure_work(h, ws + gb + 256 + 256);
    if (st != QRS_OK) return st;
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)h->d_work + 255) & ~(uintptr_t)255);
    float* wsp = reinterpret_cast<float*>(base);
    float* grad = reinterpret_cast<float*>(base + ws);
    float* loss_slot = reinterpret_cast<float*>(base + ws + gb);
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    int64_t launches = 0;
    const double kPiD = 3.14159265358979323846;
    for (int64_t t = state->step + 1; t <= last && e == cudaSuccess; ++t) {
        // the learning rate of step t in FP64, rounded once to FP32
        const double lr_t = schedule == QRS_LR_COSINE
                                ? lr * 0.5 * (1.0 + std::cos(kPiD * (double)(t - 1) / (double)total_steps))
                                : lr;
        float* loss = loss_trace ? loss_trace + (t - state->step - 1) : loss_slot;
        int l = 0;
        e = mlp_loss_grad(C, state->params, geom, targets, n, grad, loss, wsp, s, &l, prior);
        if (e == cudaSuccess) e = launch_adam(C, state->params, state->m, state->v, grad, (float)lr_t, t, s);
        launches += l + 1;
    }
    h->launches += launches;
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_proposal_train");
    state->step = last;
    return QRS_OK;
}

// Checkpoint file: the 8 bytes "QRSMLP01", int32 n_cells, int32 0, int64 step,
// int64 parameter count, then params, m, v as FP32 (host byte order, little
// endian on every supported host).
static const char kCkptMagic[8] = {'Q', 'R', 'S', 'M', 'L', 'P', '0', '1'};

qrs_status qrs_mlp_save(qrs_handle* h, const qrs_mlp_state* state, const char* path, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    h->last_error.clear();
    if (!state || !path || !cells_ok(state->n_cells) || !state->params || !state->m || !state->v || state->step < 0)
        return fail(h, QRS_ERR_ARG, "state (n_cells in [1, 32768], vectors, step >= 0) and path must be valid");
    const int64_t P = mlp_params(state->n_cells);
    std::vector<float> buf((size_t)(3 * P));
    cudaError_t e = cudaSetDevice(h->device);
    const float* src[3] = {state->params, state->m, state->v};
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(buf.data() + i * P, src[i], (size_t)P * sizeof(float), cudaMemcpyDeviceToHost,
                            (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_mlp_save");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(h, QRS_ERR_ARG, "cannot open %s for writing", path);
    const int32_t hdr32[2] = {state->n_cells, 0};
    const int64_t hdr64[2] = {state->step, P};
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(hdr32, sizeof(hdr32), 1, f) == 1 &&
              std::fwrite(hdr64, sizeof(hdr64), 1, f) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(h, QRS_ERR_ARG, "writing %s failed", path);
    return QRS_OK;
}

qrs_status qrs_mlp_load(qrs_handle* h, qrs_mlp_state* state, const char* path, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    h->last_error.clear();
    if (!state || !path || !cells_ok(state->n_cells) || !state->params || !state->m || !state->v)
        return fail(h, QRS_ERR_ARG, "state (n_cells in [1, 32768], vectors) and path must be valid");
    const int64_t P = mlp_params(state->n_cells);
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(h, QRS_ERR_ARG, "cannot open %s", path);
    char magic[8];
    int32_t hdr32[2];
    int64_t hdr64[2];
    std::vector<float> buf((size_t)(3 * P));
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
              std::fread(hdr32, sizeof(hdr32), 1, f) == 1 && std::fread(hdr64, sizeof(hdr64), 1, f) == 1;
    if (ok && (hdr32[0] != state->n_cells || hdr64[1] != P || hdr64[0] < 0)) {
        std::fclose(f);
        return fail(h, QRS_ERR_ARG, "%s holds a network of %d cells, not %d", path, (int)hdr32[0], (int)state->n_cells);
    }
    ok = ok && std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return fail(h, QRS_ERR_ARG, "%s is not a complete checkpoint", path);
    cudaError_t e = cudaSetDevice(h->device);
    float* dst[3] = {state->params, state->m, state->v};
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(dst[i], buf.data() + i * P, (size_t)P * sizeof(float), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);  // buf is released on return
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_mlp_load");
    state->step = hdr64[0];
    return QRS_OK;
}

qrs_status qrs_proposal_cdf(qrs_handle* h, int32_t n_rho, int32_t n_theta, const float* logits, float eps,
                            float beta, uint32_t* cdf, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_proposal_cdf");
    if (qrs::injected_launch_fault(h, "qrs_proposal_cdf") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    const int64_t C = (int64_t)n_rho * n_theta;
    if (n_rho < 1 || n_theta < 1 || !cells_ok(C) || !(eps > 0.0f && eps <= 1.0f))
        return fail(h, QRS_ERR_ARG, "n_rho x n_theta in [1, 32768], 0 < eps <= 1");
    if (!(beta > 0.0f && beta <= 16.0f)) return fail(h, QRS_ERR_ARG, "0 < beta <= 16");
    if (!logits || !cdf) return fail(h, QRS_ERR_ARG, "logits and cdf must be non-NULL");
    qrs_status st = ensure_work(h, (size_t)(C + n_rho) * sizeof(double) + 256);
    if (st != QRS_OK) return st;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) {
        k_prop_cdf<<<1, 1024, 0, (cudaStream_t)stream>>>(logits, n_rho, n_theta, eps, beta, cdf,
                                                         static_cast<double*>(h->d_work));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_proposal_cdf");
    ++h->launches;
    return QRS_OK;
}

}  // extern "C"
