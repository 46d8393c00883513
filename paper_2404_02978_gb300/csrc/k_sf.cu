// k_sf.cu -- K5: FP64 structure-function sums (Sec. 4.4), and the pair
// differences of synthesised values they are usually taken of.
// For every (series s, lag L): x = v[t+L] - v[t] (L >= 1) or x = v[t] (L = 0),
// summed over realisations and t as (sum x^2, sum x^4, count): per thread in
// double-float on the FP32 pipe (below), across threads and blocks in FP64.
// Grid: y = series-lag pair, x = slices of the flat (realisation, t) range.
// Each thread keeps FP64 partial sums, the block reduces them with warp
// shuffles, and one thread per block adds them to acc with FP64 atomics.
#include "qrs_internal.h"

namespace qrs {

QRS_CHECK_HOOK(check_hook_sf)

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-thread sums in double-float (hi + lo FP32 pairs, qrs_device.cuh) on the
// FP32 pipe, whose rate is 64 times the FP64 pipe's on this part: x = v1 - v0
// exactly by two-sum, x^2 and x^4 by the FMA-based exact product, sums by
// df_add (about 48 significant bits each step); a thread's partials go to FP64
// at the end.  Values of magnitude 1e9 or more (whose fourth power would leave
// the FP32 range), and NaN, are summed in FP64 instead.
__global__ void __launch_bounds__(256) k_structure_fn(const float* __restrict__ delta, int64_t n_real, int64_t n_series,
                                                      int64_t T, const int32_t* __restrict__ lags, int32_t n_lags,
                                                      double* __restrict__ acc, int* __restrict__ err)
{
    const int64_t n_pairs = n_series * (int64_t)n_lags;
    __shared__ double red[3][8];
    for (int64_t pair = blockIdx.y; pair < n_pairs; pair += gridDim.y) {  // uniform per block
        const int64_t s = pair / n_lags;
        const int l = (int)(pair - s * n_lags);
        const int64_t L = *chk(lags, l, n_lags);
        if (L < 0 || L >= T) {
            if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(err, (int)QRS_ERR_DEVICE_CHECK);
            continue;
        }
        const int64_t per = (L == 0) ? T : T - L;  // values per (realisation, series)
        const int64_t total = n_real * per;
        // the flat index i = r per + t advances by the grid stride: (r, t) are
        // carried along (one division per thread, not per value)
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const int64_t dq = stride / per, dr = stride - dq * per;
        int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        int64_t r = i / per, t = i - r * per;
        DF a2 = {0.0f, 0.0f}, a4 = {0.0f, 0.0f};
        double b2 = 0.0, b4 = 0.0;  // values too large for the FP32 fourth power
        int64_t n = 0;
        for (; i < total; i += stride) {
            const int64_t v0 = (r * n_series + s) * T, n_delta = n_real * n_series * T;
            const DF x = (L == 0) ? DF{*chk(delta, v0 + t, n_delta), 0.0f}
                                  : df_two_sum(*chk(delta, v0 + t + L, n_delta), -*chk(delta, v0 + t, n_delta));  // exact difference
            if (fabsf(x.hi) < 1.0e9f) {
                const DF x2 = df_mul(x, x);
                const DF x4 = df_mul(x2, x2);
                a2 = df_add(a2, x2);
                a4 = df_add(a4, x4);
            } else {  // x^4 would leave the FP32 range: this value in FP64 (also NaN, inf)
                const double xd = (double)x.hi + (double)x.lo, xd2 = xd * xd;
                b2 += xd2;
                b4 += xd2 * xd2;
            }
            ++n;
            r += dq;
            t += dr;
            if (t >= per) {
                t -= per;
                ++r;
            }
        }
        double s2 = ((double)a2.hi + (double)a2.lo) + b2, s4 = ((double)a4.hi + (double)a4.lo) + b4;
        double cnt = (double)n;
        s2 = warp_sum(s2);
        s4 = warp_sum(s4);
        cnt = warp_sum(cnt);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __syncthreads();  // red[] free from the previous pair
        if (lane == 0) { el(red, 0, w) = s2; el(red, 1, w) = s4; el(red, 2, w) = cnt; }
        __syncthreads();
        if (w == 0) {
            const int nw = blockDim.x >> 5;
            s2 = lane < nw ? el(red, 0, lane) : 0.0;
            s4 = lane < nw ? el(red, 1, lane) : 0.0;
            cnt = lane < nw ? el(red, 2, lane) : 0.0;
            s2 = warp_sum(s2);
            s4 = warp_sum(s4);
            cnt = warp_sum(cnt);
            if (lane == 0 && cnt > 0.0) {
                const int64_t o = (s * n_lags + l) * 3, n_acc = n_series * n_lags * 3;
                atomicAdd(chk(acc, o, n_acc), s2);
                atomicAdd(chk(acc, o + 1, n_acc), s4);
                atomicAdd(chk(acc, o + 2, n_acc), cnt);
            }
        }
    }
}

// out[r][q] = v[r][i_q] - v[r][j_q] (differential pistons, Sec. 4.4).  An
// index outside [0, n_points) gives NaN and records QRS_ERR_DEVICE_CHECK
// instead of reading out of bounds.
__global__ void k_pair_diff(const float* __restrict__ v, int64_t n_real, int64_t n_points,
                            const int2* __restrict__ pairs, int64_t n_pairs, float* __restrict__ out,
                            int* __restrict__ err)
{
    const int64_t total = n_real * n_pairs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n_pairs, q = i - r * n_pairs;
        const int2 pq = *chk(pairs, q, n_pairs);
        float d;
        if (pq.x < 0 || pq.x >= n_points || pq.y < 0 || pq.y >= n_points) {
            d = __int_as_float(0x7FC00000);
            atomicExch(err, (int)QRS_ERR_DEVICE_CHECK);
        } else {
            d = *chk(v, r * n_points + pq.x, n_real * n_points) - *chk(v, r * n_points + pq.y, n_real * n_points);
        }
        *chk(out, i, total) = d;
    }
}

cudaError_t launch_pair_diff(const float* v, int64_t n_real, int64_t n_points, const int32_t* pairs, int64_t n_pairs,
                             float* out, int num_sms, int* err, cudaStream_t s)
{
    const int64_t total = n_real * n_pairs;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
    if (blocks < 1) blocks = 1;
    k_pair_diff<<<(unsigned)blocks, 256, 0, s>>>(v, n_real, n_points, reinterpret_cast<const int2*>(pairs), n_pairs,
                                                 out, err);
    return cudaGetLastError();
}

cudaError_t launch_structure_fn(const float* delta, int64_t n_real, int64_t n_series, int64_t T, const int32_t* lags,
                                int32_t n_lags, double* acc, int num_sms, int* err, cudaStream_t s)
{
    const int64_t pairs = n_series * (int64_t)n_lags;
    const int64_t work = n_real * T;
    // about 4 CTAs per SM in total, at least one per pair, at most one per 256 values
    int64_t gx = (4LL * num_sms + pairs - 1) / pairs;
    const int64_t cap = (work + 255) / 256;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    dim3 grid((unsigned)gx, (unsigned)(pairs < 65535 ? pairs : 65535));
    k_structure_fn<<<grid, 256, 0, s>>>(delta, n_real, n_series, T, lags, n_lags, acc, err);
    return cudaGetLastError();
}

}  // namespace qrs
