// k_sf.cu -- K5: FP64 structure-function sums (Sec. 4.4), and the pair
// differences of synthesised values they are usually taken of.
// For every (series s, lag L): x = v[t+L] - v[t] (L >= 1) or x = v[t] (L = 0),
// summed over realisations and t as (sum x^2, sum x^4, count) in FP64.
// Grid: y = series-lag pair, x = slices of the flat (realisation, t) range.
// Each thread keeps FP64 partial sums, the block reduces them with warp
// shuffles, and one thread per block adds them to acc with FP64 atomics.
#include "qrs_internal.h"

namespace qrs {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_structure_fn(const float* __restrict__ delta, int64_t n_real, int64_t n_series,
                                                      int64_t T, const int32_t* __restrict__ lags, int32_t n_lags,
                                                      double* __restrict__ acc, int* __restrict__ err)
{
    const int64_t n_pairs = n_series * (int64_t)n_lags;
    __shared__ double red[3][8];
    for (int64_t pair = blockIdx.y; pair < n_pairs; pair += gridDim.y) {  // uniform per block
        const int64_t s = pair / n_lags;
        const int l = (int)(pair - s * n_lags);
        const int64_t L = lags[l];
        if (L < 0 || L >= T) {
            if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(err, (int)QRS_ERR_DEVICE_CHECK);
            continue;
        }
        const int64_t per = (L == 0) ? T : T - L;  // values per (realisation, series)
        const int64_t total = n_real * per;
        double s2 = 0.0, s4 = 0.0, cnt = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t r = i / per;
            const int64_t t = i - r * per;
            const float* v = delta + (r * n_series + s) * T;
            const double x = (L == 0) ? (double)v[t] : (double)v[t + L] - (double)v[t];
            const double x2 = x * x;
            s2 += x2;
            s4 += x2 * x2;
            cnt += 1.0;
        }
        s2 = warp_sum(s2);
        s4 = warp_sum(s4);
        cnt = warp_sum(cnt);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __syncthreads();  // red[] free from the previous pair
        if (lane == 0) { red[0][w] = s2; red[1][w] = s4; red[2][w] = cnt; }
        __syncthreads();
        if (w == 0) {
            const int nw = blockDim.x >> 5;
            s2 = lane < nw ? red[0][lane] : 0.0;
            s4 = lane < nw ? red[1][lane] : 0.0;
            cnt = lane < nw ? red[2][lane] : 0.0;
            s2 = warp_sum(s2);
            s4 = warp_sum(s4);
            cnt = warp_sum(cnt);
            if (lane == 0 && cnt > 0.0) {
                double* o = acc + (s * n_lags + l) * 3;
                atomicAdd(o, s2);
                atomicAdd(o + 1, s4);
                atomicAdd(o + 2, cnt);
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
        const int2 pq = pairs[q];
        float d;
        if (pq.x < 0 || pq.x >= n_points || pq.y < 0 || pq.y >= n_points) {
            d = __int_as_float(0x7FC00000);
            atomicExch(err, (int)QRS_ERR_DEVICE_CHECK);
        } else {
            const float* row = v + r * n_points;
            d = row[pq.x] - row[pq.y];
        }
        out[i] = d;
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
