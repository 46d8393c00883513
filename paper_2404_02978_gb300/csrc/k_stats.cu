// k_stats.cu -- K9: clusters and gaps of frequency draws (Sec. 2.3, 3.2,
// Figs. 2-3 compare jittered, random and quasi-random sampling).
//
// k_nearest_neighbour: per set of n points, each point's distance to its
//   nearest other point (Euclidean, FP32).  One thread per point; the set's
//   points are staged through shared memory in tiles; grid (point blocks, set).
// k_star_discrepancy: per set of n points in [0,1]^2, the star discrepancy
//   D* = max over corners (u, v) in ({x_i} U {1}) x ({y_j} U {1}) of
//   max(C/n - u v, u v - O/n), C the count of points with x <= u, y <= v and
//   O the count with x < u, y < v.  The counts are exact integers and u v is
//   exact in FP64 (two 24-bit significands), so the result is exact: one
//   thread per corner, points staged through shared memory, block max, then
//   an atomic max on the FP64 bit pattern (D* >= 0, so integer order is
//   numeric order).  Work (n+1)^2 n per set.
#include "qrs_internal.h"

namespace qrs {

QRS_CHECK_HOOK(check_hook_stats)

constexpr int kStatTPB = 256;
constexpr int kStatTile = 2048;  // points per shared-memory tile (16 KB)

__global__ void __launch_bounds__(kStatTPB) k_nearest_neighbour(const float2* __restrict__ pts, int64_t n,
                                                                float* __restrict__ out)
{
    __shared__ float2 tile[kStatTile];
    const int64_t set = blockIdx.y;
    const int64_t n_all = (int64_t)gridDim.y * n;
    const int64_t i = (int64_t)blockIdx.x * kStatTPB + threadIdx.x;
    const float2 me = (i < n) ? *chk(pts, set * n + i, n_all) : make_float2(0.0f, 0.0f);
    float best = __int_as_float(0x7F800000);  // +inf
    for (int64_t t0 = 0; t0 < n; t0 += kStatTile) {
        const int len = (int)((n - t0 < kStatTile) ? n - t0 : kStatTile);
        __syncthreads();
        for (int k = threadIdx.x; k < len; k += kStatTPB) el(tile, k) = *chk(pts, set * n + t0 + k, n_all);
        __syncthreads();
        for (int k = 0; k < len; ++k) {
            const float2 q = el(tile, k);
            const float dx = q.x - me.x, dy = q.y - me.y;
            const float d2 = fmaf(dx, dx, dy * dy);
            if (t0 + k != i && d2 < best) best = d2;
        }
    }
    if (i < n) *chk(out, set * n + i, n_all) = (n > 1) ? sqrtf(best) : 0.0f;
}

__global__ void __launch_bounds__(kStatTPB) k_star_discrepancy(const float2* __restrict__ pts, int64_t n,
                                                               unsigned long long* __restrict__ out)
{
    __shared__ float2 tile[kStatTile];
    __shared__ double red[kStatTPB / 32];
    const int64_t set = blockIdx.y;
    const int64_t n_all = (int64_t)gridDim.y * n;
    const int64_t corners = (n + 1) * (n + 1);
    const int64_t c = (int64_t)blockIdx.x * kStatTPB + threadIdx.x;
    const bool live = c < corners;
    const int64_t ci = live ? c / (n + 1) : 0, cj = live ? c - ci * (n + 1) : 0;
    const float u = (ci < n) ? chk(pts, set * n + ci, n_all)->x : 1.0f;
    const float v = (cj < n) ? chk(pts, set * n + cj, n_all)->y : 1.0f;
    int64_t closed = 0, open = 0;
    for (int64_t t0 = 0; t0 < n; t0 += kStatTile) {
        const int len = (int)((n - t0 < kStatTile) ? n - t0 : kStatTile);
        __syncthreads();
        for (int k = threadIdx.x; k < len; k += kStatTPB) el(tile, k) = *chk(pts, set * n + t0 + k, n_all);
        __syncthreads();
        int cc = 0, oo = 0;
        for (int k = 0; k < len; ++k) {
            const float2 q = el(tile, k);
            cc += (q.x <= u && q.y <= v) ? 1 : 0;
            oo += (q.x < u && q.y < v) ? 1 : 0;
        }
        closed += cc;
        open += oo;
    }
    double D = 0.0;
    if (live) {
        const double uv = (double)u * (double)v;
        const double a = (double)closed / (double)n - uv;
        const double b = uv - (double)open / (double)n;
        D = fmax(0.0, fmax(a, b));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) D = fmax(D, __shfl_xor_sync(0xffffffffu, D, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = D;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kStatTPB / 32; ++k) D = fmax(D, red[k]);
        atomicMax(out + set, (unsigned long long)__double_as_longlong(D));
    }
}

cudaError_t launch_nearest_neighbour(const float* pts, int64_t n_sets, int64_t n, float* out, cudaStream_t s)
{
    dim3 grid((unsigned)((n + kStatTPB - 1) / kStatTPB), (unsigned)n_sets);
    k_nearest_neighbour<<<grid, kStatTPB, 0, s>>>(reinterpret_cast<const float2*>(pts), n, out);
    return cudaGetLastError();
}

cudaError_t launch_star_discrepancy(const float* pts, int64_t n_sets, int64_t n, double* out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n_sets * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int64_t corners = (n + 1) * (n + 1);
    dim3 grid((unsigned)((corners + kStatTPB - 1) / kStatTPB), (unsigned)n_sets);
    k_star_discrepancy<<<grid, kStatTPB, 0, s>>>(reinterpret_cast<const float2*>(pts), n,
                                                 reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError();
}

}  // namespace qrs
