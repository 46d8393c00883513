// k_piston.cu -- K4/K6: differential pistons (Sec. 4.1, 4.4; Eq. 7 filter).
//
// One work item = (job, realisation).  The CTA draws the realisation's N_f
// terms into shared memory (fused draw, chunks of kPisChunk terms), then its
// warps take (aperture, 256-term slice) units round-robin: the 32 lanes split
// the slice's terms, each lane forms F A_a(|f|) (a cos 2 pi f.p - b sin 2 pi f.p)
// in amplitude-phase form, A_a(|f|) F amp cos 2 pi (f.p + psi) (one cosine;
// amp and psi as in the fused synthesis kernel), with the double-float phase
// (aperture centres lie up to hundreds of metres from the origin), and a
// warp-shuffle reduction gives the slice's partial piston.  Partials are folded in a fixed order (deterministic sums), then
// the pair differences are written.
//
// Scheduling: a single job runs as a grid-stride over its realisations; a
// batch of jobs (QRS_PISTON_PERSISTENT) runs as one persistent grid whose
// CTAs pull items from an atomic counter over a cost-sorted item order
// (largest N_f n_ap first), so uneven jobs balance across SMs.  The queue
// never waits on anything, so there is no spin to bound.  The persistent
// kernel comes in three shapes (threads per CTA x terms per slice) among
// which the host-side autotuner picks per job-set shape.
#include "qrs_internal.h"
#include "qrs_piston.h"

namespace qrs {

constexpr int kPisChunk = 2048;  // terms per shared-memory chunk
constexpr int kPisBuckets = 64;  // |f| buckets of the per-chunk counting sort (8 per octave)
constexpr int kPisSortMinAp = 8; // items with at least this many apertures sort their chunks
constexpr int kPisMaxWarps = 8;
#ifndef QRS_PISTON_GROUP
#define QRS_PISTON_GROUP 4
#endif
constexpr int kPisGroup = QRS_PISTON_GROUP;  // apertures sharing one pass over a slice's terms
#ifndef QRS_PISTON_PAIRED
#define QRS_PISTON_PAIRED 1  // 1: the group's apertures in pairs through paired FP32 instructions
#endif

// Kernel shapes the autotuner chooses from: threads per CTA and terms per
// (aperture, slice) unit.
template <int TPB, int SLICE>
struct PisShape {
    static constexpr int kTPB = TPB;
    static constexpr int kWarps = TPB / 32;
    static constexpr int kSlice = SLICE;
    static constexpr int kSlices = kPisChunk / SLICE;
};

template <int SLICES>
struct PisShared {
    float4 rec[kPisChunk];             // fx, fy, F amp, psi (turns, [0, 0.5))
    float fabs_[kPisChunk];            // |f|
    uint16_t sidx[kPisChunk];          // terms in bucket order (sorted chunks)
    int bcount[kPisMaxWarps][kPisBuckets];
    float part[kPisMaxAp][SLICES];     // per-slice partial pistons of the chunk
    float total[kPisMaxAp];
    float apx[kPisMaxAp], apy[kPisMaxAp], apD[kPisMaxAp], apd[kPisMaxAp];
    float apwD[kPisMaxAp], apwd[kPisMaxAp];  // D^2 / (D^2 - d^2), d^2 / (D^2 - d^2)
};

// Bucket of |f| for the chunk sort: the float's exponent and top three
// mantissa bits (8 buckets per octave), the top bucket holding fmax, the
// lowest collecting everything 8 octaves or more below it.
__device__ __forceinline__ int pis_bucket(float fa, int base)
{
    const int e = (int)(__float_as_uint(fa) >> 20) - base;
    return e < 0 ? 0 : (e >= kPisBuckets ? kPisBuckets - 1 : e);
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One (aperture, slice) unit: the lanes split the slice's terms [k0, k_end)
// (in bucket order through sidx when SORTED); the filter's obstruction term
// only when OBST.  Both are uniform per unit, so they select a loop instead
// of being tested per term.
template <bool SORTED, bool OBST, int SLICES>
__device__ __forceinline__ float unit_sum(const PisShared<SLICES>& sh, int k0, int k_end, float x, float y, float D,
                                          float d, float wD, float wd)
{
    float acc = 0.0f;
    for (int k = k0; k < k_end; k += 32) {
        const int j = SORTED ? (int)sh.sidx[k] : k;
        const float4 T = sh.rec[j];
        const float fa = sh.fabs_[j];
        const float A = OBST ? airy_filter_w(fa, D, d, wD, wd) : airy_g(3.14159265358979f * fa * D);
        acc = fmaf(A * T.z, __cosf(phase_df_psi(T.x, T.y, x, y, T.w) * 6.28318530717958648f), acc);
    }
    return acc;
}

// NA unobstructed apertures per unit: one pass over the terms, the record,
// |f| and index loads and the loop control shared, NA independent chains.
template <bool SORTED, int NA, int SLICES>
__device__ __forceinline__ void unit_sum_n(const PisShared<SLICES>& sh, int k0, int k_end, int a0, float (&acc)[NA])
{
    float x[NA], y[NA], D[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        x[i] = sh.apx[a0 + i];
        y[i] = sh.apy[a0 + i];
        D[i] = sh.apD[a0 + i];
        acc[i] = 0.0f;
    }
#if QRS_PISTON_PAIRED
    // apertures in pairs: one paired FP32 instruction (FFMA2 / FMUL2 / FADD2)
    // does both apertures' step, rounded as the scalar one
    static_assert(NA % 2 == 0, "apertures in pairs");
    constexpr int NP = NA / 2;
    float2 x2[NP], y2[NP], D2[NP], acc2[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        x2[q] = make_float2(x[2 * q], x[2 * q + 1]);
        y2[q] = make_float2(y[2 * q], y[2 * q + 1]);
        D2[q] = make_float2(D[2 * q], D[2 * q + 1]);
        acc2[q] = make_float2(0.0f, 0.0f);
    }
    const float2 two_pi = make_float2(6.28318530717958648f, 6.28318530717958648f);
    const float2 quarter = make_float2(0.25f, 0.25f);
    for (int k = k0; k < k_end; k += 32) {
        const int j = SORTED ? (int)sh.sidx[k] : k;
        const float4 T = sh.rec[j];
        const float piF = 3.14159265358979f * sh.fabs_[j];
        const float2 PF = make_float2(piF, piF), Tz = make_float2(T.z, T.z);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float2 xx = __fmul2_rn(PF, D2[q]);
            float2 A;
            if (xx.x < 4.0f && xx.y < 4.0f) {  // both on the series branch of airy_g
                constexpr AiryCoef K;
                const float2 u = __fmul2_rn(__fmul2_rn(quarter, xx), xx);
                A = make_float2(K.c[10], K.c[10]);
#pragma unroll
                for (int m = 9; m >= 0; --m) A = __ffma2_rn(A, u, make_float2(K.c[m], K.c[m]));
            } else if (xx.x >= 4.0f && xx.y >= 4.0f) {  // both on the large-argument branch
                A = airy_g_large2(xx);
            } else {
                A = make_float2(airy_g(xx.x), airy_g(xx.y));
            }
            const float2 ang = __fmul2_rn(phase_df2_psi(T.x, T.y, x2[q], y2[q], T.w), two_pi);
            const float2 c = make_float2(__cosf(ang.x), __cosf(ang.y));
            acc2[q] = __ffma2_rn(__fmul2_rn(A, Tz), c, acc2[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        acc[2 * q] = acc2[q].x;
        acc[2 * q + 1] = acc2[q].y;
    }
#else
    for (int k = k0; k < k_end; k += 32) {
        const int j = SORTED ? (int)sh.sidx[k] : k;
        const float4 T = sh.rec[j];
        const float piF = 3.14159265358979f * sh.fabs_[j];
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const float A = airy_g(piF * D[i]);
            acc[i] = fmaf(A * T.z, __cosf(phase_df_psi(T.x, T.y, x[i], y[i], T.w) * 6.28318530717958648f), acc[i]);
        }
    }
#endif
}

template <class S>
__device__ void piston_item(const PistonJobDev& J, int64_t r, PisShared<S::kSlices>& sh, int* err)
{
    constexpr int kPisTPB = S::kTPB, kPisWarps = S::kWarps, kPisSlice = S::kSlice;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_ap = J.n_ap;
    for (int a = tid; a < n_ap; a += kPisTPB) {
        const float2 c = J.ap_xy[a];
        sh.apx[a] = c.x; sh.apy[a] = c.y;
        const float D = J.ap_D[a], d = J.ap_d ? J.ap_d[a] : 0.0f;
        sh.apD[a] = D;
        sh.apd[a] = d;
        sh.apwD[a] = d > 0.0f ? (D * D) / (D * D - d * d) : 1.0f;
        sh.apwd[a] = d > 0.0f ? (d * d) / (D * D - d * d) : 0.0f;
        sh.total[a] = 0.0f;
    }
    const DrawParams& p = J.p;
    const uint64_t nr0 = (uint64_t)(p.real_offset + r) * (uint64_t)p.n_f;
    for (int64_t k_begin = 0; k_begin < p.n_f; k_begin += kPisChunk) {
        const int len = (int)min((int64_t)kPisChunk, p.n_f - k_begin);
        __syncthreads();  // previous chunk and aperture setup complete
        for (int q = tid; q < len; q += kPisTPB) {
            const uint64_t n = nr0 + (uint64_t)(k_begin + q);
            Words w;
            const Term t = draw_term<false, false>(p, n, k_begin + q, &w);
            float amp;
            uint32_t u;
            coef_polar_from_words(p, n, w, amp, u);
            sh.rec[q] = make_float4(t.fx, t.fy, t.F * amp, (float)u * 0x1p-24f);
            sh.fabs_[q] = sqrtf(t.fx * t.fx + t.fy * t.fy);
        }
        __syncthreads();
        // Terms in order of |f| bucket: a warp's lanes then share the Eq. 7
        // filter's branch (x = pi D |f| below or above 4) instead of paying
        // both, consecutive R2 terms having unrelated |f|.  Stable counting
        // sort: per-warp bucket counts (match_any, no atomics), offsets
        // bucket-major then warp, then ranks -- a deterministic order.
        const bool sorted = n_ap >= kPisSortMinAp;
        if (sorted) {
            static_assert(kPisWarps <= kPisMaxWarps, "bucket counters per warp");
            const int base = (int)(__float_as_uint((float)p.fmax) >> 20) - (kPisBuckets - 1);
            const int per_warp = (len + kPisTPB - 1) / kPisTPB * 32;  // items per warp, a multiple of 32
            const int q_begin = warp * per_warp, q_end = q_begin + per_warp;
            for (int b = lane; b < kPisBuckets; b += 32) sh.bcount[warp][b] = 0;
            __syncwarp();
            for (int q0 = q_begin; q0 < q_end; q0 += 32) {
                const int q = q0 + lane;
                const int b = q < len ? pis_bucket(sh.fabs_[q], base) : kPisBuckets;
                const unsigned peers = __match_any_sync(0xffffffffu, b);
                if (b < kPisBuckets && lane == __ffs(peers) - 1) sh.bcount[warp][b] += __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            if (warp == 0) {
                int t0 = 0, t1 = 0;  // bucket totals: lane holds buckets lane and lane + 32
                for (int w = 0; w < kPisWarps; ++w) {
                    t0 += sh.bcount[w][lane];
                    t1 += sh.bcount[w][lane + 32];
                }
                int i0 = t0, i1 = t1;  // inclusive scans over the lanes
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v0 = __shfl_up_sync(0xffffffffu, i0, o), v1 = __shfl_up_sync(0xffffffffu, i1, o);
                    if (lane >= o) {
                        i0 += v0;
                        i1 += v1;
                    }
                }
                int e0 = i0 - t0, e1 = __shfl_sync(0xffffffffu, i0, 31) + i1 - t1;
                for (int w = 0; w < kPisWarps; ++w) {
                    const int c0 = sh.bcount[w][lane], c1 = sh.bcount[w][lane + 32];
                    sh.bcount[w][lane] = e0;
                    sh.bcount[w][lane + 32] = e1;
                    e0 += c0;
                    e1 += c1;
                }
            }
            __syncthreads();
            for (int q0 = q_begin; q0 < q_end; q0 += 32) {
                const int q = q0 + lane;
                const int b = q < len ? pis_bucket(sh.fabs_[q], base) : kPisBuckets;
                const unsigned peers = __match_any_sync(0xffffffffu, b);
                if (b < kPisBuckets) sh.sidx[sh.bcount[warp][b] + __popc(peers & ((1u << lane) - 1u))] = (uint16_t)q;
                __syncwarp();
                if (b < kPisBuckets && lane == __ffs(peers) - 1) sh.bcount[warp][b] += __popc(peers);
                __syncwarp();
            }
            __syncthreads();
        }
        // units: (group of kPisGroup apertures, slice); a group with an
        // obstructed aperture, or the short last group, runs aperture by aperture
        const int n_sl = (len + kPisSlice - 1) / kPisSlice;
        const int units = ((n_ap + kPisGroup - 1) / kPisGroup) * n_sl;
        for (int u = warp; u < units; u += kPisWarps) {
            const int q = u / n_sl, sl = u - q * n_sl;
            const int a0 = kPisGroup * q, a1 = a0 + kPisGroup - 1;
            const int k0 = sl * kPisSlice + lane, k_end = min(len, (sl + 1) * kPisSlice);
            bool plain = a1 < n_ap;
            for (int a = a0; plain && a <= a1; ++a) plain = sh.apd[a] <= 0.0f;
            if (plain) {
                float acc[kPisGroup];
                if (sorted) unit_sum_n<true>(sh, k0, k_end, a0, acc);
                else unit_sum_n<false>(sh, k0, k_end, a0, acc);
#pragma unroll
                for (int i = 0; i < kPisGroup; ++i) {
                    const float v = warp_sum_f(acc[i]);
                    if (lane == 0) sh.part[a0 + i][sl] = v;
                }
                continue;
            }
            for (int a = a0; a <= a1 && a < n_ap; ++a) {
                const float x = sh.apx[a], y = sh.apy[a], D = sh.apD[a], d = sh.apd[a];
                const float wD = sh.apwD[a], wd = sh.apwd[a];
                float acc;
                if (sorted) {
                    acc = d > 0.0f ? unit_sum<true, true>(sh, k0, k_end, x, y, D, d, wD, wd)
                                   : unit_sum<true, false>(sh, k0, k_end, x, y, D, d, wD, wd);
                } else {
                    acc = d > 0.0f ? unit_sum<false, true>(sh, k0, k_end, x, y, D, d, wD, wd)
                                   : unit_sum<false, false>(sh, k0, k_end, x, y, D, d, wD, wd);
                }
                acc = warp_sum_f(acc);
                if (lane == 0) sh.part[a][sl] = acc;
            }
        }
        __syncthreads();
        for (int a = tid; a < n_ap; a += kPisTPB) {
            float t = sh.total[a];
            for (int sl = 0; sl < n_sl; ++sl) t += sh.part[a][sl];
            sh.total[a] = t;
        }
    }
    __syncthreads();
    if (J.piston)
        for (int a = tid; a < n_ap; a += kPisTPB) J.piston[r * n_ap + a] = sh.total[a];
    if (J.delta)
        for (int q = tid; q < J.n_pairs; q += kPisTPB) {
            const int2 pr = J.pairs[q];
            float v = 0.0f;
            if (pr.x < 0 || pr.x >= n_ap || pr.y < 0 || pr.y >= n_ap) atomicExch(err, (int)QRS_ERR_DEVICE_CHECK);
            else v = sh.total[pr.x] - sh.total[pr.y];
            J.delta[r * J.n_pairs + q] = v;
        }
    __syncthreads();  // shared state reused by the next item
}

// Single job: grid-stride over its realisations.
using PisDefault = PisShape<256, 256>;

__global__ void __launch_bounds__(256, 4) k_piston_single(PistonJobDev J, int* err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sh = *reinterpret_cast<PisShared<PisDefault::kSlices>*>(smem_raw);
    for (int64_t r = blockIdx.x; r < J.n_real; r += gridDim.x) piston_item<PisDefault>(J, r, sh, err);
}

// Batch: items (job, realisation) in cost-sorted job order, pulled from an
// atomic counter.  jobs[] sorted by descending cost, item_begin its prefix sums.
template <class S>
__global__ void __launch_bounds__(S::kTPB, 1024 / S::kTPB) k_piston_persistent(const PistonJobDev* __restrict__ jobs, int n_jobs,
                                                               int64_t n_items, unsigned long long* counter, int* err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sh = *reinterpret_cast<PisShared<S::kSlices>*>(smem_raw);
    __shared__ long long s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t g = s_item;
        __syncthreads();
        if (g >= n_items) break;
        int lo = 0, hi = n_jobs;  // last job with item_begin <= g
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (jobs[mid].item_begin <= g) lo = mid; else hi = mid;
        }
        const PistonJobDev J = jobs[lo];
        piston_item<S>(J, g - J.item_begin, sh, err);
    }
}

size_t piston_smem_bytes() { return sizeof(PisShared<PisDefault::kSlices>); }

cudaError_t launch_piston_single(const PistonJobDev& J, int num_sms, int* err, cudaStream_t s)
{
    const size_t smem = sizeof(PisShared<PisDefault::kSlices>);
    cudaError_t e = cudaFuncSetAttribute(k_piston_single, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_piston_single, 256, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > J.n_real) grid = J.n_real;
    k_piston_single<<<(unsigned)grid, 256, smem, s>>>(J, err);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_persistent_t(const PistonJobDev* d_jobs, int n_jobs, int64_t n_items,
                                       unsigned long long* d_counter, int num_sms, int* err, cudaStream_t s)
{
    const size_t smem = sizeof(PisShared<S::kSlices>);
    cudaError_t e = cudaFuncSetAttribute(k_piston_persistent<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_piston_persistent<S>, S::kTPB, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > n_items) grid = n_items;
    k_piston_persistent<S><<<(unsigned)grid, S::kTPB, smem, s>>>(d_jobs, n_jobs, n_items, d_counter, err);
    return cudaGetLastError();
}

int piston_shape_count() { return 3; }

const char* piston_shape_name(int shape)
{
    static const char* names[] = {"tpb256_slice256", "tpb256_slice128", "tpb128_slice128"};
    return (shape >= 0 && shape < 3) ? names[shape] : "?";
}

cudaError_t launch_piston_persistent(int shape, const PistonJobDev* d_jobs, int n_jobs, int64_t n_items,
                                     unsigned long long* d_counter, int num_sms, int* err, cudaStream_t s)
{
    switch (shape) {
    case 1: return launch_persistent_t<PisShape<256, 128>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    case 2: return launch_persistent_t<PisShape<128, 128>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    default: return launch_persistent_t<PisShape<256, 256>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    }
}

}  // namespace qrs
