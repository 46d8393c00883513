// k_piston.cu -- K4/K6: differential pistons (Sec. 4.1, 4.4; Eq. 7 filter).
//
// One work item = (job, realisation).  The CTA draws the realisation's N_f
// terms into shared memory (fused draw, chunks of kPisChunk terms), then its
// warps take (group of apertures, slice of terms) units round-robin: the 32
// lanes split the slice's terms, each lane forms F A_a(|f|) (a cos 2 pi f.p -
// b sin 2 pi f.p) in amplitude-phase form, A_a(|f|) F amp cos 2 pi (f.p + psi)
// (one cosine; amp and psi as in the fused synthesis kernel), with the
// double-float phase (aperture centres lie up to hundreds of metres from the
// origin), and a warp-shuffle reduction gives the slice's partial piston.
// Partials are folded in a fixed order (deterministic sums), then the pair
// differences are written.
//
// The Eq. 7 filter g(pi D |f|) of each (aperture, term):
//   - if every aperture of the job has the same (D, d), once per term, into
//     the term's amplitude (the units then evaluate no filter);
//   - else per unit, in the cheapest form valid over the unit's range of
//     x = pi D |f|: a chunk's terms are ordered by |f| bucket and the
//     apertures by D, so a unit covers a limited range of x, and its bounds
//     pick a Taylor series of 5 or 11 terms (x below 0.5, 4) or a
//     large-argument form of degree 1 or 4 (x from 16, 4 on); only a unit
//     whose range straddles x = 4 tests each term.  (More forms, e.g. 7-term
//     series below x = 1.5 and degree 2 from x = 8, were timed slower: the
//     kernel's code outgrows the instruction cache.)
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

QRS_CHECK_HOOK(check_hook_piston)

constexpr int kPisChunk = 2048;  // terms per shared-memory chunk
constexpr int kPisBuckets = 64;  // |f| buckets of the per-chunk counting sort (8 per octave)
constexpr int kPisSortMinAp = 8; // items with at least this many apertures sort their chunks
constexpr int kPisMaxWarps = 8;
constexpr int kPisGroup = 4;     // apertures sharing one pass over a slice's terms (two pairs)

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
    float pif[kPisChunk];              // pi |f|
    uint16_t sidx[kPisChunk];          // terms in bucket order (sorted chunks)
    int bcount[kPisMaxWarps][kPisBuckets];
    float part[kPisMaxAp][SLICES];     // per-slice partial pistons of the chunk
    float total[kPisMaxAp];
    float apx[kPisMaxAp], apy[kPisMaxAp], apD[kPisMaxAp], apd[kPisMaxAp];
    float apwD[kPisMaxAp], apwd[kPisMaxAp];  // D^2 / (D^2 - d^2), d^2 / (D^2 - d^2)
    uint8_t rank[kPisMaxAp];           // the job's aperture a sits in slot rank[a] (slots in order of D)
};

// The filter form a unit of unobstructed apertures takes (valid where every
// x = pi D |f| of the unit lies): Taylor series in x^2 through x^8 or x^20
// (x < 0.5, 4), the large-argument form of degree 1 or 4 in 1/x^2 (x >= 16,
// 4), or a per-term choice between the 11-term series and degree 4.
enum { kFltSer4, kFltSer10, kFltLrg1, kFltLrg4, kFltMixed };

__device__ __forceinline__ int filter_form(float x_lo, float x_hi)
{
    if (x_hi < 4.0f) return x_hi < 0.5f ? kFltSer4 : kFltSer10;
    if (x_lo >= 4.0f) return x_lo >= 16.0f ? kFltLrg1 : kFltLrg4;
    return kFltMixed;
}

// The filter of two apertures (D, D^2 pairs) at one term (pi |f| and its square).
template <int FORM>
__device__ __forceinline__ float2 filter2(float pf, float pf2, float2 D, float2 DD)
{
    if constexpr (FORM == kFltSer4) return airy_series_v2<4>(__fmul2_rn(make_float2(pf2, pf2), DD));
    else if constexpr (FORM == kFltSer10) return airy_series_v2<10>(__fmul2_rn(make_float2(pf2, pf2), DD));
    else if constexpr (FORM == kFltLrg1) return airy_large2<1>(__fmul2_rn(make_float2(pf, pf), D));
    else if constexpr (FORM == kFltLrg4) return airy_large2<4>(__fmul2_rn(make_float2(pf, pf), D));
    else {
        const float2 x = __fmul2_rn(make_float2(pf, pf), D);
        if (x.x < 4.0f && x.y < 4.0f) return airy_series_v2<10>(__fmul2_rn(x, x));
        if (x.x >= 4.0f && x.y >= 4.0f) return airy_large2<4>(x);
        return make_float2(airy_g(x.x), airy_g(x.y));
    }
}

// Bucket of pi |f| for the chunk sort: the float's exponent and top three
// mantissa bits (8 buckets per octave), the top bucket holding pi fmax, the
// lowest collecting everything 8 octaves or more below it.
__device__ __forceinline__ int pis_bucket(float v, int base)
{
    const int e = (int)(__float_as_uint(v) >> 20) - base;
    return e < 0 ? 0 : (e >= kPisBuckets ? kPisBuckets - 1 : e);
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One (aperture, slice) unit, aperture by aperture: the lanes split the
// slice's terms [k0, k_end) (in bucket order through sidx when SORTED); the
// filter's obstruction term only when OBST.  Both are uniform per unit, so
// they select a loop instead of being tested per term.
template <bool SORTED, bool OBST, int SLICES>
__device__ __forceinline__ float unit_sum(const PisShared<SLICES>& sh, int k0, int k_end, float x, float y, float D,
                                          float d, float wD, float wd)
{
    float acc = 0.0f;
    for (int k = k0; k < k_end; k += 32) {
        const int j = SORTED ? (int)el(sh.sidx, k) : k;
        const float4 T = el(sh.rec, j);
        const float pf = el(sh.pif, j);
        const float A = OBST ? fmaf(wD, airy_g(pf * D), -wd * airy_g(pf * d)) : airy_g(pf * D);
        acc = fmaf(A * T.z, __cosf(phase_df_psi(T.x, T.y, x, y, T.w) * 6.28318530717958648f), acc);
    }
    return acc;
}

// kPisGroup unobstructed apertures (slots a0 ..) per unit: one pass over the
// terms, the record, pi |f| and index loads and the loop control shared, two
// pairs of apertures through paired FP32 instructions (FFMA2 / FMUL2 /
// FADD2, each element rounded as the scalar instruction); the filter in
// the form FORM.
template <int FORM, bool SORTED, int SLICES>
__device__ __forceinline__ void unit_sum_group(const PisShared<SLICES>& sh, int k0, int k_end, int a0,
                                               float (&acc)[kPisGroup])
{
    constexpr int NP = kPisGroup / 2;
    float2 x2[NP], y2[NP], D2[NP], DD2[NP], acc2[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        x2[q] = make_float2(el(sh.apx, a0 + 2 * q), el(sh.apx, a0 + 2 * q + 1));
        y2[q] = make_float2(el(sh.apy, a0 + 2 * q), el(sh.apy, a0 + 2 * q + 1));
        D2[q] = make_float2(el(sh.apD, a0 + 2 * q), el(sh.apD, a0 + 2 * q + 1));
        DD2[q] = __fmul2_rn(D2[q], D2[q]);
        acc2[q] = make_float2(0.0f, 0.0f);
    }
    const float2 two_pi = make_float2(6.28318530717958648f, 6.28318530717958648f);
    for (int k = k0; k < k_end; k += 32) {
        const int j = SORTED ? (int)el(sh.sidx, k) : k;
        const float4 T = el(sh.rec, j);
        const float pf = el(sh.pif, j);
        const float pf2 = (FORM <= kFltSer10) ? pf * pf : 0.0f;
        const float2 Tz = make_float2(T.z, T.z);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float2 A = filter2<FORM>(pf, pf2, D2[q], DD2[q]);
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
}

// Sorted chunks: the unit's form.  (Unsorted chunks, of items with few
// apertures, run the per-term choice: their units span the whole |f| range.)
template <int SLICES>
__device__ __forceinline__ void unit_sum_group_form(int form, const PisShared<SLICES>& sh, int k0, int k_end, int a0,
                                                    float (&acc)[kPisGroup])
{
    switch (form) {
    case kFltSer4: unit_sum_group<kFltSer4, true>(sh, k0, k_end, a0, acc); break;
    case kFltSer10: unit_sum_group<kFltSer10, true>(sh, k0, k_end, a0, acc); break;
    case kFltLrg1: unit_sum_group<kFltLrg1, true>(sh, k0, k_end, a0, acc); break;
    case kFltLrg4: unit_sum_group<kFltLrg4, true>(sh, k0, k_end, a0, acc); break;
    default: unit_sum_group<kFltMixed, true>(sh, k0, k_end, a0, acc); break;
    }
}

// NA apertures per unit when the Eq. 7 filter is already in the term records
// (every aperture of the job has the same D and d): the phase, one cosine and
// the accumulation per (aperture, term), pairs of apertures in paired FP32
// instructions.  NA even, or 1 for a lone aperture.
template <int NA, int SLICES>
__device__ __forceinline__ void unit_sum_prefiltered(const PisShared<SLICES>& sh, int k0, int k_end, int a0,
                                                     float (&acc)[NA])
{
    if constexpr (NA == 1) {
        const float x = el(sh.apx, a0), y = el(sh.apy, a0);
        float s = 0.0f;
        for (int k = k0; k < k_end; k += 32) {
            const float4 T = el(sh.rec, k);
            s = fmaf(T.z, __cosf(phase_df_psi(T.x, T.y, x, y, T.w) * 6.28318530717958648f), s);
        }
        acc[0] = s;
    } else {
        static_assert(NA % 2 == 0, "apertures in pairs");
        constexpr int NP = NA / 2;
        float2 x2[NP], y2[NP], acc2[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            x2[q] = make_float2(el(sh.apx, a0 + 2 * q), el(sh.apx, a0 + 2 * q + 1));
            y2[q] = make_float2(el(sh.apy, a0 + 2 * q), el(sh.apy, a0 + 2 * q + 1));
            acc2[q] = make_float2(0.0f, 0.0f);
        }
        const float2 two_pi = make_float2(6.28318530717958648f, 6.28318530717958648f);
        for (int k = k0; k < k_end; k += 32) {
            const float4 T = el(sh.rec, k);
            const float2 Tz = make_float2(T.z, T.z);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 ang = __fmul2_rn(phase_df2_psi(T.x, T.y, x2[q], y2[q], T.w), two_pi);
                acc2[q] = __ffma2_rn(Tz, make_float2(__cosf(ang.x), __cosf(ang.y)), acc2[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            acc[2 * q] = acc2[q].x;
            acc[2 * q + 1] = acc2[q].y;
        }
    }
}

template <class S>
__device__ void piston_item(const PistonJobDev& J, int64_t r, PisShared<S::kSlices>& sh, int* err)
{
    constexpr int kPisTPB = S::kTPB, kPisWarps = S::kWarps, kPisSlice = S::kSlice;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_ap = J.n_ap;
    // The apertures take slots in order of D (ties by index): a group of
    // apertures that share a pass over the terms then has close diameters,
    // so that its range of pi D |f| is narrow.  Each aperture's sum is formed
    // the same way in any slot.  The slots are ranked in shared memory: the
    // diameters first, then every aperture's rank against them.
    // When every aperture has the same (D, d), the Eq. 7 filter is a function
    // of the term alone: it is taken once per term into the record's
    // amplitude, and the units evaluate no filter (and need no |f| order).
    const float D0 = *chk(J.ap_D, 0, n_ap), d0 = J.ap_d ? *chk(J.ap_d, 0, n_ap) : 0.0f;
    bool same = true;
    for (int a = tid; a < n_ap; a += kPisTPB) {
        const float D = *chk(J.ap_D, a, n_ap), d = J.ap_d ? *chk(J.ap_d, a, n_ap) : 0.0f;
        el(sh.apwD, a) = D;  // staging: the diameters in job order
        same = same && D == D0 && d == d0;
    }
    const bool prefilter = __syncthreads_and(same) != 0;
    // order key: the float's bits mapped to an unsigned total order (any bit
    // pattern, NaN included, gets a distinct slot: the slots are a permutation)
    auto key = [](float v) {
        const uint32_t u = __float_as_uint(v);
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    };
    int my_slot[(kPisMaxAp + kPisTPB - 1) / kPisTPB];
#pragma unroll
    for (int i = 0; i < (kPisMaxAp + kPisTPB - 1) / kPisTPB; ++i) {
        const int a = tid + i * kPisTPB;
        my_slot[i] = 0;
        if (a < n_ap) {
            const uint32_t ka = key(el(sh.apwD, a));
            int s = 0;
            for (int b = 0; b < n_ap; ++b) {
                const uint32_t kb = key(el(sh.apwD, b));
                s += (kb < ka || (kb == ka && b < a)) ? 1 : 0;
            }
            my_slot[i] = s;
        }
    }
    __syncthreads();  // the staged diameters are read; the slots may be written
#pragma unroll
    for (int i = 0; i < (kPisMaxAp + kPisTPB - 1) / kPisTPB; ++i) {
        const int a = tid + i * kPisTPB;
        if (a < n_ap) {
            const int s = my_slot[i];
            const float D = *chk(J.ap_D, a, n_ap), d = J.ap_d ? *chk(J.ap_d, a, n_ap) : 0.0f;
            const float2 c = *chk(J.ap_xy, a, n_ap);
            el(sh.rank, a) = (uint8_t)s;
            el(sh.apx, s) = c.x; el(sh.apy, s) = c.y;
            el(sh.apD, s) = D;
            el(sh.apd, s) = d;
            el(sh.apwD, s) = d > 0.0f ? (D * D) / (D * D - d * d) : 1.0f;
            el(sh.apwd, s) = d > 0.0f ? (d * d) / (D * D - d * d) : 0.0f;
            el(sh.total, s) = 0.0f;
        }
    }
    const float wD0 = d0 > 0.0f ? (D0 * D0) / (D0 * D0 - d0 * d0) : 1.0f;
    const float wd0 = d0 > 0.0f ? (d0 * d0) / (D0 * D0 - d0 * d0) : 0.0f;
    const DrawParams& p = J.p;
    const uint64_t nr0 = (uint64_t)(p.real_offset + r) * (uint64_t)p.n_f;
    for (int64_t k_begin = 0; k_begin < p.n_f; k_begin += kPisChunk) {
        const int len = (int)min((int64_t)kPisChunk, p.n_f - k_begin);
        __syncthreads();  // previous chunk and aperture setup complete
        for (int q = tid; q < len; q += kPisTPB) {
            const uint64_t n = nr0 + (uint64_t)(k_begin + q);
            Words w;
            const Term t = draw_term<false, false>(p, n, k_begin + q, &w);
            float Fa;
            uint32_t u;
            term_amp_polar(p, n, w, t.var, t.F, Fa, u);
            const float fa = fast_abs_f(t.fx * t.fx + t.fy * t.fy);
            if (prefilter) Fa = airy_filter_w(fa, D0, d0, wD0, wd0) * Fa;
            el(sh.rec, q) = make_float4(t.fx, t.fy, Fa, (float)u * 0x1p-24f);
            el(sh.pif, q) = 3.14159265358979f * fa;
        }
        __syncthreads();
        // Terms in order of |f| bucket: a warp's lanes then take the same
        // filter form, and a slice covers a narrow range of |f|, consecutive
        // R2 terms having unrelated |f|.  Stable counting sort: per-warp
        // bucket counts (match_any, no atomics), offsets bucket-major then
        // warp, then ranks -- a deterministic order.
        const bool sorted = !prefilter && n_ap >= kPisSortMinAp;
        if (sorted) {
            static_assert(kPisWarps <= kPisMaxWarps, "bucket counters per warp");
            const int base = (int)(__float_as_uint(3.14159265358979f * (float)p.fmax) >> 20) - (kPisBuckets - 1);
            const int per_warp = (len + kPisTPB - 1) / kPisTPB * 32;  // items per warp, a multiple of 32
            const int q_begin = warp * per_warp, q_end = q_begin + per_warp;
            for (int b = lane; b < kPisBuckets; b += 32) el(sh.bcount, warp, b) = 0;
            __syncwarp();
            for (int q0 = q_begin; q0 < q_end; q0 += 32) {
                const int q = q0 + lane;
                const int b = q < len ? pis_bucket(el(sh.pif, q), base) : kPisBuckets;
                const unsigned peers = __match_any_sync(0xffffffffu, b);
                if (b < kPisBuckets && lane == __ffs(peers) - 1) el(sh.bcount, warp, b) += __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            if (warp == 0) {
                int t0 = 0, t1 = 0;  // bucket totals: lane holds buckets lane and lane + 32
                for (int w = 0; w < kPisWarps; ++w) {
                    t0 += el(sh.bcount, w, lane);
                    t1 += el(sh.bcount, w, lane + 32);
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
                    const int c0 = el(sh.bcount, w, lane), c1 = el(sh.bcount, w, lane + 32);
                    el(sh.bcount, w, lane) = e0;
                    el(sh.bcount, w, lane + 32) = e1;
                    e0 += c0;
                    e1 += c1;
                }
            }
            __syncthreads();
            for (int q0 = q_begin; q0 < q_end; q0 += 32) {
                const int q = q0 + lane;
                const int b = q < len ? pis_bucket(el(sh.pif, q), base) : kPisBuckets;
                const unsigned peers = __match_any_sync(0xffffffffu, b);
                if (b < kPisBuckets) el(sh.sidx, el(sh.bcount, warp, b) + __popc(peers & ((1u << lane) - 1u))) = (uint16_t)q;
                __syncwarp();
                if (b < kPisBuckets && lane == __ffs(peers) - 1) el(sh.bcount, warp, b) += __popc(peers);
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
            if (prefilter) {
                if (a1 < n_ap) {
                    float acc[kPisGroup];
                    unit_sum_prefiltered<kPisGroup>(sh, k0, k_end, a0, acc);
#pragma unroll
                    for (int i = 0; i < kPisGroup; ++i) {
                        const float v = warp_sum_f(acc[i]);
                        if (lane == 0) el(sh.part, a0 + i, sl) = v;
                    }
                } else {
                    for (int a = a0; a < n_ap; ++a) {
                        float acc[1];
                        unit_sum_prefiltered<1>(sh, k0, k_end, a, acc);
                        const float v = warp_sum_f(acc[0]);
                        if (lane == 0) el(sh.part, a, sl) = v;
                    }
                }
                continue;
            }
            bool plain = a1 < n_ap;
            for (int a = a0; plain && a <= a1; ++a) plain = el(sh.apd, a) <= 0.0f;
            if (plain) {
                float acc[kPisGroup];
                if (sorted) {
                    // The unit's filter arguments x = fl(pi |f| D) lie between
                    // those of its smallest pi |f| and D and of its largest
                    // (rounding is monotonic), so these bounds pick a form
                    // valid for every term of the unit.
                    float f_lo = 3.402823466e38f, f_hi = 0.0f;
                    for (int k = k0; k < k_end; k += 32) {
                        const float pf = el(sh.pif, el(sh.sidx, k));
                        f_lo = fminf(f_lo, pf);
                        f_hi = fmaxf(f_hi, pf);
                    }
                    // pi |f| >= 0: the float bits order as the values
                    f_lo = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(f_lo)));
                    f_hi = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(f_hi)));
                    float D_lo = el(sh.apD, a0), D_hi = D_lo;
                    for (int a = a0 + 1; a <= a1; ++a) {
                        D_lo = fminf(D_lo, el(sh.apD, a));
                        D_hi = fmaxf(D_hi, el(sh.apD, a));
                    }
                    unit_sum_group_form(filter_form(f_lo * D_lo, f_hi * D_hi), sh, k0, k_end, a0, acc);
                } else {
                    unit_sum_group<kFltMixed, false>(sh, k0, k_end, a0, acc);
                }
#pragma unroll
                for (int i = 0; i < kPisGroup; ++i) {
                    const float v = warp_sum_f(acc[i]);
                    if (lane == 0) el(sh.part, a0 + i, sl) = v;
                }
                continue;
            }
            for (int a = a0; a <= a1 && a < n_ap; ++a) {
                const float x = el(sh.apx, a), y = el(sh.apy, a), D = el(sh.apD, a), d = el(sh.apd, a);
                const float wD = el(sh.apwD, a), wd = el(sh.apwd, a);
                float acc;
                if (sorted) {
                    acc = d > 0.0f ? unit_sum<true, true>(sh, k0, k_end, x, y, D, d, wD, wd)
                                   : unit_sum<true, false>(sh, k0, k_end, x, y, D, d, wD, wd);
                } else {
                    acc = d > 0.0f ? unit_sum<false, true>(sh, k0, k_end, x, y, D, d, wD, wd)
                                   : unit_sum<false, false>(sh, k0, k_end, x, y, D, d, wD, wd);
                }
                acc = warp_sum_f(acc);
                if (lane == 0) el(sh.part, a, sl) = acc;
            }
        }
        __syncthreads();
        for (int a = tid; a < n_ap; a += kPisTPB) {
            float t = el(sh.total, a);
            for (int sl = 0; sl < n_sl; ++sl) t += el(sh.part, a, sl);
            el(sh.total, a) = t;
        }
    }
    __syncthreads();
    if (J.piston)
        for (int a = tid; a < n_ap; a += kPisTPB) *chk(J.piston, r * n_ap + a, J.n_real * n_ap) = el(sh.total, el(sh.rank, a));
    if (J.delta)
        for (int q = tid; q < J.n_pairs; q += kPisTPB) {
            const int2 pr = *chk(J.pairs, q, J.n_pairs);
            float v = 0.0f;
            if (pr.x < 0 || pr.x >= n_ap || pr.y < 0 || pr.y >= n_ap) atomicExch(err, (int)QRS_ERR_DEVICE_CHECK);
            else v = el(sh.total, el(sh.rank, pr.x)) - el(sh.total, el(sh.rank, pr.y));
            *chk(J.delta, r * J.n_pairs + q, J.n_real * J.n_pairs) = v;
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
            if (chk(jobs, mid, n_jobs)->item_begin <= g) lo = mid; else hi = mid;
        }
        const PistonJobDev J = *chk(jobs, lo, n_jobs);
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

// The autotuner's candidates (threads per CTA, terms per (group, slice)
// unit): more, shorter slices balance short draws (small N_f) across the
// warps; longer ones amortise each unit's form choice and reduction.
int piston_shape_count() { return 5; }

const char* piston_shape_name(int shape)
{
    static const char* names[] = {"tpb256_slice256", "tpb256_slice128", "tpb128_slice128", "tpb256_slice64",
                                  "tpb128_slice256"};
    return (shape >= 0 && shape < 5) ? names[shape] : "?";
}

cudaError_t launch_piston_persistent(int shape, const PistonJobDev* d_jobs, int n_jobs, int64_t n_items,
                                     unsigned long long* d_counter, int num_sms, int* err, cudaStream_t s)
{
    switch (shape) {
    case 1: return launch_persistent_t<PisShape<256, 128>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    case 2: return launch_persistent_t<PisShape<128, 128>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    case 3: return launch_persistent_t<PisShape<256, 64>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    case 4: return launch_persistent_t<PisShape<128, 256>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    default: return launch_persistent_t<PisShape<256, 256>>(d_jobs, n_jobs, n_items, d_counter, num_sms, err, s);
    }
}

}  // namespace qrs
