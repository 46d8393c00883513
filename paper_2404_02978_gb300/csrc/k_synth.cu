// k_synth.cu -- K2: fused per-realisation draw + cosine-accumulate (Eq. 3 at
// arbitrary points): the point-bound prepass that picks the phase path, the
// anchored kernel (k_synth_anchor) and the exact kernel (k_synth_fused); both
// kernels are launched and the one whose path does not apply returns at once.
//
// Work decomposition of the exact kernel.  A work item is (realisation r, tile of TPB*PPT points);
// items are numbered realisation-major and each CTA of a persistent grid (a
// whole number of CTAs per SM) takes one contiguous range of them, so it
// visits few realisations.  The N_f terms of the current realisation are
// drawn by the CTA itself (Philox + R2 + domain map, draw_term) into shared
// memory once and reused by every tile of that realisation in its range;
// two CTAs of 128 threads with 12 points each share an SM (registers capped
// for that: the points give each thread 12 independent chains per term);
// N_f beyond the shared-memory chunk is processed in chunks re-drawn per
// item.  Each thread keeps PPT points in registers (strided by TPB, so the
// loads and stores of a warp are coalesced) and loops over the terms, read
// as one broadcast 16-byte shared-memory record per term.
//
// Amplitude-phase form: the term F (a cos 2 pi phi - b sin 2 pi phi) of Eq. 3
// is F amp cos 2 pi (phi + u 2^-24), with (amp, u) the Box-Muller radius and
// 24-bit angle (or, for the literal Eq. 3 coefficients, sqrt2 R_n and R_u),
// the angle's top bit moved into the sign of amp (u < 2^23): one cosine per
// (point, term) instead of a sine and a cosine.  Records:
//   fixed-point path: {Fx, Fy (int32 scaled 2^a), F amp, u (uint32)}; the
//     offset u 2^(a+b-24) joins the 64-bit phase word as the addend of its
//     first multiply-add, exactly
//   double-float path: {fx, fy (float), F amp, psi = u 2^-24 in [0, 0.5)}
// The phase path is uniform per launch: fixed point when fbound * xbound
// <= 128 (its quantisation error, about max(fbound xbound 2^-30, 2^-25) turns
// with the cap on a + b, is then below the double-float path's),
// double-float otherwise.  Where the scales allow
// a + b = 55 (fbound * xbound <= 64 with room in the ceilings), the fraction
// is the low 23 bits of the phase word's high half and needs no shift.
//
// Anchored path (Eq. 3 unchanged; its own kernel, k_synth_anchor): each
// thread takes kAnchorPPT (16) consecutive points, and the group's first and
// last points are its two anchors.  Per term the thread reduces the phase of
// the two anchors only, exactly (fixed point, or double-float where the
// point bound is too large for it); every point adds its FP32 offset from
// the nearer anchor, 2 pi (fx dx + fy dy), to that anchor's phase in
// radians, so a (point, term) costs three paired FP32 instructions and the
// cosine instead of two wide integer multiply-adds (or the double-float
// reduction).  The offset's rounding error grows with f . dx, so the path
// applies only where the prepass finds every point within dbound of its
// anchor with fbound * dbound <= kAnchorTurns (8 turns): the error of a term
// is then at most a few 2^-24 of 2 pi (1.5 + 2 fbound dbound) radians, and
// the terms with large f . dx are those with small amplitudes.  Scattered
// points take the exact paths.  The anchored kernel takes its terms in small
// chunks per realisation segment and carries each point's running sum from
// chunk to chunk in the output, so three CTAs fit on an SM.
//
// Accumulation: every 64 terms a partial sum is folded into the running sum,
// which keeps the FP32 rounding error of N_f = 4096..16384-term sums near
// 1e-7 of the field's standard deviation.
#include "qrs_internal.h"

namespace qrs {

QRS_CHECK_HOOK(check_hook_synth)

// Tunables (compile-time; the defaults are the measured best on GB300).
#ifndef QRS_SYNTH_PPT
#define QRS_SYNTH_PPT 12     // points per thread
#endif
#ifndef QRS_SYNTH_MINB
#define QRS_SYNTH_MINB 2     // minimum resident CTAs per SM (register cap)
#endif
#ifndef QRS_SYNTH_UNROLL
#define QRS_SYNTH_UNROLL 8   // term-loop unroll
#endif
#ifndef QRS_SYNTH_GROUP
#define QRS_SYNTH_GROUP 64   // terms per partial sum
#endif
#ifndef QRS_SYNTH_FOLD
#define QRS_SYNTH_FOLD 1     // 1: fixed-point turns -> radians in one FFMA
#endif
#ifndef QRS_SYNTH_PAIRED
#define QRS_SYNTH_PAIRED 1   // 1: paired FP32 instructions (two points per FFMA2) where they apply
#endif

#ifndef QRS_SYNTH_ANCHOR
#define QRS_SYNTH_ANCHOR 1   // 1: the anchored path where the point groups allow it
#endif

#ifndef QRS_SYNTH_TPB
#define QRS_SYNTH_TPB 128    // threads per CTA
#endif
constexpr int kSynthTPB = QRS_SYNTH_TPB;
constexpr int kSynthPPT = QRS_SYNTH_PPT;
constexpr int kSynthTile = kSynthTPB * kSynthPPT;
constexpr int kSynthChunkMax = 4096;  // terms cached per CTA (64 KB)

// The anchored kernel's own tunables (compile-time; defaults measured best on
// GB300): threads per CTA, points per thread (= the anchor group), minimum
// resident CTAs per SM, terms per shared-memory chunk, term-loop unroll.
#ifndef QRS_ANCHOR_TPB
#define QRS_ANCHOR_TPB 128
#endif
#ifndef QRS_ANCHOR_PPT
#define QRS_ANCHOR_PPT 16
#endif
#ifndef QRS_ANCHOR_MINB
#define QRS_ANCHOR_MINB 3
#endif
#ifndef QRS_ANCHOR_CHUNK
#define QRS_ANCHOR_CHUNK 2048
#endif
#ifndef QRS_ANCHOR_UNROLL
#define QRS_ANCHOR_UNROLL 16
#endif
constexpr int kAnchorTPB = QRS_ANCHOR_TPB;
constexpr int kAnchorPPT = QRS_ANCHOR_PPT;
constexpr int kAnchorTile = kAnchorTPB * kAnchorPPT;
constexpr int kAnchorChunk = QRS_ANCHOR_CHUNK;
constexpr int kAnchorUnroll = QRS_ANCHOR_UNROLL;
static_assert(kAnchorPPT % 2 == 0 && kAnchorPPT >= 2, "anchor groups hold pairs of points");

constexpr int kSynthGroup = QRS_SYNTH_GROUP;
constexpr int kSynthUnroll = QRS_SYNTH_UNROLL;
static_assert(kAnchorChunk % kSynthGroup == 0, "anchored chunks hold whole partial sums");
// Largest a + b of the fixed-point phase: 55 where the paired path can take
// the fraction from the high word, 54 (funnel-shift extraction) otherwise.
constexpr int kSynthMaxAB = (QRS_SYNTH_PAIRED && QRS_SYNTH_FOLD) ? 55 : 54;
// The anchored path needs the radian fold and the paired instructions.
constexpr bool kAnchorBuilt = QRS_SYNTH_ANCHOR && QRS_SYNTH_PAIRED && QRS_SYNTH_FOLD;
constexpr double kAnchorTurns = 8.0;  // ceiling of fbound * dbound on the anchored path
// Shared memory per cached term of the anchored kernel: the 16-byte record
// and {2 pi fx, 2 pi fy, C} with C the term's 64-bit addend of the
// fixed-point phase word (phase offset and rounding bias), formed once in
// the draw instead of once per thread.
constexpr int kAnchorTermBytes = (int)(sizeof(float4) + sizeof(float4));

// The anchor of a point of its group (first point a0, last point a1): the
// nearer in the max norm, ties to a0.  Returns true for a1 and the FP32
// offset from the chosen anchor in d.  The prepass and the kernel call the
// same function, so the offsets the kernel uses are those the prepass bounds.
__device__ __forceinline__ bool anchor_pick(float2 v, float2 a0, float2 a1, float2& d)
{
    const float dx0 = v.x - a0.x, dy0 = v.y - a0.y;
    const float dx1 = v.x - a1.x, dy1 = v.y - a1.y;
    const bool second = fmaxf(fabsf(dx1), fabsf(dy1)) < fmaxf(fabsf(dx0), fabsf(dy0));
    d = second ? make_float2(dx1, dy1) : make_float2(dx0, dy0);
    return second;
}

// Prepass: one CTA computes the point bound max(|x|, |y|) into out[0] and the
// anchor bound (the largest offset of a point from its anchor, over the
// groups of kAnchorPPT consecutive points; +inf if a coordinate is not finite)
// into out[1], without atomics or zeroing; the synthesis kernel reads both
// to pick its phase path and scales.
__global__ void k_point_bound(const float2* __restrict__ xy, int64_t n, float* __restrict__ out)
{
    static_assert(32 % kAnchorPPT == 0, "an anchor group is a whole part of a warp");
    float m = 0.0f, dm = 0.0f;
    bool finite = true;
    const int lane = threadIdx.x & 31;
    const int first = lane & ~(kAnchorPPT - 1);  // lane of the group's first point
    // each pass reads blockDim.x consecutive points (coalesced); a group's
    // points sit in kAnchorPPT neighbouring lanes and meet through shuffles
    // (four passes' loads issued together, so that a single CTA keeps enough
    // of them in flight)
    constexpr int kLoads = 4;
    for (int64_t base = 0; base < n; base += (int64_t)kLoads * blockDim.x) {
        float2 v[kLoads];
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const int64_t i = base + (int64_t)u * blockDim.x + threadIdx.x;
            v[u] = i < n ? xy[i] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const int64_t i = base + (int64_t)u * blockDim.x + threadIdx.x;
            const int64_t g0 = i - (lane - first);
            const int64_t left = n - g0;
            const int nv = left <= 0 ? 1 : (left < kAnchorPPT ? (int)left : kAnchorPPT);
            const float2 a0 = make_float2(__shfl_sync(0xffffffffu, v[u].x, first),
                                          __shfl_sync(0xffffffffu, v[u].y, first));
            const float2 a1 = make_float2(__shfl_sync(0xffffffffu, v[u].x, first + nv - 1),
                                          __shfl_sync(0xffffffffu, v[u].y, first + nv - 1));
            if (i < n) {
                finite = finite && isfinite(v[u].x) && isfinite(v[u].y);
                m = fmaxf(m, fmaxf(fabsf(v[u].x), fabsf(v[u].y)));
                float2 d;
                anchor_pick(v[u], a0, a1, d);
                dm = fmaxf(dm, fmaxf(fabsf(d.x), fabsf(d.y)));
            }
        }
    }
    if (!finite) dm = INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    }
    __shared__ float wmax[2][32];
    if ((threadIdx.x & 31) == 0) {
        wmax[0][threadIdx.x >> 5] = m;
        wmax[1][threadIdx.x >> 5] = dm;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool live = threadIdx.x < (blockDim.x >> 5);
        m = live ? wmax[0][threadIdx.x] : 0.0f;
        dm = live ? wmax[1][threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        }
        if (threadIdx.x == 0) {
            out[0] = m;
            out[1] = dm;
        }
    }
}

cudaError_t launch_point_bound(const float* xy, int64_t n_points, float* d_bound, cudaStream_t s)
{
    k_point_bound<<<1, 1024, 0, s>>>(reinterpret_cast<const float2*>(xy), n_points, d_bound);
    return cudaGetLastError();
}

// The fixed-point path with paired FP32 instructions (FFMA2, two points per
// instruction): the turn-to-radian conversion and the accumulating FMA of
// points 2i and 2i + 1 share one instruction each.  Each element is rounded
// exactly as the scalar fmaf would round it, so the sums are the scalar
// path's bit for bit.  The term's phase offset and the rounding bias form
// the 64-bit addend C of the phase word once per term.  HI: a + b = 55, the
// fraction bits are the low bits of the phase word's high half (no shift).
template <bool HI>
__device__ __forceinline__ void accumulate_chunk_fx_paired(const float4* __restrict__ st, int len,
                                                           const int32_t (&X)[kSynthPPT], const int32_t (&Y)[kSynthPPT],
                                                           float (&acc)[kSynthPPT], const FixedScales& z)
{
    static_assert(kSynthPPT % 2 == 0, "points in pairs");
    constexpr int NP = kSynthPPT / 2;
    const float2 two_pi = make_float2(6.28318530717958648f, 6.28318530717958648f);
    const float2 neg_two_pi = make_float2(-6.28318530717958648f, -6.28318530717958648f);
    for (int k0 = 0; k0 < len; k0 += kSynthGroup) {
        const int k1 = min(k0 + kSynthGroup, len);
        float2 part[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) part[q] = make_float2(0.0f, 0.0f);
#pragma unroll kSynthUnroll
        for (int k = k0; k < k1; ++k) {
            const float4 T = *chk(st, k, (int64_t)len);
            const float2 A = make_float2(T.z, T.z);
            const uint64_t C = (uint64_t)__float_as_uint(T.w) * z.psi_mul + z.bias;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const int32_t Fx = __float_as_int(T.x), Fy = __float_as_int(T.y);
                const uint32_t m0 = HI ? phase_fx_word_hi(Fx, Fy, X[2 * q], Y[2 * q], C)
                                       : phase_fx_word(Fx, Fy, X[2 * q], Y[2 * q], C, z.shift);
                const uint32_t m1 = HI ? phase_fx_word_hi(Fx, Fy, X[2 * q + 1], Y[2 * q + 1], C)
                                       : phase_fx_word(Fx, Fy, X[2 * q + 1], Y[2 * q + 1], C, z.shift);
                const float2 mant = make_float2(__uint_as_float((m0 & 0x007FFFFFu) | 0x3F800000u),
                                                __uint_as_float((m1 & 0x007FFFFFu) | 0x3F800000u));
                const float2 ang = __ffma2_rn(mant, two_pi, neg_two_pi);  // (1 + t) 2 pi - 2 pi
                const float2 c = make_float2(__cosf(ang.x), __cosf(ang.y));
                part[q] = __ffma2_rn(A, c, part[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            acc[2 * q] += part[q].x;
            acc[2 * q + 1] += part[q].y;
        }
    }
}

// The anchored path's term loop.  Per term: the exact phases of the two
// anchors in radians -- fixed point (PH = kAnchorFxHi / kAnchorFx: the
// anchors' int32 coordinates in X0..Y1, [0, 2 pi)) or double-float
// (PH = kAnchorDf: their float bits, |phase| <= 3 pi) -- then per pair of
// points one FFMA2 picks the anchor's phase (S = 0 or 1 against
// D = A1 - A0; exact for S = 0, within one ulp of A1 for S = 1), two FFMA2
// add 2 pi fx dx and 2 pi fy dy, and the cosine and the accumulating FFMA2
// follow as in the exact paths.
constexpr int kAnchorFxHi = 0, kAnchorFx = 1, kAnchorDf = 2;

template <int PH, bool DY0>
__device__ __forceinline__ void accumulate_chunk_anchor(const float4* __restrict__ st, const float4* __restrict__ sw,
                                                        int len, int32_t X0, int32_t Y0, int32_t X1, int32_t Y1,
                                                        const float2 (&DX)[kAnchorPPT / 2],
                                                        const float2 (&DY)[kAnchorPPT / 2],
                                                        const float2 (&S)[kAnchorPPT / 2], float (&acc)[kAnchorPPT],
                                                        const FixedScales& z)
{
    constexpr int NP = kAnchorPPT / 2;
    const float2 two_pi = make_float2(6.28318530717958648f, 6.28318530717958648f);
    const float2 XA = make_float2(__int_as_float(X0), __int_as_float(X1));
    const float2 YA = make_float2(__int_as_float(Y0), __int_as_float(Y1));
    for (int k0 = 0; k0 < len; k0 += kSynthGroup) {
        const int k1 = min(k0 + kSynthGroup, len);
        float2 part[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) part[q] = make_float2(0.0f, 0.0f);
#pragma unroll kAnchorUnroll
        for (int k = k0; k < k1; ++k) {
            const float4 T = *chk(st, k, (int64_t)len);
            const float4 W = *chk(sw, k, (int64_t)len);
            float a0, a1;
            if constexpr (PH == kAnchorDf) {
                const float2 A01 = __fmul2_rn(phase_df2_psi(T.x, T.y, XA, YA, T.w), two_pi);
                a0 = A01.x;
                a1 = A01.y;
            } else {
                const uint64_t C = ((uint64_t)__float_as_uint(W.w) << 32) | (uint64_t)__float_as_uint(W.z);
                const int32_t Fx = __float_as_int(T.x), Fy = __float_as_int(T.y);
                const uint32_t m0 = PH == kAnchorFxHi ? phase_fx_word_hi(Fx, Fy, X0, Y0, C)
                                                      : phase_fx_word(Fx, Fy, X0, Y0, C, z.shift);
                const uint32_t m1 = PH == kAnchorFxHi ? phase_fx_word_hi(Fx, Fy, X1, Y1, C)
                                                      : phase_fx_word(Fx, Fy, X1, Y1, C, z.shift);
                const float2 A01 = __ffma2_rn(make_float2(__uint_as_float((m0 & 0x007FFFFFu) | 0x3F800000u),
                                                          __uint_as_float((m1 & 0x007FFFFFu) | 0x3F800000u)),
                                              two_pi, make_float2(-6.28318530717958648f, -6.28318530717958648f));
                a0 = A01.x;
                a1 = A01.y;
            }
            const float2 A0 = make_float2(a0, a0);
            const float2 D = make_float2(a1 - a0, a1 - a0);
            const float2 TX = make_float2(W.x, W.x), TY = make_float2(W.y, W.y);
            const float2 A = make_float2(T.z, T.z);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 ang = __ffma2_rn(S[q], D, A0);
                ang = __ffma2_rn(TX, DX[q], ang);
                if constexpr (!DY0) ang = __ffma2_rn(TY, DY[q], ang);  // DY0: every dy is 0, fma(ty, 0, a) = a
                const float2 c = make_float2(__cosf(ang.x), __cosf(ang.y));
                part[q] = __ffma2_rn(A, c, part[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            acc[2 * q] += part[q].x;
            acc[2 * q + 1] += part[q].y;
        }
    }
}

// The double-float path with paired FP32 instructions: phase_df2_psi of
// points 2i and 2i + 1 (their coordinates as float bits in X, Y), the
// turn-to-radian product and the accumulating FMA two points at a time, each
// lane rounded as in the scalar path.
__device__ __forceinline__ void accumulate_chunk_df_paired(const float4* __restrict__ st, int len,
                                                           const int32_t (&X)[kSynthPPT], const int32_t (&Y)[kSynthPPT],
                                                           float (&acc)[kSynthPPT])
{
    constexpr int NP = kSynthPPT / 2;
    const float2 two_pi = make_float2(6.28318530717958648f, 6.28318530717958648f);
    float2 px[NP], py[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        px[q] = make_float2(__int_as_float(X[2 * q]), __int_as_float(X[2 * q + 1]));
        py[q] = make_float2(__int_as_float(Y[2 * q]), __int_as_float(Y[2 * q + 1]));
    }
    for (int k0 = 0; k0 < len; k0 += kSynthGroup) {
        const int k1 = min(k0 + kSynthGroup, len);
        float2 part[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) part[q] = make_float2(0.0f, 0.0f);
#pragma unroll kSynthUnroll
        for (int k = k0; k < k1; ++k) {
            const float4 T = *chk(st, k, (int64_t)len);
            const float2 A = make_float2(T.z, T.z);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 ang = __fmul2_rn(phase_df2_psi(T.x, T.y, px[q], py[q], T.w), two_pi);
                const float2 c = make_float2(__cosf(ang.x), __cosf(ang.y));
                part[q] = __ffma2_rn(A, c, part[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            acc[2 * q] += part[q].x;
            acc[2 * q + 1] += part[q].y;
        }
    }
}

template <bool FIXED>
__device__ __forceinline__ void accumulate_chunk(const float4* __restrict__ st, int len, const int32_t (&X)[kSynthPPT],
                                                 const int32_t (&Y)[kSynthPPT], float (&acc)[kSynthPPT],
                                                 const FixedScales& z)
{
    for (int k0 = 0; k0 < len; k0 += kSynthGroup) {
        const int k1 = min(k0 + kSynthGroup, len);
        float part[kSynthPPT];
#pragma unroll
        for (int j = 0; j < kSynthPPT; ++j) part[j] = 0.0f;
#pragma unroll kSynthUnroll
        for (int k = k0; k < k1; ++k) {
            const float4 T = *chk(st, k, (int64_t)len);
            const uint64_t C = FIXED ? (uint64_t)__float_as_uint(T.w) * z.psi_mul + z.bias : 0ull;
#pragma unroll
            for (int j = 0; j < kSynthPPT; ++j) {
                float ang;
                if (FIXED) {
#if QRS_SYNTH_FOLD
                    ang = phase_fx_rad(__float_as_int(T.x), __float_as_int(T.y), X[j], Y[j], C, z.shift);
#else
                    ang = phase_fx(__float_as_int(T.x), __float_as_int(T.y), X[j], Y[j], C, z.shift) *
                          6.28318530717958648f;
#endif
                } else {
                    ang = phase_df_psi(T.x, T.y, __int_as_float(X[j]), __int_as_float(Y[j]), T.w) *
                          6.28318530717958648f;
                }
                part[j] = fmaf(T.z, __cosf(ang), part[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kSynthPPT; ++j) acc[j] += part[j];
    }
}

// Draws terms [k_begin, k_begin + len) of realisation r into the CTA's
// shared-memory records (and, for the anchored path, 2 pi (fx, fy) and the
// fixed-point addend C).
template <int TPB>
__device__ __forceinline__ void draw_chunk(const DrawParams& p, const FixedScales& z, int64_t r, int64_t k_begin,
                                           int len, int chunk, float4* __restrict__ sterm, float4* __restrict__ sw,
                                           bool anchored)
{
    const uint64_t n0 = (uint64_t)(p.real_offset + r) * (uint64_t)p.n_f + (uint64_t)k_begin;
    for (int q = threadIdx.x; q < len; q += TPB) {
        Words w;
        const Term t = draw_term<false, false>(p, n0 + (uint64_t)q, k_begin + q, &w);
        float amp;
        uint32_t u;
        coef_polar_from_words(p, n0 + (uint64_t)q, w, amp, u);
        float4 rec;
        if (z.use_fixed) {
            rec.x = __int_as_float(__float2int_rn(t.fx * z.fscale));
            rec.y = __int_as_float(__float2int_rn(t.fy * z.fscale));
            rec.w = __uint_as_float(u);
        } else {
            rec.x = t.fx;
            rec.y = t.fy;
            rec.w = (float)u * 0x1p-24f;
        }
        rec.z = t.F * amp;
        *chk(sterm, q, (int64_t)chunk) = rec;
        if (anchored) {
            const uint64_t C = z.use_fixed ? (uint64_t)u * z.psi_mul + z.bias : 0ull;
            *chk(sw, q, (int64_t)chunk) = make_float4(t.fx * 6.28318530717958648f, t.fy * 6.28318530717958648f,
                                                      __uint_as_float((uint32_t)C), __uint_as_float((uint32_t)(C >> 32)));
        }
    }
}

// The exact paths: a thread's points strided by the CTA width (coalesced),
// each (point, term) phase formed in full.
__device__ __forceinline__ void synth_items_exact(const DrawParams& p, const float2* __restrict__ xy, int64_t P,
                                                  float* __restrict__ out, const FixedScales& z, int chunk,
                                                  int64_t n_tiles, int64_t n_items, float4* __restrict__ sterm)
{
    const int64_t G = gridDim.x;
    const int64_t it0 = (n_items * (int64_t)blockIdx.x) / G;
    const int64_t it1 = (n_items * ((int64_t)blockIdx.x + 1)) / G;
    const int n_chunks = (int)((p.n_f + chunk - 1) / chunk);
    int64_t cached_r = -1;
    int cached_c = -1;
    for (int64_t item = it0; item < it1; ++item) {
        const int64_t r = item / n_tiles;
        const int64_t tile = item - r * n_tiles;
        const int64_t base = tile * kSynthTile;
        int32_t X[kSynthPPT], Y[kSynthPPT];
        float acc[kSynthPPT];
#pragma unroll
        for (int j = 0; j < kSynthPPT; ++j) {
            const int64_t m = base + j * kSynthTPB + threadIdx.x;
            const float2 v = (m < P) ? *chk(xy, m, P) : make_float2(0.0f, 0.0f);
            if (z.use_fixed) {
                X[j] = __float2int_rn(v.x * z.xscale);
                Y[j] = __float2int_rn(v.y * z.xscale);
            } else {
                X[j] = __float_as_int(v.x);
                Y[j] = __float_as_int(v.y);
            }
            acc[j] = 0.0f;
        }
        for (int c = 0; c < n_chunks; ++c) {
            const int64_t k_begin = (int64_t)c * chunk;
            const int len = (int)min((int64_t)chunk, p.n_f - k_begin);
            if (r != cached_r || c != cached_c) {
                __syncthreads();  // previous chunk fully consumed
                draw_chunk<kSynthTPB>(p, z, r, k_begin, len, chunk, sterm, nullptr, false);
                __syncthreads();
                cached_r = r;
                cached_c = c;
            }
            if (z.use_fixed) {
#if QRS_SYNTH_PAIRED && QRS_SYNTH_FOLD
                if (z.shift == 32) accumulate_chunk_fx_paired<true>(sterm, len, X, Y, acc, z);
                else accumulate_chunk_fx_paired<false>(sterm, len, X, Y, acc, z);
#else
                accumulate_chunk<true>(sterm, len, X, Y, acc, z);
#endif
            } else {
#if QRS_SYNTH_PAIRED
                accumulate_chunk_df_paired(sterm, len, X, Y, acc);
#else
                accumulate_chunk<false>(sterm, len, X, Y, acc, z);
#endif
            }
        }
        const int64_t n_out = (n_items / n_tiles) * P;
#pragma unroll
        for (int j = 0; j < kSynthPPT; ++j) {
            const int64_t m = base + j * kSynthTPB + threadIdx.x;
            if (m < P) *chk(out, r * P + m, n_out) = acc[j];
        }
    }
}

// Whether the anchored path applies to a launch: every point lies within
// dbound of its anchor with fbound * dbound <= kAnchorTurns (the anchors'
// phases are exact on either reduction, so the point bound does not enter).  Both kernels evaluate it from the same
// prepass output, so exactly one of them does the work.
__device__ __forceinline__ bool anchor_applies(const FixedScales& z, float fbound, const float* d_bound,
                                               int allow_anchor)
{
    (void)z;
    return kAnchorBuilt && allow_anchor != 0 && (double)fbound * (double)d_bound[1] <= kAnchorTurns;
}

// The anchored kernel.  Work items and their split over the persistent grid
// are those of k_synth_fused (realisation-major (realisation, tile) items, one
// contiguous range per CTA), with tiles of kAnchorTPB x kAnchorPPT points and
// each thread's kAnchorPPT consecutive points one anchor group.  The terms
// are taken chunk by chunk for each realisation of the range: the CTA draws a
// chunk once and runs every tile of that realisation through it, carrying each
// point's running sum from chunk to chunk in `out` (an FP32 store and reload,
// so the sums are those of one pass over all terms).  Chunks therefore stay
// small (kAnchorChunk terms) and several CTAs fit on an SM.
// d_bound: [0] the point bound, [1] the anchor bound (k_point_bound).
__global__ void __launch_bounds__(kAnchorTPB, QRS_ANCHOR_MINB) k_synth_anchor(DrawParams p, const float2* __restrict__ xy,
                                                              int64_t P, float* __restrict__ out,
                                                              const float* __restrict__ d_bound, float fbound,
                                                              int chunk, int64_t n_tiles, int64_t n_items,
                                                              int allow_anchor)
{
    extern __shared__ float4 sterm[];
    float4* sw = reinterpret_cast<float4*>(sterm + chunk);
    const FixedScales z = fixed_scales(fbound, d_bound[0], true, kSynthMaxAB);
    if (!anchor_applies(z, fbound, d_bound, allow_anchor)) return;  // k_synth_fused does the work
    constexpr int NP = kAnchorPPT / 2;
    const int64_t G = gridDim.x;
    const int64_t it0 = (n_items * (int64_t)blockIdx.x) / G;
    const int64_t it1 = (n_items * ((int64_t)blockIdx.x + 1)) / G;
    const int n_chunks = (int)((p.n_f + chunk - 1) / chunk);
    const int64_t n_out = (n_items / n_tiles) * P;
    for (int64_t seg = it0; seg < it1;) {
        const int64_t r = seg / n_tiles;
        const int64_t seg_end = min(it1, (r + 1) * n_tiles);  // this range's items of realisation r
        for (int c = 0; c < n_chunks; ++c) {
            const int64_t k_begin = (int64_t)c * chunk;
            const int len = (int)min((int64_t)chunk, p.n_f - k_begin);
            __syncthreads();  // previous chunk fully consumed
            draw_chunk<kAnchorTPB>(p, z, r, k_begin, len, chunk, sterm, sw, true);
            __syncthreads();
            for (int64_t item = seg; item < seg_end; ++item) {
                const int64_t tile = item - r * n_tiles;
                const int64_t g0 = tile * kAnchorTile + (int64_t)threadIdx.x * kAnchorPPT;
                const int64_t rem = P - g0;
                const int nv = rem <= 0 ? 0 : (rem < kAnchorPPT ? (int)rem : kAnchorPPT);  // valid points
                const float2 a0 = nv > 0 ? *chk(xy, g0, P) : make_float2(0.0f, 0.0f);
                const float2 a1 = nv > 0 ? *chk(xy, g0 + nv - 1, P) : make_float2(0.0f, 0.0f);
                // the anchors as the phase reduction takes them: int32 at scale 2^b, or float bits
                const int32_t X0 = z.use_fixed ? __float2int_rn(a0.x * z.xscale) : __float_as_int(a0.x);
                const int32_t Y0 = z.use_fixed ? __float2int_rn(a0.y * z.xscale) : __float_as_int(a0.y);
                const int32_t X1 = z.use_fixed ? __float2int_rn(a1.x * z.xscale) : __float_as_int(a1.x);
                const int32_t Y1 = z.use_fixed ? __float2int_rn(a1.y * z.xscale) : __float_as_int(a1.y);
                float2 DX[NP], DY[NP], S[NP];
                float acc[kAnchorPPT];
                bool dy0 = true;  // every point on its anchor's row (grids in row order, tracks along x)
#pragma unroll
                for (int j = 0; j < kAnchorPPT; ++j) {
                    float2 d = make_float2(0.0f, 0.0f);
                    const bool second = j < nv && anchor_pick(*chk(xy, g0 + j, P), a0, a1, d);
                    if (j & 1) {
                        DX[j >> 1].y = d.x;
                        DY[j >> 1].y = d.y;
                        S[j >> 1].y = second ? 1.0f : 0.0f;
                    } else {
                        DX[j >> 1].x = d.x;
                        DY[j >> 1].x = d.y;
                        S[j >> 1].x = second ? 1.0f : 0.0f;
                    }
                    acc[j] = (c > 0 && j < nv) ? *chk(out, r * P + g0 + j, n_out) : 0.0f;
                    dy0 = dy0 && d.y == 0.0f;
                }
                // a warp whose offsets are all along x drops the y product: the
                // same sums bit for bit, one paired instruction fewer per pair
                dy0 = __all_sync(0xffffffffu, dy0);
                if (nv == 0) continue;  // past the last point (the last tile's idle warps skip the terms)
                if (!z.use_fixed) {
                    if (dy0) accumulate_chunk_anchor<kAnchorDf, true>(sterm, sw, len, X0, Y0, X1, Y1, DX, DY, S, acc, z);
                    else accumulate_chunk_anchor<kAnchorDf, false>(sterm, sw, len, X0, Y0, X1, Y1, DX, DY, S, acc, z);
                } else if (z.shift == 32) {
                    if (dy0) accumulate_chunk_anchor<kAnchorFxHi, true>(sterm, sw, len, X0, Y0, X1, Y1, DX, DY, S, acc, z);
                    else accumulate_chunk_anchor<kAnchorFxHi, false>(sterm, sw, len, X0, Y0, X1, Y1, DX, DY, S, acc, z);
                } else {
                    if (dy0) accumulate_chunk_anchor<kAnchorFx, true>(sterm, sw, len, X0, Y0, X1, Y1, DX, DY, S, acc, z);
                    else accumulate_chunk_anchor<kAnchorFx, false>(sterm, sw, len, X0, Y0, X1, Y1, DX, DY, S, acc, z);
                }
#pragma unroll
                for (int j = 0; j < kAnchorPPT; ++j)
                    if (j < nv) *chk(out, r * P + g0 + j, n_out) = acc[j];
            }
        }
        seg = seg_end;
    }
}

// The exact kernel.  d_bound: [0] the point bound, [1] the anchor bound
// (k_point_bound); it returns at once where the anchored path applies
// (k_synth_anchor, launched beside it, does the work).
__global__ void __launch_bounds__(kSynthTPB, QRS_SYNTH_MINB) k_synth_fused(DrawParams p, const float2* __restrict__ xy, int64_t P,
                                                           float* __restrict__ out, const float* __restrict__ d_bound,
                                                           float fbound, int chunk, int64_t n_tiles, int64_t n_items,
                                                           int allow_anchor)
{
    extern __shared__ float4 sterm[];
    const FixedScales z = fixed_scales(fbound, d_bound[0], QRS_SYNTH_FOLD != 0, kSynthMaxAB);
    if (anchor_applies(z, fbound, d_bound, allow_anchor)) return;  // use_fixed does not depend on the fold
    synth_items_exact(p, xy, P, out, z, chunk, n_tiles, n_items, sterm);
}

// The fused form after the prepass has written d_bound[0..1]: the anchored
// kernel and the exact kernel, each a persistent grid of num_sms x its
// resident CTAs per SM; the one whose path does not apply returns at once.
static cudaError_t launch_fused_kernel(int num_sms, const float* d_bound, const DrawParams& p, const float* xy,
                                      int64_t n_points, int64_t n_real, float* out, int allow_anchor, cudaStream_t s,
                                      int64_t* launched = nullptr)
{
    const float fbound = (float)freq_bound(p);
    if (kAnchorBuilt && allow_anchor) {
        const int chunk = (int)(p.n_f < kAnchorChunk ? p.n_f : kAnchorChunk);
        const size_t smem = (size_t)chunk * kAnchorTermBytes;
        cudaError_t e = cudaFuncSetAttribute(k_synth_anchor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kAnchorChunk * kAnchorTermBytes);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_synth_anchor, kAnchorTPB, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        const int64_t n_tiles = (n_points + kAnchorTile - 1) / kAnchorTile;
        const int64_t n_items = n_tiles * n_real;
        int64_t grid = (int64_t)num_sms * per_sm;
        if (grid > n_items) grid = n_items;
        k_synth_anchor<<<(unsigned)grid, kAnchorTPB, smem, s>>>(p, reinterpret_cast<const float2*>(xy), n_points,
                                                                out, d_bound, fbound, chunk, n_tiles, n_items,
                                                                allow_anchor);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launched) ++*launched;
    }
    const int chunk = (int)(p.n_f < kSynthChunkMax ? p.n_f : kSynthChunkMax);
    const size_t smem = (size_t)chunk * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_synth_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSynthChunkMax * sizeof(float4)));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_synth_fused, kSynthTPB, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t n_tiles = (n_points + kSynthTile - 1) / kSynthTile;
    const int64_t n_items = n_tiles * n_real;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > n_items) grid = n_items;
    k_synth_fused<<<(unsigned)grid, kSynthTPB, smem, s>>>(p, reinterpret_cast<const float2*>(xy), n_points, out,
                                                          d_bound, fbound, chunk, n_tiles, n_items, allow_anchor);
    return cudaGetLastError();
}

cudaError_t launch_synth_fused(qrs_handle* h, const DrawParams& p, const float* xy, int64_t n_points, int64_t n_real,
                               float* out, cudaStream_t s)
{
    cudaError_t e = launch_point_bound(xy, n_points, h->d_xbound, s);
    if (e != cudaSuccess) return e;
    ++h->launches;
    return launch_fused_kernel(h->num_sms, h->d_xbound, p, xy, n_points, n_real, out, h->synth_anchor, s,
                               &h->launches);
}

}  // namespace qrs

namespace qrs {

// Same two launches as launch_synth_fused (point-bound prepass, then the fused
// kernel), for callers that bring their own device scratch instead of a
// handle: `d_bound` (two floats) receives the point and anchor bounds;
// `num_sms` sizes the grid; allow_anchor as the handle's switch.
cudaError_t launch_synth_fused_raw(int num_sms, float* d_bound, const DrawParams& p, const float* xy,
                                   int64_t n_points, int64_t n_real, float* out, int allow_anchor, cudaStream_t s)
{
    cudaError_t e = launch_point_bound(xy, n_points, d_bound, s);
    if (e != cudaSuccess) return e;
    return launch_fused_kernel(num_sms, d_bound, p, xy, n_points, n_real, out, allow_anchor, s);
}

}  // namespace qrs
