// k_gemm.cu -- K3: the shared-draw form of Eq. 3 as a tensor-core GEMM.
//
// When a batch of R realisations shares one frequency draw (the frequencies
// of realisation real_offset; each column r has its own coefficients and
// optionally its own r0, L0), Eq. 3 for all points and columns is one matrix
// product
//     out^T[m][r] = sum_k' A[m][k'] B[r][k'],   k' over 2 N_f,
//     A = [cos 2 pi phi_mk | sin 2 pi phi_mk]       (the basis; points x 2 N_f)
//     B = [F_kr a_kr | -F_kr b_kr]                  (coefficients; R x 2 N_f)
// computed on the 5th-generation tensor cores in split precision:
//   3XTF32: x = hi + lo with hi, lo TF32 (11-bit significands); the product is
//           A_hi B_hi + A_hi B_lo + A_lo B_hi (kind::tf32), ~FP32 accuracy.
//   BF16X3: the same with BF16 halves (kind::f16, BF16 in, FP32 accumulate).
//   TF32:   single pass, each operand rounded once to TF32, A B (kind::tf32):
//           about 2^-11 relative per product, several 1e-4 of the field's
//           standard deviation per value.
//
// Launches: k_point_bound (phase path), k_gemm_freq (the shared draw, FP64
// map, into the basis representation), k_gemm_coef (B, hi and lo, into the
// workspace, K'-contiguous rows so TMA can stream them), k_gemm_main.
//
// k_gemm_main: a persistent grid, one CTA per SM, walking work items
// (256-column block, 128-point tile), tile fastest, so the CTAs at work at
// one time share a column block's coefficient tiles in L2.  Warps:
//   warp 0      TMA producer: B_hi and B_lo tiles (256 rows x 128 B, 128-byte
//               swizzle) per K chunk into a 2-stage ring (mbarrier complete_tx);
//   warp 1      TMEM allocator (512 columns: two 128 x 256 FP32 segment
//               slots) and single-thread MMA issuer: 3 x 4 tcgen05.mma per K
//               chunk into the segment's slot, one commit per segment of kSeg
//               chunks (6 TF32, 8 BF16, 18 single TF32); the slots alternate,
//               so the MMAs never wait for a promotion;
//   warp 2      frequency ring: bulk-copies each chunk's basis frequencies
//               into an 8-slot shared-memory ring, up to 8 chunks ahead;
//   warps 4-11  promoters, two per TMEM lane quarter (128 columns each): after
//               each segment they hand the slot to the CTA's FP32 master in L2
//               (promote_red: := slot, then += slot by FP32 reductions in L2),
//               free the slot, and after an item's last segment store
//               out[r][m] = slot + master (coalesced over m).  The tensor
//               core's accumulation loses about 2^-26 per step with a
//               consistent sign, so long chains drift; segments bound it;
//   warps 12-   basis producers, two or four per 32-row block, each taking a
//               share of the chunk's terms: evaluate cos/sin (fixed-point or
//               double-float phase, MUFU sin/cos), split hi/lo and write their
//               16-byte pieces of the row in the swizzled A tiles,
//               fence.proxy.async, one arrival per warp.
// Every mbarrier wait is bounded in time; on time-out the CTA raises an abort
// flag, records QRS_ERR_TIMEOUT in the device error word, waits (bounded) for
// its TMA copies and MMAs in flight, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "qrs_internal.h"
#include "qrs_sm100.cuh"
#include "qrs_tc_split.cuh"

// Basis producer warps (4: one per row block; 8 / 16: two / four, splitting
// the terms) and the TMEM columns a promoter thread holds at a time (32 or
// 16), per precision: BF16X3 has twice the basis elements per K chunk and
// gains from 16 producers (promoters then read 16 columns to fit the
// registers); 3XTF32 is fastest with 8; single-pass TF32, with a third of
// the MMA work per chunk, with 16 (its promoters also read 16 columns).
#ifndef QRS_GEMM_PRODUCERS_TF32
#define QRS_GEMM_PRODUCERS_TF32 8
#endif
#ifndef QRS_GEMM_PRODUCERS_BF16
#define QRS_GEMM_PRODUCERS_BF16 16
#endif
#ifndef QRS_GEMM_PRODUCERS_TF32_SINGLE
#define QRS_GEMM_PRODUCERS_TF32_SINGLE 16  // one product per K chunk: the basis is the pace (8.15 -> 7.45 ms)
#endif
#ifndef QRS_GEMM_PROMOTE_COLS_TF32
#define QRS_GEMM_PROMOTE_COLS_TF32 32
#endif
#ifndef QRS_GEMM_PROMOTE_COLS_BF16
#define QRS_GEMM_PROMOTE_COLS_BF16 16
#endif

namespace qrs {

QRS_CHECK_HOOK(check_hook_gemm)

constexpr int kGM = 128;                                   // points per tile (UMMA M, TMEM lanes)
constexpr int kGN = 256;                                   // columns per block (UMMA N)
constexpr int kGStages = 2;
constexpr int kGTileA = kGM * 128;                         // 16 KB
constexpr int kGTileB = kGN * 128;                         // 32 KB
constexpr int kGStageBytes = 2 * kGTileA + 2 * kGTileB;    // A hi/lo + B hi/lo = 96 KB
constexpr int kGFreqSlots = 8;                             // frequency ring, filled ahead by warp 2
constexpr int kGFreqBytes = 256;                           // one chunk's basis frequencies (<= 32 x 8 B)
constexpr int kGPromoters = 8;                             // promoter warps, two per TMEM lane quarter
template <int PREC>
struct GemmShape {
    static constexpr bool kBF16 = !GemmCfg<PREC>::kTF32;
    static constexpr bool kSingle = !GemmCfg<PREC>::kSplit;  // single-pass TF32
    static constexpr int kProducers =
        kBF16 ? QRS_GEMM_PRODUCERS_BF16 : (kSingle ? QRS_GEMM_PRODUCERS_TF32_SINGLE : QRS_GEMM_PRODUCERS_TF32);
    static constexpr int kPromoteCols = (kBF16 || kSingle) ? QRS_GEMM_PROMOTE_COLS_BF16 : QRS_GEMM_PROMOTE_COLS_TF32;
    static constexpr int kThreads = 128 + 32 * (kGPromoters + kProducers);
    static constexpr bool kTmemMaster = GemmCfg<PREC>::kTF32 && GemmCfg<PREC>::kSplit;  // 3XTF32
    static_assert(kProducers == 4 || kProducers == 8 || kProducers == 16, "producer warps");
    static_assert(kPromoteCols == 32 || kPromoteCols == 16, "promotion width");
};
constexpr int kGSmemBytes = kGStages * kGStageBytes + kGFreqSlots * kGFreqBytes + 512 + 1024;  // + barriers, slack
constexpr long long kGWaitCycles = 4000000000LL;           // ~2 s of SM clock per wait

struct GemmArgs {
    const float2* xy;
    int64_t P;
    float* out;
    int64_t n_real;     // valid columns
    int64_t R_pad;      // rows of each B half (multiple of 256)
    int64_t n_chunks;   // K chunks (2 N_f_pad / elements per row)
    int64_t n_tiles;    // 128-point tiles
    int64_t n_items;    // work items (column block, point tile), tile fastest
    float* master;      // [gridDim.x][4][256][32] FP32 segment sums of the CTAs' current items (L2)
    const int2* fbasis; // [N_f_pad] basis frequency (Fx, Fy) or float bits (fx, fy)
    const float* d_xbound;
    float fbound;
    int* err;
    long long inject_wait;  // > 0: the MMA thread first waits this many cycles on a barrier nothing arrives at
};

// ------------------------------------------------------------- prep kernels
// The shared draw: frequencies of realisation real_offset in the basis
// representation, and (|f|^2, J, A) for the weights (A: the aperture filter, 1 if none).
__global__ void k_gemm_freq(DrawParams p, int64_t nf_pad, const float* __restrict__ d_xbound, float fbound,
                            int2* __restrict__ fbasis, float4* __restrict__ fw)
{
    const FixedScales z = fixed_scales(fbound, *d_xbound, true);
    const uint64_t n0 = (uint64_t)p.real_offset * (uint64_t)p.n_f;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nf_pad; k += (int64_t)gridDim.x * blockDim.x) {
        if (k < p.n_f) {
            const Term t = draw_term<false>(p, n0 + (uint64_t)k, k);
            if (z.use_fixed)
                *chk(fbasis, k, nf_pad) = make_int2(__float2int_rn(t.fx * z.fscale), __float2int_rn(t.fy * z.fscale));
            else
                *chk(fbasis, k, nf_pad) = make_int2(__float_as_int(t.fx), __float_as_int(t.fy));
            *chk(fw, k, nf_pad) = make_float4(t.fx * t.fx + t.fy * t.fy, t.J, t.A, 0.0f);
        } else {
            *chk(fbasis, k, nf_pad) = make_int2(0, 0);
            *chk(fw, k, nf_pad) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
}

template <int PREC>
__device__ __forceinline__ void split_store(void* hi_base, void* lo_base, int64_t idx, int64_t n, float x)
{
    if (!chk_ok(idx, 1, n)) return;
    if (!GemmCfg<PREC>::kSplit) {  // single pass: the TF32 rounding only
        static_cast<uint32_t*>(hi_base)[idx] = tf32_rna_bits(x);
    } else if (GemmCfg<PREC>::kTF32) {
        uint32_t h, l;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
        const float r = x - __uint_as_float(h);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
        static_cast<uint32_t*>(hi_base)[idx] = h;
        static_cast<uint32_t*>(lo_base)[idx] = l;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        static_cast<__nv_bfloat16*>(hi_base)[idx] = h;
        static_cast<__nv_bfloat16*>(lo_base)[idx] = l;
    }
}

// B[r][k'] (hi half then lo half, R_pad rows each, 2 nf_pad columns; the hi
// half only for single-pass TF32):
// chunk c holds terms [c T, (c+1) T); column c 2T + j = cos part (F a) of
// term c T + j, column c 2T + T + j = sin part (-F b).  Column r draws its
// coefficients from stream point (real_offset + r) N_f + k; its weight uses
// (r0, L0) = col_psd[r] when given.  Rows r >= n_real and terms k >= N_f are 0.
template <int PREC>
__global__ void k_gemm_coef(DrawParams p, int64_t nf_pad, int64_t n_real, int64_t R_pad,
                            const float4* __restrict__ fw, const double* __restrict__ col_psd, double c_vk,
                            void* __restrict__ B)
{
    constexpr int T = GemmCfg<PREC>::kTermsPerChunk;
    const int64_t r = blockIdx.y;
    __shared__ float s_c, s_a;
    if (threadIdx.x == 0) {
        if (col_psd && r < n_real) {
            const double r0 = *chk(col_psd, 2 * r, 2 * n_real), L0 = *chk(col_psd, 2 * r + 1, 2 * n_real);
            s_c = (float)(c_vk * pow(r0, -5.0 / 3.0));
            s_a = p.psd_a == 0.0f ? 0.0f : (float)(1.0 / (L0 * L0));
        } else {
            s_c = p.psd_c;
            s_a = p.psd_a;
        }
    }
    __syncthreads();
    const float pc = s_c, pa = s_a;
    const int64_t Kp = 2 * nf_pad;
    unsigned char* hi = static_cast<unsigned char*>(B);
    unsigned char* lo = hi + (size_t)R_pad * Kp * GemmCfg<PREC>::kElemBytes;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nf_pad; k += (int64_t)gridDim.x * blockDim.x) {
        float cc = 0.0f, cs = 0.0f;
        if (r < n_real && k < p.n_f) {
            const float4 w = *chk(fw, k, nf_pad);
            const float F = sqrtf(psd_w(pc, pa, w.x) * w.y * p.inv_nf) * w.z;  // w.z: aperture filter
            const float2 ab = draw_coef(p, (uint64_t)(p.real_offset + r) * (uint64_t)p.n_f + (uint64_t)k);
            cc = F * ab.x;
            cs = -(F * ab.y);
        }
        const int64_t c = k / T, j = k - c * T;
        const int64_t row = r * Kp;
        split_store<PREC>(hi, lo, row + c * 2 * T + j, R_pad * Kp, cc);
        split_store<PREC>(hi, lo, row + c * 2 * T + T + j, R_pad * Kp, cs);
    }
}

// ------------------------------------------------------------ main kernel
// One producer thread's share of a K chunk's A tile: basis row `row` (the
// point with scaled coordinates X, Y / float coordinates pt), 16-byte term
// groups [grp0, grp0 + NG) of the cos half and of the sin half, split hi/lo
// into the swizzled tiles.
template <int PREC, int NG>
__device__ __forceinline__ void produce_basis(const int2* __restrict__ fb, unsigned char* Ahi, unsigned char* Alo,
                                              int row, int grp0, const FixedScales& z, int32_t X, int32_t Y, float2 pt)
{
    using Cfg = GemmCfg<PREC>;
    constexpr int TPG = Cfg::kTermsPer16B;
    const float2 two_pi = make_float2(6.28318530717958648f, 6.28318530717958648f);
    const float2 neg_two_pi = make_float2(-6.28318530717958648f, -6.28318530717958648f);
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
        const int grp = grp0 + gi;
        float cv[TPG], sv[TPG];
#pragma unroll
        for (int t = 0; t < TPG; t += 2) {  // two terms per paired FP32 instruction
            const int2 f0 = *chk(fb, grp * TPG + t, Cfg::kTermsPerChunk);
            const int2 f1 = *chk(fb, grp * TPG + t + 1, Cfg::kTermsPerChunk);
            float2 ang;
            if (z.use_fixed) {
                const uint32_t m0 = phase_fx_word(f0.x, f0.y, X, Y, z.bias, z.shift);
                const uint32_t m1 = phase_fx_word(f1.x, f1.y, X, Y, z.bias, z.shift);
                ang = __ffma2_rn(make_float2(__uint_as_float((m0 & 0x007FFFFFu) | 0x3F800000u),
                                             __uint_as_float((m1 & 0x007FFFFFu) | 0x3F800000u)),
                                 two_pi, neg_two_pi);
            } else {
                ang = __fmul2_rn(phase_df2f(make_float2(__int_as_float(f0.x), __int_as_float(f1.x)),
                                            make_float2(__int_as_float(f0.y), __int_as_float(f1.y)), pt.x, pt.y),
                                 two_pi);
            }
            sv[t] = __sinf(ang.x);
            cv[t] = __cosf(ang.x);
            sv[t + 1] = __sinf(ang.y);
            cv[t + 1] = __cosf(ang.y);
        }
        const uint32_t oc = sm100::sw128_offset((uint32_t)row, (uint32_t)grp);
        const uint32_t os = sm100::sw128_offset((uint32_t)row, (uint32_t)(4 + grp));
        uint4 hi, lo;
        pack16<PREC>(cv, hi, lo);
        if (chk_ok(oc, 16, kGTileA)) {
            *reinterpret_cast<uint4*>(Ahi + oc) = hi;
            if (Cfg::kSplit) *reinterpret_cast<uint4*>(Alo + oc) = lo;
        }
        pack16<PREC>(sv, hi, lo);
        if (chk_ok(os, 16, kGTileA)) {
            *reinterpret_cast<uint4*>(Ahi + os) = hi;
            if (Cfg::kSplit) *reinterpret_cast<uint4*>(Alo + os) = lo;
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(GemmShape<PREC>::kThreads, 1) k_gemm_main(const __grid_constant__ CUtensorMap tmapB,
                                                                           GemmArgs g)
{
    using Cfg = GemmCfg<PREC>;
    constexpr int kGProducers = GemmShape<PREC>::kProducers;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* fring = smem + kGStages * kGStageBytes;
    uint64_t* fullA = reinterpret_cast<uint64_t*>(fring + kGFreqSlots * kGFreqBytes);
    uint64_t* fullB = fullA + kGStages;
    uint64_t* empty = fullB + kGStages;
    uint64_t* seg_full = empty + kGStages;  // [2], one per TMEM segment slot
    uint64_t* seg_free = seg_full + 2;      // [2]
    uint64_t* fullF = seg_free + 2;
    uint64_t* freeF = fullF + kGFreqSlots;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(freeF + kGFreqSlots);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint64_t* never = reinterpret_cast<uint64_t*>(tmem_slot + 2);  // fault injection: no thread arrives here

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_chunks = g.n_chunks;
    const int64_t n_seg = (n_chunks + Cfg::kSeg - 1) / Cfg::kSeg;
    // 3XTF32 keeps its FP32 master in TMEM (one slot, the MMAs wait for each
    // promotion; no memory traffic beside its operand streams), the other
    // modes in L2 (two slots, the MMAs never wait; promote_red) -- whichever
    // measured faster.  Segment J's slot, and the parities of its barriers:
    constexpr bool kTmemMaster = GemmShape<PREC>::kTmemMaster;
    auto slot_of = [](int64_t J) { return kTmemMaster ? 0 : (int)(J & 1); };
    auto use_of = [](int64_t J) { return (uint32_t)((kTmemMaster ? J : (J >> 1)) & 1); };  // J-th use of its slot

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            sm100::mbar_init(&fullA[s], kGProducers);  // one arrival per producer warp
            sm100::mbar_init(&fullB[s], 1);
            sm100::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            sm100::mbar_init(&seg_full[b], 1);
            sm100::mbar_init(&seg_free[b], kGPromoters);  // one arrival per promoter warp
        }
        for (int s = 0; s < kGFreqSlots; ++s) {
            sm100::mbar_init(&fullF[s], 1);
            sm100::mbar_init(&freeF[s], kGProducers);
        }
        sm100::mbar_init(never, 1);
        *abort_flag = 0;
        sm100::fence_barrier_init();
    }
    if (warp == 1) sm100::tmem_alloc(tmem_slot, 512);
    if (warp == 0 && lane == 0) sm100::prefetch_tmap(&tmapB);
    sm100::tc_fence_before();
    __syncthreads();
    sm100::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;  // two 256-column regions: slots 0, 1 (or master, slot)

    auto stageA_hi = [&](int s) { return smem + s * kGStageBytes; };
    auto stageA_lo = [&](int s) { return smem + s * kGStageBytes + kGTileA; };
    auto stageB_hi = [&](int s) { return smem + s * kGStageBytes + 2 * kGTileA; };
    auto stageB_lo = [&](int s) { return smem + s * kGStageBytes + 2 * kGTileA + kGTileB; };
    auto ringF = [&](int64_t i) { return fring + (i % kGFreqSlots) * kGFreqBytes; };
    auto timeout = [&]() {
        *abort_flag = 1;
        atomicExch(g.err, (int)QRS_ERR_TIMEOUT);
    };
    int64_t mma_segments = 0;  // segments the MMA thread committed (teardown)
    constexpr uint32_t kFreqChunkBytes = Cfg::kTermsPerChunk * sizeof(int2);
    static_assert(kFreqChunkBytes <= kGFreqBytes, "frequency chunk fits its ring slot");

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer
        if (lane == 0) {
            int64_t gc = 0, issued = 0;
            bool stop = false;
            for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
                const int64_t rblk = it / g.n_tiles;
                for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                    const int s = (int)(gc % kGStages);
                    const uint32_t ph = (uint32_t)((gc / kGStages) & 1);
                    if (*abort_flag || (gc >= kGStages && !sm100::mbar_wait(&empty[s], ph ^ 1u, abort_flag, kGWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    sm100::mbar_arrive_expect_tx(&fullB[s], (Cfg::kSplit ? 2u : 1u) * kGTileB);
                    const int32_t x = (int32_t)(i * Cfg::kElemsPerRow);
                    sm100::tma_load_2d(stageB_hi(s), &tmapB, &fullB[s], x, (int32_t)(rblk * kGN));
                    if (Cfg::kSplit)
                        sm100::tma_load_2d(stageB_lo(s), &tmapB, &fullB[s], x, (int32_t)(g.R_pad + rblk * kGN));
                    issued = gc + 1;
                }
            }
            if (*abort_flag) {  // let copies in flight land before the CTA exits
                for (int64_t i = (issued > kGStages ? issued - kGStages : 0); i < issued; ++i)
                    sm100::mbar_wait_for(&fullB[i % kGStages], (uint32_t)((i / kGStages) & 1), kGWaitCycles / 8);
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = sm100::idesc_f32acc(Cfg::kFormat, kGM, kGN);
            // Host-side fault injection (QRS_FAULT=timeout): a bounded wait that
            // runs out before any MMA is issued; the CTA then unwinds through its
            // time-out path (abort flag, error word, drained copies, TMEM freed).
            if (g.inject_wait > 0 && !sm100::mbar_wait(never, 0u, abort_flag, g.inject_wait) && !*abort_flag)
                timeout();
            int64_t J = 0, gc = 0;
            bool stop = *abort_flag != 0;
            for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
                int64_t i = 0;
                for (int64_t j = 0; j < n_seg; ++j, ++J) {
                    const int b = slot_of(J);
                    const int64_t Jp = J - (kTmemMaster ? 1 : 2);  // the slot's previous segment
                    if (*abort_flag ||
                        (Jp >= 0 && !sm100::mbar_wait(&seg_free[b], use_of(Jp), abort_flag, kGWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    const int64_t i_end = ((j + 1) * Cfg::kSeg < n_chunks) ? (j + 1) * Cfg::kSeg : n_chunks;
                    const uint32_t tmem_seg = tmem_base + (uint32_t)((kTmemMaster ? 1 : b) * kGN);
                    bool first = true;
                    for (; i < i_end; ++i, ++gc) {
                        const int s = (int)(gc % kGStages);
                        const uint32_t ph = (uint32_t)((gc / kGStages) & 1);
                        if (!sm100::mbar_wait(&fullA[s], ph, abort_flag, kGWaitCycles) ||
                            !sm100::mbar_wait(&fullB[s], ph, abort_flag, kGWaitCycles)) {
                            if (!*abort_flag) timeout();
                            stop = true;
                            break;
                        }
                        sm100::tc_fence_after();
                        const uint32_t ahi = sm100::smem_u32(stageA_hi(s)), alo = sm100::smem_u32(stageA_lo(s));
                        const uint32_t bhi = sm100::smem_u32(stageB_hi(s)), blo = sm100::smem_u32(stageB_lo(s));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {  // four 32-byte K steps per 128-byte row
                            const uint32_t off = (uint32_t)kk * 32u;
                            const uint64_t dAh = sm100::desc_k_sw128(ahi + off), dAl = sm100::desc_k_sw128(alo + off);
                            const uint64_t dBh = sm100::desc_k_sw128(bhi + off), dBl = sm100::desc_k_sw128(blo + off);
                            sm100::mma<Cfg::kTF32>(tmem_seg, dAh, dBh, idesc, first ? 0u : 1u);
                            first = false;
                            if (Cfg::kSplit) {
                                sm100::mma<Cfg::kTF32>(tmem_seg, dAh, dBl, idesc, 1u);
                                sm100::mma<Cfg::kTF32>(tmem_seg, dAl, dBh, idesc, 1u);
                            }
                        }
                        sm100::mma_commit(&empty[s]);  // frees stage s once these MMAs complete
                    }
                    sm100::mma_commit(&seg_full[b]);  // segment done (or cut short by an abort)
                    mma_segments = J + 1;
                    if (stop) break;
                }
            }
        }
    } else if (warp == 2) {
        // -------------------------------------------- frequency ring filler
        if (lane == 0) {
            int64_t gc = 0, issued = 0;
            bool stop = false;
            for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
                for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                    const int f = (int)(gc % kGFreqSlots);
                    if (*abort_flag || (gc >= kGFreqSlots &&
                                        !sm100::mbar_wait(&freeF[f], (uint32_t)(((gc / kGFreqSlots) & 1) ^ 1),
                                                          abort_flag, kGWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    if (chk_ok(i * Cfg::kTermsPerChunk, Cfg::kTermsPerChunk, n_chunks * Cfg::kTermsPerChunk)) {
                        sm100::mbar_arrive_expect_tx(&fullF[f], kFreqChunkBytes);
                        sm100::bulk_load(ringF(gc), g.fbasis + i * Cfg::kTermsPerChunk, kFreqChunkBytes, &fullF[f]);
                    } else {
                        sm100::mbar_arrive(&fullF[f]);  // checked build: the slot keeps its old frequencies
                    }
                    issued = gc + 1;
                }
            }
            if (*abort_flag) {
                for (int64_t i = (issued > kGFreqSlots ? issued - kGFreqSlots : 0); i < issued; ++i)
                    sm100::mbar_wait_for(&fullF[i % kGFreqSlots], (uint32_t)((i / kGFreqSlots) & 1), kGWaitCycles / 8);
            }
        }
    } else if (warp >= 4 && warp < 4 + kGPromoters) {
        // ------------------------------------------------------ promoters
        constexpr int PC = GemmShape<PREC>::kPromoteCols;
        constexpr int kSpan = kGN / (kGPromoters / 4);  // columns per promoter warp
        const int quarter = warp & 3;                   // TMEM lanes [32 quarter, 32 quarter + 32)
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int col0 = ((warp - 4) >> 2) * kSpan;
        const int64_t n_master = (int64_t)gridDim.x * kGN * kGM;
        const int64_t mq_off = (int64_t)blockIdx.x * kGN * kGM + (int64_t)quarter * kGN * 32;
        int64_t J = 0;
        bool stop = false;
        for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
            const int64_t rblk = it / g.n_tiles, tile = it - rblk * g.n_tiles;
            const int64_t m = tile * kGM + row;
            for (int64_t j = 0; j < n_seg; ++j, ++J) {
                const int b = slot_of(J);
                if (!sm100::mbar_wait(&seg_full[b], use_of(J), abort_flag, kGWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                sm100::tc_fence_after();
                auto store = [&](int c, float v) {
                    const int64_t r = rblk * kGN + c;
                    // streaming store: the field is not read again, the coefficient tiles are
                    if (m < g.P && r < g.n_real) __stcs(chk(g.out, r * g.P + m, g.n_real * g.P), v);
                };
                if (kTmemMaster)
                    promote_tmem<PC>(tmem_base + lane_off, tmem_base + (uint32_t)kGN + lane_off, j, j == n_seg - 1,
                                     col0, kSpan, store);
                else
                    promote_red<PC>(g.master, n_master, mq_off, tmem_base + (uint32_t)(b * kGN) + lane_off, lane, j,
                                    j == n_seg - 1, col0, kSpan, store);
                sm100::tc_fence_before();
                __syncwarp();
                if (lane == 0) sm100::mbar_arrive(&seg_free[b]);
            }
        }
    } else if (warp >= 4 + kGPromoters) {
        // ------------------------------------------- basis producers
        const int pw = warp - 4 - kGPromoters;     // producer warp
        const int row = (pw & 3) * 32 + lane;      // its row block
        constexpr int kGroups = 4 / (kGProducers / 4);
        const int grp0 = (pw >> 2) * kGroups;      // its term groups [grp0, grp0 + kGroups)
        const FixedScales z = fixed_scales(g.fbound, *g.d_xbound, true);
        int64_t gc = 0;
        bool stop = false;
        for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
            const int64_t tile = it % g.n_tiles;
            const int64_t m = tile * kGM + row;
            const float2 pt = (m < g.P) ? *chk(g.xy, m, g.P) : make_float2(0.0f, 0.0f);
            const int32_t X = __float2int_rn(pt.x * z.xscale), Y = __float2int_rn(pt.y * z.xscale);
            for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                const int s = (int)(gc % kGStages);
                const uint32_t ph = (uint32_t)((gc / kGStages) & 1);
                if (*abort_flag || (gc >= kGStages && !sm100::mbar_wait(&empty[s], ph ^ 1u, abort_flag, kGWaitCycles)) ||
                    !sm100::mbar_wait(&fullF[gc % kGFreqSlots], (uint32_t)((gc / kGFreqSlots) & 1), abort_flag,
                                      kGWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                produce_basis<PREC, kGroups>(reinterpret_cast<const int2*>(ringF(gc)), stageA_hi(s), stageA_lo(s), row,
                                             grp0, z, X, Y, pt);
                sm100::fence_proxy_async_smem();  // each thread: its row writes -> async proxy
                __syncwarp();
                if (lane == 0) {
                    sm100::mbar_arrive(&fullA[s]);
                    sm100::mbar_arrive(&freeF[gc % kGFreqSlots]);
                }
            }
        }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        if (*abort_flag && lane == 0 && mma_segments > 0) {  // MMAs in flight finish before TMEM is freed
            const int64_t Jl = mma_segments - 1;
            sm100::mbar_wait_for(&seg_full[slot_of(Jl)], use_of(Jl), kGWaitCycles / 8);
        }
        __syncwarp();
        sm100::tc_fence_after();
        sm100::tmem_dealloc(tmem_base, 512);
    }
}

// ------------------------------------------------------------ CTA pairs
// k_gemm_pair: the same product on clusters of two CTAs (two SMs) sharing
// one tcgen05.mma of M = 256 (cta_group::2).  A work item is (256-column
// block, pair of 128-point tiles); CTA rank q builds the basis of tile
// 2 p + q (A: its own 128 rows) and TMA-loads columns [128 q, 128 q + 128) of
// the block's coefficient tiles (B: each CTA half of the 256 rows), so each
// SM stages half the coefficient bytes per K chunk and the tensor cores read
// each B row once for both tiles.  Each CTA's TMEM holds the 128 x 256
// accumulator of its own tile; its promoters promote and store it as in
// k_gemm_main, with two slots and the master in L2 for every mode.  Three 64 KB
// stages.  Cross-SM signals: the odd CTA's relay threads forward its
// stage-ready (A written and B landed) and slot-free phases to the even CTA,
// one cluster-scope release each; the MMA commits arrive at empty[s] and
// seg_full[b] in both CTAs (multicast).  A time-out in either CTA raises both
// abort flags; both meet at a cluster barrier before TMEM is freed.
constexpr int kPGStages = 3;
constexpr int kPGTileB = (kGN / 2) * 128;                        // 16 KB: this CTA's half of the columns
constexpr int kPGStageBytes = 2 * kGTileA + 2 * kPGTileB;        // 64 KB
constexpr int kPGSmemBytes = kPGStages * kPGStageBytes + kGFreqSlots * kGFreqBytes + 512 + 1024;

template <int PREC>
__global__ void __launch_bounds__(GemmShape<PREC>::kThreads, 1) k_gemm_pair(const __grid_constant__ CUtensorMap tmapB,
                                                                           GemmArgs g)
{
    using Cfg = GemmCfg<PREC>;
    constexpr int kGProducers = GemmShape<PREC>::kProducers;
    // every mode keeps two TMEM slots and its master in L2 here: with half the
    // coefficient bytes per SM the L2 reductions no longer cost more than the
    // MMAs' waits for a TMEM-resident promotion (3XTF32: 12.4 against 13.7 ms)
    constexpr bool kTmemMaster = false;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* fring = smem + kPGStages * kPGStageBytes;
    uint64_t* fullA = reinterpret_cast<uint64_t*>(fring + kGFreqSlots * kGFreqBytes);
    uint64_t* fullB = fullA + kPGStages;
    uint64_t* peerF = fullB + kPGStages;  // even CTA: the odd CTA's stage s is ready
    uint64_t* empty = peerF + kPGStages;
    uint64_t* seg_full = empty + kPGStages;  // [2]
    uint64_t* seg_free = seg_full + 2;       // [2]
    uint64_t* fullF = seg_free + 2;
    uint64_t* freeF = fullF + kGFreqSlots;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(freeF + kGFreqSlots);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint64_t* never = reinterpret_cast<uint64_t*>(tmem_slot + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = sm100::cluster_ctarank();
    const bool leader = rank == 0;
    const int64_t cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
    const int64_t n_chunks = g.n_chunks;
    const int64_t n_seg = (n_chunks + Cfg::kSeg - 1) / Cfg::kSeg;
    const int64_t n_tp = (g.n_tiles + 1) >> 1;  // tile pairs per column block
    auto slot_of = [](int64_t J) { return kTmemMaster ? 0 : (int)(J & 1); };
    auto use_of = [](int64_t J) { return (uint32_t)((kTmemMaster ? J : (J >> 1)) & 1); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPGStages; ++s) {
            sm100::mbar_init(&fullA[s], kGProducers);
            sm100::mbar_init(&fullB[s], 1);
            sm100::mbar_init(&peerF[s], 1);
            sm100::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            sm100::mbar_init(&seg_full[b], 1);
            sm100::mbar_init(&seg_free[b], leader ? kGPromoters + 1 : kGPromoters);  // + the odd CTA's relay
        }
        for (int s = 0; s < kGFreqSlots; ++s) {
            sm100::mbar_init(&fullF[s], 1);
            sm100::mbar_init(&freeF[s], kGProducers);
        }
        sm100::mbar_init(never, 1);
        *abort_flag = 0;
        sm100::fence_barrier_init();
    }
    if (warp == 1) sm100::tmem_alloc_pair(tmem_slot, 512);
    if (warp == 0 && lane == 0) sm100::prefetch_tmap(&tmapB);
    sm100::tc_fence_before();
    sm100::cluster_sync();  // both CTAs' barriers initialised before any remote arrival
    sm100::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto stageA_hi = [&](int s) { return smem + s * kPGStageBytes; };
    auto stageA_lo = [&](int s) { return smem + s * kPGStageBytes + kGTileA; };
    auto stageB_hi = [&](int s) { return smem + s * kPGStageBytes + 2 * kGTileA; };
    auto stageB_lo = [&](int s) { return smem + s * kPGStageBytes + 2 * kGTileA + kPGTileB; };
    auto ringF = [&](int64_t i) { return fring + (i % kGFreqSlots) * kGFreqBytes; };
    const uint32_t peer_abort = sm100::mapa_shared((const void*)abort_flag, rank ^ 1u);
    auto timeout = [&]() {
        *abort_flag = 1;
        sm100::st_remote_u32(peer_abort, 1u);
        atomicExch(g.err, (int)QRS_ERR_TIMEOUT);
    };
    int64_t mma_segments = 0;
    constexpr uint32_t kFreqChunkBytes = Cfg::kTermsPerChunk * sizeof(int2);

    if (warp == 0) {
        // ---------------------------- TMA producer: this CTA's half of B
        if (lane == 0) {
            int64_t gc = 0, issued = 0;
            bool stop = false;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                const int64_t rblk = it / n_tp;
                const int32_t y0 = (int32_t)(rblk * kGN + rank * (kGN / 2));
                for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                    const int s = (int)(gc % kPGStages);
                    const uint32_t ph = (uint32_t)((gc / kPGStages) & 1);
                    if (*abort_flag ||
                        (gc >= kPGStages && !sm100::mbar_wait(&empty[s], ph ^ 1u, abort_flag, kGWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    sm100::mbar_arrive_expect_tx(&fullB[s], (Cfg::kSplit ? 2u : 1u) * kPGTileB);
                    const int32_t x = (int32_t)(i * Cfg::kElemsPerRow);
                    sm100::tma_load_2d(stageB_hi(s), &tmapB, &fullB[s], x, y0);
                    if (Cfg::kSplit) sm100::tma_load_2d(stageB_lo(s), &tmapB, &fullB[s], x, (int32_t)g.R_pad + y0);
                    issued = gc + 1;
                }
            }
            if (*abort_flag) {
                for (int64_t i = (issued > kPGStages ? issued - kPGStages : 0); i < issued; ++i)
                    sm100::mbar_wait_for(&fullB[i % kPGStages], (uint32_t)((i / kPGStages) & 1), kGWaitCycles / 8);
            }
        }
    } else if (warp == 1) {
        if (leader && lane == 0) {
            // ------------------------------------ MMA issuer (even CTA)
            constexpr uint32_t idesc = sm100::idesc_f32acc(Cfg::kFormat, 2 * kGM, kGN);
            if (g.inject_wait > 0 && !sm100::mbar_wait(never, 0u, abort_flag, g.inject_wait) && !*abort_flag)
                timeout();
            int64_t J = 0, gc = 0;
            bool stop = *abort_flag != 0;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                int64_t i = 0;
                for (int64_t j = 0; j < n_seg; ++j, ++J) {
                    const int b = slot_of(J);
                    const int64_t Jp = J - (kTmemMaster ? 1 : 2);
                    if (*abort_flag ||
                        (Jp >= 0 && !sm100::mbar_wait_cluster(&seg_free[b], use_of(Jp), abort_flag, kGWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    const int64_t i_end = ((j + 1) * Cfg::kSeg < n_chunks) ? (j + 1) * Cfg::kSeg : n_chunks;
                    const uint32_t tmem_seg = tmem_base + (uint32_t)((kTmemMaster ? 1 : b) * kGN);
                    bool first = true;
                    for (; i < i_end; ++i, ++gc) {
                        const int s = (int)(gc % kPGStages);
                        const uint32_t ph = (uint32_t)((gc / kPGStages) & 1);
                        if (!sm100::mbar_wait(&fullA[s], ph, abort_flag, kGWaitCycles) ||
                            !sm100::mbar_wait(&fullB[s], ph, abort_flag, kGWaitCycles) ||
                            !sm100::mbar_wait_cluster(&peerF[s], ph, abort_flag, kGWaitCycles)) {
                            if (!*abort_flag) timeout();
                            stop = true;
                            break;
                        }
                        sm100::tc_fence_after();
                        const uint32_t ahi = sm100::smem_u32(stageA_hi(s)), alo = sm100::smem_u32(stageA_lo(s));
                        const uint32_t bhi = sm100::smem_u32(stageB_hi(s)), blo = sm100::smem_u32(stageB_lo(s));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t off = (uint32_t)kk * 32u;
                            const uint64_t dAh = sm100::desc_k_sw128(ahi + off), dAl = sm100::desc_k_sw128(alo + off);
                            const uint64_t dBh = sm100::desc_k_sw128(bhi + off), dBl = sm100::desc_k_sw128(blo + off);
                            sm100::mma_pair<Cfg::kTF32>(tmem_seg, dAh, dBh, idesc, first ? 0u : 1u);
                            first = false;
                            if (Cfg::kSplit) {
                                sm100::mma_pair<Cfg::kTF32>(tmem_seg, dAh, dBl, idesc, 1u);
                                sm100::mma_pair<Cfg::kTF32>(tmem_seg, dAl, dBh, idesc, 1u);
                            }
                        }
                        sm100::mma_commit_pair(&empty[s], (uint16_t)3);
                    }
                    sm100::mma_commit_pair(&seg_full[b], (uint16_t)3);
                    mma_segments = J + 1;
                    if (stop) break;
                }
            }
        } else if (!leader && lane == 0) {
            // -------------- relay (odd CTA): stage s ready -> even CTA
            const uint32_t remote0 = sm100::mapa_shared(peerF, 0u);
            int64_t gc = 0;
            bool stop = false;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                    const int s = (int)(gc % kPGStages);
                    const uint32_t ph = (uint32_t)((gc / kPGStages) & 1);
                    if (!sm100::mbar_wait(&fullA[s], ph, abort_flag, kGWaitCycles) ||
                        !sm100::mbar_wait(&fullB[s], ph, abort_flag, kGWaitCycles)) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    sm100::mbar_arrive_remote(remote0 + (uint32_t)(s * sizeof(uint64_t)));
                }
            }
        }
    } else if (warp == 2) {
        // -------------------------------------------- frequency ring filler
        if (lane == 0) {
            int64_t gc = 0, issued = 0;
            bool stop = false;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                    const int f = (int)(gc % kGFreqSlots);
                    if (*abort_flag || (gc >= kGFreqSlots &&
                                        !sm100::mbar_wait(&freeF[f], (uint32_t)(((gc / kGFreqSlots) & 1) ^ 1),
                                                          abort_flag, kGWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    if (chk_ok(i * Cfg::kTermsPerChunk, Cfg::kTermsPerChunk, n_chunks * Cfg::kTermsPerChunk)) {
                        sm100::mbar_arrive_expect_tx(&fullF[f], kFreqChunkBytes);
                        sm100::bulk_load(ringF(gc), g.fbasis + i * Cfg::kTermsPerChunk, kFreqChunkBytes, &fullF[f]);
                    } else {
                        sm100::mbar_arrive(&fullF[f]);
                    }
                    issued = gc + 1;
                }
            }
            if (*abort_flag) {
                for (int64_t i = (issued > kGFreqSlots ? issued - kGFreqSlots : 0); i < issued; ++i)
                    sm100::mbar_wait_for(&fullF[i % kGFreqSlots], (uint32_t)((i / kGFreqSlots) & 1), kGWaitCycles / 8);
            }
        }
    } else if (warp == 3) {
        // ---------------- relay (odd CTA): slot read -> even CTA
        if (!leader && lane == 0) {
            const uint32_t remote0 = sm100::mapa_shared(seg_free, 0u);
            int64_t J = 0;
            bool stop = false;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                for (int64_t j = 0; j < n_seg; ++j, ++J) {
                    const int b = slot_of(J);
                    if (!sm100::mbar_wait(&seg_free[b], use_of(J), abort_flag, kGWaitCycles)) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    sm100::mbar_arrive_remote(remote0 + (uint32_t)(b * sizeof(uint64_t)));
                }
            }
        }
    } else if (warp >= 4 && warp < 4 + kGPromoters) {
        // ------------------------------------------------------ promoters
        constexpr int PC = GemmShape<PREC>::kPromoteCols;
        constexpr int kSpan = kGN / (kGPromoters / 4);
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int col0 = ((warp - 4) >> 2) * kSpan;
        const int64_t n_master = (int64_t)gridDim.x * kGN * kGM;
        const int64_t mq_off = (int64_t)blockIdx.x * kGN * kGM + (int64_t)quarter * kGN * 32;
        int64_t J = 0;
        bool stop = false;
        for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
            const int64_t rblk = it / n_tp, tp = it - rblk * n_tp;
            const int64_t m = (2 * tp + rank) * kGM + row;
            for (int64_t j = 0; j < n_seg; ++j, ++J) {
                const int b = slot_of(J);
                if (!sm100::mbar_wait(&seg_full[b], use_of(J), abort_flag, kGWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                sm100::tc_fence_after();
                auto store = [&](int c, float v) {
                    const int64_t r = rblk * kGN + c;
                    // streaming store: the field is not read again, the coefficient tiles are
                    if (m < g.P && r < g.n_real) __stcs(chk(g.out, r * g.P + m, g.n_real * g.P), v);
                };
                if (kTmemMaster)
                    promote_tmem<PC>(tmem_base + lane_off, tmem_base + (uint32_t)kGN + lane_off, j, j == n_seg - 1,
                                     col0, kSpan, store);
                else
                    promote_red<PC>(g.master, n_master, mq_off, tmem_base + (uint32_t)(b * kGN) + lane_off, lane, j,
                                    j == n_seg - 1, col0, kSpan, store);
                sm100::tc_fence_before();
                __syncwarp();
                if (lane == 0) sm100::mbar_arrive(&seg_free[b]);
            }
        }
    } else if (warp >= 4 + kGPromoters) {
        // ------------------------------------------- basis producers
        const int pw = warp - 4 - kGPromoters;
        const int row = (pw & 3) * 32 + lane;
        constexpr int kGroups = 4 / (kGProducers / 4);
        const int grp0 = (pw >> 2) * kGroups;
        const FixedScales z = fixed_scales(g.fbound, *g.d_xbound, true);
        int64_t gc = 0;
        bool stop = false;
        for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
            const int64_t tp = it % n_tp;
            const int64_t m = (2 * tp + rank) * kGM + row;
            const float2 pt = (m < g.P) ? *chk(g.xy, m, g.P) : make_float2(0.0f, 0.0f);
            const int32_t X = __float2int_rn(pt.x * z.xscale), Y = __float2int_rn(pt.y * z.xscale);
            for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                const int s = (int)(gc % kPGStages);
                const uint32_t ph = (uint32_t)((gc / kPGStages) & 1);
                if (*abort_flag ||
                    (gc >= kPGStages && !sm100::mbar_wait(&empty[s], ph ^ 1u, abort_flag, kGWaitCycles)) ||
                    !sm100::mbar_wait(&fullF[gc % kGFreqSlots], (uint32_t)((gc / kGFreqSlots) & 1), abort_flag,
                                      kGWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                produce_basis<PREC, kGroups>(reinterpret_cast<const int2*>(ringF(gc)), stageA_hi(s), stageA_lo(s), row,
                                             grp0, z, X, Y, pt);
                sm100::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    sm100::mbar_arrive(&fullA[s]);
                    sm100::mbar_arrive(&freeF[gc % kGFreqSlots]);
                }
            }
        }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0 && leader && *abort_flag && mma_segments > 0) {
        const int64_t Jl = mma_segments - 1;  // the pair's MMAs in flight finish first
        sm100::mbar_wait_cluster_for(&seg_full[slot_of(Jl)], use_of(Jl), kGWaitCycles / 8);
    }
    __syncwarp();
    sm100::cluster_sync();  // neither CTA frees TMEM or exits while the pair still works on it
    if (warp == 1) {
        sm100::tc_fence_after();
        sm100::tmem_dealloc_pair(tmem_base, 512);
    }
}

// ------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

size_t gemm_workspace_bytes(int mode, int64_t n_f, int64_t n_real, int num_sms)
{
    const bool bf16 = mode == QRS_SYNTH_GEMM_BF16X3;
    const int T = bf16 ? GemmCfg<QRS_SYNTH_GEMM_BF16X3>::kTermsPerChunk : GemmCfg<QRS_SYNTH_GEMM_3XTF32>::kTermsPerChunk;
    const int eb = bf16 ? 2 : 4;
    const int halves = mode == QRS_SYNTH_GEMM_TF32 ? 1 : 2;
    const int64_t nf_pad = (n_f + T - 1) / T * T;
    const int64_t R_pad = (n_real + kGN - 1) / kGN * kGN;
    const size_t b = (size_t)halves * R_pad * (2 * nf_pad) * eb;  // hi (and lo) halves
    return 256 + b + (size_t)nf_pad * (sizeof(int2) + sizeof(float4)) + 1024 +
           (size_t)num_sms * kGN * kGM * sizeof(float);  // the CTAs' FP32 masters
}

static void gemm_pair_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute (&at)[1], unsigned grid, int threads,
                             cudaStream_t s)
{
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = kPGSmemBytes;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

// Clusters of two k_gemm_pair CTAs the GPU holds at once (cached per handle
// and mode); 0 when pairs are switched off (QRS_GEMM_PAIR=0 at qrs_create)
// or unavailable.
template <int PREC>
static int gemm_pair_clusters(qrs_handle* h)
{
    int& c = h->gemm_pair_clusters[PREC == QRS_SYNTH_GEMM_3XTF32 ? 0 : PREC == QRS_SYNTH_GEMM_BF16X3 ? 1 : 2];
    if (!h->gemm_pair) return 0;
    if (c == 0) {
        int n = 0;
        cudaError_t e =
            cudaFuncSetAttribute(k_gemm_pair<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPGSmemBytes);
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            gemm_pair_config(cfg, at, (unsigned)(h->num_sms & ~1), GemmShape<PREC>::kThreads, nullptr);
            e = cudaOccupancyMaxActiveClusters(&n, k_gemm_pair<PREC>, &cfg);
        }
        if (e != cudaSuccess) cudaGetLastError();  // the single-CTA kernel serves instead
        c = (e == cudaSuccess && n > 0) ? (n < h->num_sms / 2 ? n : h->num_sms / 2) : -1;
    }
    return c > 0 ? c : 0;
}

template <int PREC>
static cudaError_t launch_gemm_t(qrs_handle* h, const DrawParams& p, const float* xy, int64_t P, int64_t n_real,
                                 const double* col_psd, double c_vk, float* out, cudaStream_t s)
{
    using Cfg = GemmCfg<PREC>;
    constexpr int T = Cfg::kTermsPerChunk;
    const int64_t nf_pad = (p.n_f + T - 1) / T * T;
    const int64_t Kp = 2 * nf_pad;
    const int64_t R_pad = (n_real + kGN - 1) / kGN * kGN;
    // workspace: [B hi | B lo][R_pad][Kp], fbasis[nf_pad], fw[nf_pad]
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)h->d_work + 255) & ~(uintptr_t)255);
    void* B = base;
    const size_t bbytes = (size_t)(Cfg::kSplit ? 2 : 1) * R_pad * Kp * Cfg::kElemBytes;
    int2* fbasis = reinterpret_cast<int2*>(base + bbytes);
    float4* fw = reinterpret_cast<float4*>(fbasis + nf_pad);
    float* master = reinterpret_cast<float*>(((uintptr_t)(fw + nf_pad) + 255) & ~(uintptr_t)255);

    cudaError_t e = launch_point_bound(xy, P, h->d_xbound, s);
    if (e != cudaSuccess) return e;
    const float fbound = (float)freq_bound(p);
    k_gemm_freq<<<(unsigned)((nf_pad + 255) / 256), 256, 0, s>>>(p, nf_pad, h->d_xbound, fbound, fbasis, fw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 cg((unsigned)std::min<int64_t>((nf_pad + 255) / 256, 64), (unsigned)R_pad);
    k_gemm_coef<PREC><<<cg, 256, 0, s>>>(p, nf_pad, n_real, R_pad, fw, col_psd, c_vk, B);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // CTA pairs for the split modes when there are point tiles to pair and the
    // GPU can hold a pair (single-pass TF32, with a third of the MMA work per
    // chunk, measured faster on single CTAs: 8.3 against 10.3 ms per batch)
    const int64_t n_tiles = (P + kGM - 1) / kGM;
    int clusters = 0;
    if constexpr (Cfg::kSplit) clusters = n_tiles >= 2 ? gemm_pair_clusters<PREC>(h) : 0;
    PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap tmap;
    const cuuint64_t gdim[2] = {(cuuint64_t)Kp, (cuuint64_t)((Cfg::kSplit ? 2 : 1) * R_pad)};
    const cuuint64_t gstride[1] = {(cuuint64_t)(Kp * Cfg::kElemBytes)};
    const cuuint32_t box[2] = {(cuuint32_t)Cfg::kElemsPerRow, (cuuint32_t)(clusters > 0 ? kGN / 2 : kGN)};
    const cuuint32_t estride[2] = {1, 1};
    CUresult cr = encode(&tmap, Cfg::kTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B,
                         gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;

    GemmArgs a;
    a.xy = reinterpret_cast<const float2*>(xy);
    a.P = P;
    a.out = out;
    a.n_real = n_real;
    a.R_pad = R_pad;
    a.n_chunks = Kp / Cfg::kElemsPerRow;
    a.n_tiles = n_tiles;
    a.n_items = (clusters > 0 ? (n_tiles + 1) / 2 : n_tiles) * (R_pad / kGN);
    a.master = master;
    a.fbasis = fbasis;
    a.d_xbound = h->d_xbound;
    a.fbound = fbound;
    a.err = h->d_err;
    a.inject_wait = 0;
    if (h->fault & kFaultTimeout) {  // one-shot: this launch only
        a.inject_wait = 2000000;     // about 1 ms of SM clock
        h->fault &= ~kFaultTimeout;
    }
    if constexpr (Cfg::kSplit) {
        if (clusters > 0) {
            const int64_t nc = a.n_items < clusters ? a.n_items : clusters;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            gemm_pair_config(cfg, at, (unsigned)(2 * nc), GemmShape<PREC>::kThreads, s);
            return cudaLaunchKernelEx(&cfg, k_gemm_pair<PREC>, tmap, a);
        }
    }
    e = cudaFuncSetAttribute(k_gemm_main<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t ctas = a.n_items < h->num_sms ? a.n_items : h->num_sms;  // persistent: one CTA per SM
    k_gemm_main<PREC><<<(unsigned)ctas, GemmShape<PREC>::kThreads, kGSmemBytes, s>>>(tmap, a);
    return cudaGetLastError();
}

cudaError_t launch_synth_gemm(qrs_handle* h, int mode, const DrawParams& p, const float* xy, int64_t P, int64_t n_real,
                              const double* col_psd, double c_vk, float* out, cudaStream_t s)
{
    if (mode == QRS_SYNTH_GEMM_3XTF32)
        return launch_gemm_t<QRS_SYNTH_GEMM_3XTF32>(h, p, xy, P, n_real, col_psd, c_vk, out, s);
    if (mode == QRS_SYNTH_GEMM_TF32)
        return launch_gemm_t<QRS_SYNTH_GEMM_TF32>(h, p, xy, P, n_real, col_psd, c_vk, out, s);
    return launch_gemm_t<QRS_SYNTH_GEMM_BF16X3>(h, p, xy, P, n_real, col_psd, c_vk, out, s);
}

}  // namespace qrs
