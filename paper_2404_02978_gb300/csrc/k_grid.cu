// k_grid.cu -- K6: Eq. 3 on a tensor-product point set, as one tensor-core
// product per realisation (the separable form).
//
// When the points form a grid {x_i} x {y_j} (a pupil sampled on a regular
// grid, with or without a mask), each harmonic of Eq. 3 factors:
//     e^{i 2 pi (fx x_i + fy y_j)} = e^{i 2 pi fx x_i} e^{i 2 pi fy y_j},
// and with c = F (a + i b), Re[c e^{i(tx + ty)}] =
//     cos tx (Fa cos ty - Fb sin ty) - sin tx (Fa sin ty + Fb cos ty).
// and the identity is symmetric in tx and ty.  So realisation r on the grid
// is one real matrix product over k' in 2 N_f:
//     chi_r(x_i, y_j) = sum_k' U[i][k'] V[j][k'],
//     U[i] = [F(a cos - b sin)(2 pi fx_k x_i) | -F(a sin + b cos)(..)]  (x side)
//     V[j] = [cos 2 pi fy_k y_j | sin 2 pi fy_k y_j]                   (y side)
// per K chunk of T terms (cos half, then sin half); QRS_GRID_COEF_X=0 puts
// the coefficient products on the y side instead.  Building U and V costs
// (n_x + n_y) N_f sin/cos pairs per realisation instead of n_x n_y N_f, and
// the product runs on the 5th-generation tensor cores in split precision
// (3XTF32: hi/lo TF32 halves, A_hi B_hi + A_hi B_lo + A_lo B_hi; BF16X3 the
// same with BF16 halves), accumulated in TMEM.
//
// Launches: k_grid_bound (max |x|, |y|: picks the phase path and scales),
// then per slab of realisations k_grid_draw (Philox + R2 + FP64 map, the same
// draw as every other form; records {Fx, Fy, F a, F b} in HBM) and
// k_grid_main.
//
// k_grid_main: a persistent grid, one CTA per SM, walking work items
// (realisation, 128-column x tile, 256-row y block), realisation-major, so
// neighbouring CTAs share a realisation's draw records in L2.  Warps:
//   warp 1      TMEM allocator (512 columns: two 128 x 256 FP32 segment
//               slots) and single-thread MMA issuer: 3 x 4 tcgen05.mma per K
//               chunk into the segment's slot, a commit per segment, the two
//               slots alternating so the MMAs never wait for a promotion;
//   warp 2      record ring: bulk-copies each chunk's draw records into an
//               8-slot shared-memory ring, up to 8 chunks ahead;
//   promoters  (4 or 8 warps from warp 4): after each segment, master +=
//               slot in FP32 (tcgen05.ld of the slot; the master is the CTA's
//               128 KB scratch in L2, each element owned by one thread, lanes
//               along x so every access is coalesced).  The tensor core's
//               accumulation drifts by about 2^-26 per step with a consistent
//               sign, so segments bound the chain.  After the last segment
//               they store the tile (lanes along x: coalesced);
//   producers  (8, 12 or 16 warps after them): build the chunk's x rows and
//               y rows -- phase (fixed point or double-float), MUFU sin/cos,
//               the coefficient products on one side (the x side by
//               default: 128 rows per tile instead of 256), hi/lo split,
//               16-byte stores into the 128-byte-swizzled K-major tiles;
//               fence.proxy.async; one arrival per warp.
// Every mbarrier wait is bounded in time; on time-out the CTA raises an abort
// flag, records QRS_ERR_TIMEOUT in the device error word, waits (bounded)
// for its copies and MMAs in flight, frees TMEM and returns.
#include "qrs_internal.h"
#include "qrs_sm100.cuh"
#include "qrs_tc_split.cuh"

#ifndef QRS_GRID_PRODUCERS
#define QRS_GRID_PRODUCERS 16  // producer warps: 8 (threads share an x row and own a y row), 12, 16
#endif
#ifndef QRS_GRID_PROMOTERS
#define QRS_GRID_PROMOTERS 4   // promoter warps: 4 (256 columns each) or 8 (128)
#endif
#ifndef QRS_GRID_PROMOTE_COLS
#define QRS_GRID_PROMOTE_COLS 16  // TMEM columns a promoter thread holds at a time (32 or 16)
#endif
#ifndef QRS_GRID_COEF_X
#define QRS_GRID_COEF_X 1      // coefficients on the x side (128 rows per tile) instead of the y side (256)
#endif

namespace qrs {

QRS_CHECK_HOOK(check_hook_grid)

constexpr int kXM = 128;                                  // x values per tile (UMMA M, TMEM lanes)
constexpr int kXN = 256;                                  // y values per block (UMMA N)
constexpr int kXStages = 2;
constexpr int kXTileA = kXM * 128;                        // 16 KB
constexpr int kXTileB = kXN * 128;                        // 32 KB
constexpr int kXStageBytes = 2 * kXTileA + 2 * kXTileB;   // U hi/lo + V hi/lo = 96 KB
constexpr int kXRecSlots = 8;
constexpr int kXRecBytes = 512;                           // one chunk's records (<= 32 x 16 B)
constexpr int kXProducers = QRS_GRID_PRODUCERS;
constexpr int kXPromoters = QRS_GRID_PROMOTERS;
constexpr bool kXCoefX = QRS_GRID_COEF_X != 0;
constexpr int kXThreads = 128 + 32 * (kXPromoters + kXProducers);
static_assert(kXProducers == 8 || kXProducers == 12 || kXProducers == 16, "producer warps");
static_assert(kXPromoters == 4 || kXPromoters == 8, "promoter warps");
constexpr int kXStageFloats = 2 * QRS_GRID_PROMOTE_COLS * 32;  // two promotion staging buffers per promoter warp
constexpr int kXSmemBytes =
    kXStages * kXStageBytes + kXRecSlots * kXRecBytes + 512 + kXPromoters * kXStageFloats * 4 + 1024;
constexpr long long kXWaitCycles = 4000000000LL;          // ~2 s of SM clock per wait
constexpr size_t kXSlabBytes = (size_t)256 << 20;         // draw records per slab of realisations

struct GridArgs {
    const float* x;
    int64_t nx;
    const float* y;
    int64_t ny;
    const int32_t* index;  // [ny][nx] output point of each grid node (< 0: none), or null (dense)
    int64_t P;
    float* out;
    int64_t r0;            // output row of the slab's first realisation
    int64_t n_chunks;      // K chunks per realisation
    int64_t nf_pad;
    int64_t n_mt, n_nb, n_items;
    int64_t out_rows;      // realisations in `out` (bounds-checked build)
    int64_t rec_rows;      // realisations in this slab of `rec`
    const int4* rec;       // [slab realisations][nf_pad] {Fx|fx, Fy|fy, F a, F b}
    float* master;         // [gridDim.x][kXN][kXM] FP32 accumulators of the CTAs' current items
    const float* d_bound;
    float fbound;
    int* err;
};

// max(|x|, |y|) over both coordinate vectors (one CTA, no atomics).
__global__ void k_grid_bound(const float* __restrict__ x, int64_t nx, const float* __restrict__ y, int64_t ny,
                             float* __restrict__ out)
{
    float m = 0.0f;
    for (int64_t i = threadIdx.x; i < nx; i += blockDim.x) m = fmaxf(m, fabsf(x[i]));
    for (int64_t i = threadIdx.x; i < ny; i += blockDim.x) m = fmaxf(m, fabsf(y[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (blockDim.x >> 5)) ? wmax[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *out = m;
    }
}

// Draw records of realisations [p.real_offset, p.real_offset + n_real):
// frequencies in the phase path's representation and the coefficient
// products F a, F b (terms k >= N_f are zero records).
__global__ void k_grid_draw(DrawParams p, int64_t n_real, int64_t nf_pad, const float* __restrict__ d_bound,
                            float fbound, int4* __restrict__ rec)
{
    const FixedScales z = fixed_scales(fbound, *d_bound, true);
    const int64_t total = n_real * nf_pad;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / nf_pad, k = q - r * nf_pad;
        int4 v = make_int4(0, 0, 0, 0);
        if (k < p.n_f) {
            const Term t = draw_term<false>(p, (uint64_t)(p.real_offset + r) * (uint64_t)p.n_f + (uint64_t)k, k);
            if (z.use_fixed) {
                v.x = __float2int_rn(t.fx * z.fscale);
                v.y = __float2int_rn(t.fy * z.fscale);
            } else {
                v.x = __float_as_int(t.fx);
                v.y = __float_as_int(t.fy);
            }
            v.z = __float_as_int(t.F * t.a);
            v.w = __float_as_int(t.F * t.b);
        }
        *chk(rec, q, total) = v;
    }
}

// One coordinate's phase 2 pi f x mod 2 pi, in radians.  Fixed point: the
// exact 64-bit product of the scaled integers, 23 fraction bits of the turn
// into a float mantissa, one FFMA to radians in [0, 2 pi).  Double-float: the
// error-free product, its integer part removed exactly, in (-pi, pi].
template <bool FIXED>
__device__ __forceinline__ float phase1_rad(int32_t F, int32_t X, float f, float x, uint64_t bias, uint32_t shift)
{
    if (FIXED) {
        const uint64_t acc = bias + (uint64_t)((int64_t)F * (int64_t)X);
        const uint32_t m = __funnelshift_rc((uint32_t)acc, (uint32_t)(acc >> 32), shift);
        return fmaf(__int_as_float((m & 0x007FFFFFu) | 0x3F800000u), 6.28318530717958648f, -6.28318530717958648f);
    } else {
        const float p1 = __fmul_rn(f, x);
        const float e1 = __fmaf_rn(f, x, -p1);
        const float n1 = __fsub_rn(__fadd_rn(p1, 12582912.0f), 12582912.0f);
        return __fadd_rn(__fsub_rn(p1, n1), e1) * 6.28318530717958648f;
    }
}

// One operand row of a K chunk, 16-byte groups [g0, g0 + NG) of each half:
// the harmonic of coordinate x (SIDE 0: fx x, SIDE 1: fy y) for the chunk's
// terms, plain (cos | sin) or, with COEF, weighted by the coefficients
// (F(a cos - b sin) | -F(a sin + b cos)); split hi/lo into the swizzled tile.
template <int PREC, bool FIXED, int SIDE, bool COEF, int NG, int TILE_BYTES>
__device__ __forceinline__ void produce_row(const int4* __restrict__ rr, unsigned char* hi_t, unsigned char* lo_t,
                                            int row, int g0, int32_t Xq, float xf, uint64_t bias, uint32_t shift)
{
    constexpr int TPG = GemmCfg<PREC>::kTermsPer16B;
    constexpr int T = GemmCfg<PREC>::kTermsPerChunk;
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
        const int grp = g0 + gi;
        float cv[TPG], sv[TPG];
#pragma unroll
        for (int t = 0; t < TPG; ++t) {
            const int4 r = *chk(rr, grp * TPG + t, T);
            const int32_t fq = SIDE == 0 ? r.x : r.y;
            const float ang = phase1_rad<FIXED>(fq, Xq, __int_as_float(fq), xf, bias, shift);
            const float sn = __sinf(ang), cs = __cosf(ang);
            if (COEF) {
                const float Fa = __int_as_float(r.z), Fb = __int_as_float(r.w);
                cv[t] = fmaf(Fa, cs, -(Fb * sn));
                sv[t] = -fmaf(Fa, sn, Fb * cs);
            } else {
                cv[t] = cs;
                sv[t] = sn;
            }
        }
        uint4 h, l;
        const uint32_t oc = sm100::sw128_offset((uint32_t)row, (uint32_t)grp);
        const uint32_t os = sm100::sw128_offset((uint32_t)row, (uint32_t)(4 + grp));
        pack16<PREC>(cv, h, l);
        if (chk_ok(oc, 16, TILE_BYTES)) {
            *reinterpret_cast<uint4*>(hi_t + oc) = h;
            *reinterpret_cast<uint4*>(lo_t + oc) = l;
        }
        pack16<PREC>(sv, h, l);
        if (chk_ok(os, 16, TILE_BYTES)) {
            *reinterpret_cast<uint4*>(hi_t + os) = h;
            *reinterpret_cast<uint4*>(lo_t + os) = l;
        }
    }
}

// A producer thread's share of a chunk.  8 warps: thread t builds half of x
// row t mod 128 (groups 2 (t / 128) + {0, 1}) and all of y row t; 12 warps:
// threads 0-127 build x rows, 128-383 y rows; 16 warps: threads 0-255 the
// x half rows, 256-511 the y rows.
template <int PREC, bool FIXED>
__device__ __forceinline__ void produce_share(const int4* __restrict__ rr, unsigned char* Ahi, unsigned char* Alo,
                                              unsigned char* Bhi, unsigned char* Blo, int t, int32_t XA, float xa,
                                              int32_t YB, float yb, uint64_t bias, uint32_t shift)
{
    constexpr bool CX = kXCoefX, CY = !kXCoefX;
    if (kXProducers == 8) {
        produce_row<PREC, FIXED, 0, CX, 2, kXTileA>(rr, Ahi, Alo, t & 127, 2 * (t >> 7), XA, xa, bias, shift);
        produce_row<PREC, FIXED, 1, CY, 4, kXTileB>(rr, Bhi, Blo, t, 0, YB, yb, bias, shift);
    } else if (kXProducers == 12) {
        if (t < kXM) produce_row<PREC, FIXED, 0, CX, 4, kXTileA>(rr, Ahi, Alo, t, 0, XA, xa, bias, shift);
        else produce_row<PREC, FIXED, 1, CY, 4, kXTileB>(rr, Bhi, Blo, t - kXM, 0, YB, yb, bias, shift);
    } else {
        if (t < 2 * kXM) produce_row<PREC, FIXED, 0, CX, 2, kXTileA>(rr, Ahi, Alo, t & 127, 2 * (t >> 7), XA, xa, bias, shift);
        else produce_row<PREC, FIXED, 1, CY, 4, kXTileB>(rr, Bhi, Blo, t - 2 * kXM, 0, YB, yb, bias, shift);
    }
}

// Output store of a promoted value: grid node (xi, yj) of realisation row
// orow, through the node -> point index when there is one.
__device__ __forceinline__ void store_node(const GridArgs& g, int64_t orow, int64_t xi, int64_t yj, float v)
{
    if (xi >= g.nx || yj >= g.ny) return;
    const int64_t node = yj * g.nx + xi;
    if (g.index) {
        const int32_t pidx = *chk(g.index, node, g.nx * g.ny);
        if (pidx >= 0 && pidx < g.P) *chk(g.out, orow * g.P + pidx, g.out_rows * g.P) = v;
        else if (pidx >= g.P) atomicExch(g.err, (int)QRS_ERR_DEVICE_CHECK);
    } else {
        *chk(g.out, orow * g.ny * g.nx + node, g.out_rows * g.ny * g.nx) = v;
    }
}

// The single-CTA kernel's segment promotion: as promote_red (the master in
// L2 as [quarter][column][32 lanes], := slot, += slot, slot + master at the
// last segment), but each 16- or 32-column piece of the warp is staged in
// shared memory and handed to L2 as one bulk copy / bulk FP32 reduction by
// lane 0 (two staging buffers alternate; lane 0 waits until the operation
// before the previous one has read its buffer).  Returns with every bulk
// operation issued; the caller waits for them (bulk_wait) before the CTA
// exits.  (With 4 promoter warps this beats per-lane reductions; the pair
// kernel's 8 promoter warps use promote_red.)
template <int PC, class Store>
__device__ __forceinline__ void promote_segment(const GridArgs& g, uint32_t slot_q, int64_t mq_off, float* stage,
                                                int lane, int64_t j, bool last, int col0, int span, Store&& store)
{
    const int64_t n_master = (int64_t)gridDim.x * kXN * kXM;
    float* mq = g.master + mq_off;
    if (last && j > 0) {
        if (lane == 0) sm100::bulk_wait<0>();
        __syncwarp();
        sm100::fence_proxy_async_global();
    }
    int buf = 0;
#pragma unroll 1
    for (int c0 = col0; c0 < col0 + span; c0 += PC) {
        uint32_t v[PC];
        sm100::tmem_ld_cols(slot_q + (uint32_t)c0, v);
        sm100::tmem_ld_wait();
        if (last) {
            if (j > 0) {
#pragma unroll
                for (int q = 0; q < PC; ++q)
                    v[q] = __float_as_uint(__uint_as_float(v[q]) +
                                           *chk(g.master, mq_off + (int64_t)(c0 + q) * 32 + lane, n_master));
            }
#pragma unroll
            for (int q = 0; q < PC; ++q) store(c0 + q, __uint_as_float(v[q]));
        } else {
            float* sb = stage + buf * PC * 32;
            if (lane == 0) sm100::bulk_wait_read<1>();
            __syncwarp();
#pragma unroll
            for (int q = 0; q < PC; ++q) sb[q * 32 + lane] = __uint_as_float(v[q]);
            sm100::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0 && chk_ok(mq_off + (int64_t)c0 * 32, PC * 32, n_master)) {
                if (j == 0) sm100::bulk_store(mq + (int64_t)c0 * 32, sb, PC * 32 * 4);
                else sm100::bulk_reduce_add_f32(mq + (int64_t)c0 * 32, sb, PC * 32 * 4);
                sm100::bulk_commit();
            }
            buf ^= 1;
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(kXThreads, 1) k_grid_main(const __grid_constant__ GridArgs g)
{
    using Cfg = GemmCfg<PREC>;
    constexpr int T = Cfg::kTermsPerChunk;
    static_assert(T / Cfg::kTermsPer16B == 4, "four 16-byte groups per half row");
    static_assert(T * 16 <= kXRecBytes, "a chunk's records fit their ring slot");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* rring = smem + kXStages * kXStageBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(rring + kXRecSlots * kXRecBytes);
    uint64_t* empty = full + kXStages;
    uint64_t* seg_full = empty + kXStages;  // [2], one per TMEM segment slot
    uint64_t* seg_free = seg_full + 2;      // [2]
    uint64_t* fullR = seg_free + 2;
    uint64_t* freeR = fullR + kXRecSlots;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(freeR + kXRecSlots);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* pstage = reinterpret_cast<float*>(rring + kXRecSlots * kXRecBytes + 512);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_chunks = g.n_chunks;
    const int64_t n_seg = (n_chunks + Cfg::kSeg - 1) / Cfg::kSeg;
    const int64_t per_real = g.n_mt * g.n_nb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kXStages; ++s) {
            sm100::mbar_init(&full[s], kXProducers);
            sm100::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            sm100::mbar_init(&seg_full[b], 1);
            sm100::mbar_init(&seg_free[b], kXPromoters);
        }
        for (int s = 0; s < kXRecSlots; ++s) {
            sm100::mbar_init(&fullR[s], 1);
            sm100::mbar_init(&freeR[s], kXProducers);
        }
        *abort_flag = 0;
        sm100::fence_barrier_init();
    }
    if (warp == 1) sm100::tmem_alloc(tmem_slot, 512);
    sm100::tc_fence_before();
    __syncthreads();
    sm100::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;  // slot b: columns [256 b, 256 b + 256)

    auto stageA_hi = [&](int s) { return smem + s * kXStageBytes; };
    auto stageA_lo = [&](int s) { return smem + s * kXStageBytes + kXTileA; };
    auto stageB_hi = [&](int s) { return smem + s * kXStageBytes + 2 * kXTileA; };
    auto stageB_lo = [&](int s) { return smem + s * kXStageBytes + 2 * kXTileA + kXTileB; };
    auto ringR = [&](int64_t i) { return rring + (i % kXRecSlots) * kXRecBytes; };
    auto timeout = [&]() {
        *abort_flag = 1;
        atomicExch(g.err, (int)QRS_ERR_TIMEOUT);
    };
    int64_t mma_segments = 0;

    if (warp == 1) {
        // ---------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = sm100::idesc_f32acc(Cfg::kFormat, kXM, kXN);
            int64_t J = 0, gc = 0;
            bool stop = false;
            for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
                int64_t i = 0;
                for (int64_t j = 0; j < n_seg; ++j, ++J) {
                    const int b = (int)(J & 1);
                    if (*abort_flag || (J >= 2 && !sm100::mbar_wait(&seg_free[b], (uint32_t)(((J - 2) >> 1) & 1),
                                                                     abort_flag, kXWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    const int64_t i_end = ((j + 1) * Cfg::kSeg < n_chunks) ? (j + 1) * Cfg::kSeg : n_chunks;
                    const uint32_t tmem_seg = tmem_base + (uint32_t)(b * kXN);
                    bool first = true;
                    for (; i < i_end; ++i, ++gc) {
                        const int s = (int)(gc % kXStages);
                        const uint32_t ph = (uint32_t)((gc / kXStages) & 1);
                        if (!sm100::mbar_wait(&full[s], ph, abort_flag, kXWaitCycles)) {
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
                            sm100::mma<Cfg::kTF32>(tmem_seg, dAh, dBh, idesc, first ? 0u : 1u);
                            first = false;
                            sm100::mma<Cfg::kTF32>(tmem_seg, dAh, dBl, idesc, 1u);
                            sm100::mma<Cfg::kTF32>(tmem_seg, dAl, dBh, idesc, 1u);
                        }
                        sm100::mma_commit(&empty[s]);
                    }
                    sm100::mma_commit(&seg_full[b]);
                    mma_segments = J + 1;
                    if (stop) break;
                }
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------- record ring
        if (lane == 0) {
            int64_t gc = 0;
            bool stop = false;
            for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
                const int64_t r = it / per_real;
                const int4* src = g.rec + r * g.nf_pad;
                for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                    const int f = (int)(gc % kXRecSlots);
                    if (*abort_flag ||
                        (gc >= kXRecSlots && !sm100::mbar_wait(&freeR[f], (uint32_t)(((gc / kXRecSlots) & 1) ^ 1),
                                                               abort_flag, kXWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    if (chk_ok(r * g.nf_pad + i * T, T, g.rec_rows * g.nf_pad)) {
                        sm100::mbar_arrive_expect_tx(&fullR[f], (uint32_t)(T * 16));
                        sm100::bulk_load(ringR(gc), src + i * T, (uint32_t)(T * 16), &fullR[f]);
                    } else {
                        sm100::mbar_arrive(&fullR[f]);  // checked build: the slot keeps its old records
                    }
                }
            }
            if (*abort_flag) {  // copies in flight land before the CTA exits
                for (int64_t i = (gc > kXRecSlots ? gc - kXRecSlots : 0); i < gc; ++i)
                    sm100::mbar_wait_for(&fullR[i % kXRecSlots], (uint32_t)((i / kXRecSlots) & 1), kXWaitCycles / 8);
            }
        }
    } else if (warp >= 4 && warp < 4 + kXPromoters) {
        // ------------------------------------------------------ promoters
        constexpr int kSpan = kXN / (kXPromoters / 4);  // columns per promoter warp
        constexpr int PC = QRS_GRID_PROMOTE_COLS;
        static_assert(PC == 32 || PC == 16, "promotion width");
        static_assert((kSpan / PC) % 2 == 0, "an even number of pieces per segment (staging buffers alternate)");
        const int quarter = warp & 3;                   // TMEM lanes [32 quarter, 32 quarter + 32)
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int col0 = ((warp - 4) >> 2) * kSpan;
        const int64_t mq_off = (int64_t)blockIdx.x * kXN * kXM + (int64_t)quarter * kXN * 32;
        float* stage = pstage + (warp - 4) * 2 * PC * 32;
        int64_t J = 0;
        bool stop = false;
        for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
            const int64_t r = it / per_real, rem = it - r * per_real;
            const int64_t mt = rem / g.n_nb, nb = rem - mt * g.n_nb;
            const int64_t xi = mt * kXM + row;
            const int64_t orow = g.r0 + r;
            for (int64_t j = 0; j < n_seg; ++j, ++J) {
                const int b = (int)(J & 1);
                if (!sm100::mbar_wait(&seg_full[b], (uint32_t)((J >> 1) & 1), abort_flag, kXWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                sm100::tc_fence_after();
                promote_segment<PC>(g, tmem_base + (uint32_t)(b * kXN) + lane_off, mq_off, stage, lane, j,
                                    j == n_seg - 1, col0, kSpan,
                                    [&](int c, float v) { store_node(g, orow, xi, nb * kXN + c, v); });
                sm100::tc_fence_before();
                __syncwarp();
                if (lane == 0) sm100::mbar_arrive(&seg_free[b]);
            }
        }
        if (lane == 0) sm100::bulk_wait<0>();  // staging buffers are read before the CTA exits
    } else if (warp >= 4 + kXPromoters) {
        // ------------------------------------------------------ producers
        const int t = (warp - 4 - kXPromoters) * 32 + lane;
        const int xrow = kXProducers == 8 ? (t & 127) : kXProducers == 12 ? (t < kXM ? t : -1)
                                                                           : (t < 2 * kXM ? (t & 127) : -1);
        const int yrow = kXProducers == 8 ? t : kXProducers == 12 ? (t >= kXM ? t - kXM : -1)
                                                                  : (t >= 2 * kXM ? t - 2 * kXM : -1);
        const FixedScales z = fixed_scales(g.fbound, *g.d_bound, true);
        int64_t gc = 0;
        bool stop = false;
        for (int64_t it = blockIdx.x; it < g.n_items && !stop; it += gridDim.x) {
            const int64_t r = it / per_real, rem = it - r * per_real;
            const int64_t mt = rem / g.n_nb, nb = rem - mt * g.n_nb;
            const int64_t xi = mt * kXM + xrow, yj = nb * kXN + yrow;
            const float xa = (xrow >= 0 && xi < g.nx) ? *chk(g.x, xi, g.nx) : 0.0f;
            const float yb = (yrow >= 0 && yj < g.ny) ? *chk(g.y, yj, g.ny) : 0.0f;
            const int32_t XA = __float2int_rn(xa * z.xscale), YB = __float2int_rn(yb * z.xscale);
            for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                const int s = (int)(gc % kXStages);
                const uint32_t ph = (uint32_t)((gc / kXStages) & 1);
                if (*abort_flag ||
                    (gc >= kXStages && !sm100::mbar_wait(&empty[s], ph ^ 1u, abort_flag, kXWaitCycles)) ||
                    !sm100::mbar_wait(&fullR[gc % kXRecSlots], (uint32_t)((gc / kXRecSlots) & 1), abort_flag,
                                      kXWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                const int4* rr = reinterpret_cast<const int4*>(ringR(gc));
                if (z.use_fixed)
                    produce_share<PREC, true>(rr, stageA_hi(s), stageA_lo(s), stageB_hi(s), stageB_lo(s), t, XA, xa,
                                              YB, yb, z.bias, z.shift);
                else
                    produce_share<PREC, false>(rr, stageA_hi(s), stageA_lo(s), stageB_hi(s), stageB_lo(s), t, XA, xa,
                                               YB, yb, z.bias, z.shift);
                sm100::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    sm100::mbar_arrive(&full[s]);
                    sm100::mbar_arrive(&freeR[gc % kXRecSlots]);
                }
            }
        }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        if (*abort_flag && lane == 0 && mma_segments > 0) {  // MMAs in flight finish before TMEM is freed
            const int64_t Jl = mma_segments - 1;
            sm100::mbar_wait_for(&seg_full[Jl & 1], (uint32_t)((Jl >> 1) & 1), kXWaitCycles / 8);
        }
        __syncwarp();
        sm100::tc_fence_after();
        sm100::tmem_dealloc(tmem_base, 512);
    }
}

// ------------------------------------------------------------ CTA pairs
// k_grid_pair: the same product on a cluster of two CTAs (two SMs) sharing
// one tcgen05.mma of M = 256 (cta_group::2).  A work item is (realisation,
// pair of 128-column x tiles, 256-row y block): CTA rank q builds the x rows
// of tile 2 p + q (with the coefficient products) and y rows [128 q, 128 q +
// 128) of the block, so each SM produces 256 operand rows per K chunk instead
// of 384; the even CTA issues the MMAs for both (A: each CTA's own x rows; B:
// the two y halves), and each CTA's TMEM receives the 128 x 256 accumulator of
// its own x tile, promoted and stored by its own promoters as in k_grid_main.
// Three 64 KB stages.  Barriers: each CTA's producer and promoter warps
// arrive at their own full[s] and seg_free[b]; in the odd CTA one relay
// thread per barrier kind forwards each completed phase to the even CTA's
// barrier with a single release at cluster scope (a remote arrival from
// every warp would put a cluster-wide memory barrier on each of them); the
// MMA commits arrive at empty[s] and seg_full[b] in both CTAs (multicast).  A time-out in either CTA raises both abort flags;
// both CTAs meet at a cluster barrier before TMEM is freed, so no MMA of the
// pair is in flight and no remote arrival is pending when either exits.
// Producer warps per CTA, per precision: 8 (whole rows) or 16 (half rows).
// BF16X3 has twice the basis elements per K chunk and gains from 16; 3XTF32
// is fastest with 8 (less per-chunk synchronisation per element).
#ifndef QRS_GRID_PAIR_PRODUCERS_TF32
#define QRS_GRID_PAIR_PRODUCERS_TF32 8
#endif
#ifndef QRS_GRID_PAIR_PRODUCERS_BF16
#define QRS_GRID_PAIR_PRODUCERS_BF16 16
#endif

constexpr int kPStages = 3;
constexpr int kPHalfN = 128;                                   // y rows per CTA
constexpr int kPTileA = kXM * 128;                             // 16 KB
constexpr int kPTileB = kPHalfN * 128;                         // 16 KB
constexpr int kPStageBytes = 2 * kPTileA + 2 * kPTileB;        // 64 KB
// Promoter warps per CTA (4, 8 or 16, sharing each TMEM lane quarter's 256
// columns): the L2 reductions of a segment's slot then run from that many
// warps in parallel.
#ifndef QRS_GRID_PAIR_PROMOTERS_TF32
#define QRS_GRID_PAIR_PROMOTERS_TF32 8
#endif
#ifndef QRS_GRID_PAIR_PROMOTERS_BF16
#define QRS_GRID_PAIR_PROMOTERS_BF16 8
#endif
template <int PREC>
struct PairShape {
    static constexpr int kProducers =
        GemmCfg<PREC>::kTF32 ? QRS_GRID_PAIR_PRODUCERS_TF32 : QRS_GRID_PAIR_PRODUCERS_BF16;
    static constexpr int kPromoters =
        GemmCfg<PREC>::kTF32 ? QRS_GRID_PAIR_PROMOTERS_TF32 : QRS_GRID_PAIR_PROMOTERS_BF16;
    static constexpr int kThreads = 128 + 32 * (kPromoters + kProducers);
    static_assert(kProducers == 8 || kProducers == 16, "pair producer warps");
    static_assert(kPromoters == 4 || kPromoters == 8 || kPromoters == 16, "pair promoter warps");
};
// The operand stages, then the record ring and barriers, inside a region that
// extends 16 KB past the last stage's B tile (a read of twice a tile's rows
// from any tile start stays inside the CTA's allocation).
constexpr int kPRingOff = kPStages * kPStageBytes;
constexpr int kPSmemBytes = kPStages * kPStageBytes + 16 * 1024 + 1024;
static_assert(kPSmemBytes <= 232448 && kXSmemBytes <= 232448, "shared memory per CTA");
static_assert(kPRingOff + kXRecSlots * kXRecBytes + 512 <= kPStages * kPStageBytes + 16 * 1024, "ring fits the pad");

template <int PREC, bool FIXED, int NPROD>
__device__ __forceinline__ void produce_share_pair(const int4* __restrict__ rr, unsigned char* Ahi, unsigned char* Alo,
                                                   unsigned char* Bhi, unsigned char* Blo, int t, int32_t XA, float xa,
                                                   int32_t YB, float yb, uint64_t bias, uint32_t shift)
{
    constexpr bool CX = kXCoefX, CY = !kXCoefX;
    if (NPROD == 8) {
        if (t < kXM) produce_row<PREC, FIXED, 0, CX, 4, kPTileA>(rr, Ahi, Alo, t, 0, XA, xa, bias, shift);
        else produce_row<PREC, FIXED, 1, CY, 4, kPTileB>(rr, Bhi, Blo, t - kXM, 0, YB, yb, bias, shift);
    } else {
        if (t < 2 * kXM) produce_row<PREC, FIXED, 0, CX, 2, kPTileA>(rr, Ahi, Alo, t & 127, 2 * (t >> 7), XA, xa, bias, shift);
        else produce_row<PREC, FIXED, 1, CY, 2, kPTileB>(rr, Bhi, Blo, (t - 2 * kXM) & 127, 2 * ((t - 2 * kXM) >> 7), YB, yb,
                                                bias, shift);
    }
}

template <int PREC>
__global__ void __launch_bounds__(PairShape<PREC>::kThreads, 1) k_grid_pair(const __grid_constant__ GridArgs g)
{
    using Cfg = GemmCfg<PREC>;
    constexpr int kPProducers = PairShape<PREC>::kProducers;
    constexpr int kPPromoters = PairShape<PREC>::kPromoters;
    constexpr int T = Cfg::kTermsPerChunk;
    static_assert(T / Cfg::kTermsPer16B == 4, "four 16-byte groups per half row");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* rring = smem + kPRingOff;
    uint64_t* full = reinterpret_cast<uint64_t*>(rring + kXRecSlots * kXRecBytes);
    uint64_t* empty = full + kPStages;
    uint64_t* seg_full = empty + kPStages;  // [2]
    uint64_t* seg_free = seg_full + 2;      // [2]
    uint64_t* fullR = seg_free + 2;
    uint64_t* freeR = fullR + kXRecSlots;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(freeR + kXRecSlots);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = sm100::cluster_ctarank();
    const bool leader = rank == 0;
    const int64_t cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
    const int64_t n_chunks = g.n_chunks;
    const int64_t n_seg = (n_chunks + Cfg::kSeg - 1) / Cfg::kSeg;
    const int64_t n_mp = (g.n_mt + 1) >> 1;
    const int64_t per_real = n_mp * g.n_nb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPStages; ++s) {
            sm100::mbar_init(&full[s], leader ? kPProducers + 1 : kPProducers);  // + the peer's relay
            sm100::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            sm100::mbar_init(&seg_full[b], 1);
            sm100::mbar_init(&seg_free[b], leader ? kPPromoters + 1 : kPPromoters);
        }
        for (int s = 0; s < kXRecSlots; ++s) {
            sm100::mbar_init(&fullR[s], 1);
            sm100::mbar_init(&freeR[s], kPProducers);
        }
        *abort_flag = 0;
        sm100::fence_barrier_init();
    }
    if (warp == 1) sm100::tmem_alloc_pair(tmem_slot, 512);
    sm100::tc_fence_before();
    sm100::cluster_sync();  // both CTAs' barriers initialised before any remote arrival
    sm100::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto stageA_hi = [&](int s) { return smem + s * kPStageBytes; };
    auto stageA_lo = [&](int s) { return smem + s * kPStageBytes + kPTileA; };
    auto stageB_hi = [&](int s) { return smem + s * kPStageBytes + 2 * kPTileA; };
    auto stageB_lo = [&](int s) { return smem + s * kPStageBytes + 2 * kPTileA + kPTileB; };
    auto ringR = [&](int64_t i) { return rring + (i % kXRecSlots) * kXRecBytes; };
    const uint32_t peer_abort = sm100::mapa_shared((const void*)abort_flag, rank ^ 1u);
    auto timeout = [&]() {
        *abort_flag = 1;
        sm100::st_remote_u32(peer_abort, 1u);
        atomicExch(g.err, (int)QRS_ERR_TIMEOUT);
    };
    int64_t mma_segments = 0;

    if (warp == 1) {
        // ------------------------------------------ MMA issuer (even CTA)
        if (leader && lane == 0) {
            constexpr uint32_t idesc = sm100::idesc_f32acc(Cfg::kFormat, 2 * kXM, kXN);
            int64_t J = 0, gc = 0;
            bool stop = false;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                int64_t i = 0;
                for (int64_t j = 0; j < n_seg; ++j, ++J) {
                    const int b = (int)(J & 1);
                    if (*abort_flag ||
                        (J >= 2 && !sm100::mbar_wait_cluster(&seg_free[b], (uint32_t)(((J - 2) >> 1) & 1), abort_flag,
                                                             kXWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    const int64_t i_end = ((j + 1) * Cfg::kSeg < n_chunks) ? (j + 1) * Cfg::kSeg : n_chunks;
                    const uint32_t tmem_seg = tmem_base + (uint32_t)(b * kXN);
                    bool first = true;
                    for (; i < i_end; ++i, ++gc) {
                        const int s = (int)(gc % kPStages);
                        const uint32_t ph = (uint32_t)((gc / kPStages) & 1);
                        if (!sm100::mbar_wait_cluster(&full[s], ph, abort_flag, kXWaitCycles)) {
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
                            sm100::mma_pair<Cfg::kTF32>(tmem_seg, dAh, dBl, idesc, 1u);
                            sm100::mma_pair<Cfg::kTF32>(tmem_seg, dAl, dBh, idesc, 1u);
                        }
                        sm100::mma_commit_pair(&empty[s], (uint16_t)3);
                    }
                    sm100::mma_commit_pair(&seg_full[b], (uint16_t)3);
                    mma_segments = J + 1;
                    if (stop) break;
                }
            }
        }
    } else if (warp == 0 || warp == 3) {
        // ------------------------------------ relays (odd CTA): one release
        // at cluster scope per event instead of one per arriving warp.
        // Warp 0 forwards each completed phase of the local full[s] (all
        // producer warps wrote their operand rows) to the even CTA's full[s];
        // warp 3 each completed phase of seg_free[b] (all promoter warps
        // have read the slot).
        if (!leader && lane == 0) {
            uint64_t* local = warp == 0 ? full : seg_free;
            const int n_bar = warp == 0 ? kPStages : 2;
            const uint32_t remote0 = sm100::mapa_shared(local, 0u);
            const int64_t per_item = warp == 0 ? n_chunks : n_seg;
            int64_t e = 0;
            bool stop = false;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                for (int64_t i = 0; i < per_item; ++i, ++e) {
                    const int s = (int)(e % n_bar);
                    if (!sm100::mbar_wait(&local[s], (uint32_t)((e / n_bar) & 1), abort_flag, kXWaitCycles)) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    sm100::mbar_arrive_remote(remote0 + (uint32_t)(s * sizeof(uint64_t)));
                }
            }
        }
    } else if (warp == 2) {
        // ------------------------------------------------- record ring
        if (lane == 0) {
            int64_t gc = 0;
            bool stop = false;
            for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
                const int64_t r = it / per_real;
                const int4* src = g.rec + r * g.nf_pad;
                for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                    const int f = (int)(gc % kXRecSlots);
                    if (*abort_flag ||
                        (gc >= kXRecSlots && !sm100::mbar_wait(&freeR[f], (uint32_t)(((gc / kXRecSlots) & 1) ^ 1),
                                                               abort_flag, kXWaitCycles))) {
                        if (!*abort_flag) timeout();
                        stop = true;
                        break;
                    }
                    if (chk_ok(r * g.nf_pad + i * T, T, g.rec_rows * g.nf_pad)) {
                        sm100::mbar_arrive_expect_tx(&fullR[f], (uint32_t)(T * 16));
                        sm100::bulk_load(ringR(gc), src + i * T, (uint32_t)(T * 16), &fullR[f]);
                    } else {
                        sm100::mbar_arrive(&fullR[f]);  // checked build: the slot keeps its old records
                    }
                }
            }
            if (*abort_flag) {
                for (int64_t i = (gc > kXRecSlots ? gc - kXRecSlots : 0); i < gc; ++i)
                    sm100::mbar_wait_for(&fullR[i % kXRecSlots], (uint32_t)((i / kXRecSlots) & 1), kXWaitCycles / 8);
            }
        }
    } else if (warp >= 4 && warp < 4 + kPPromoters) {
        // ------------------------------------------------------ promoters
        constexpr int PC = QRS_GRID_PROMOTE_COLS;
        constexpr int kSpan = kXN / (kPPromoters / 4);  // columns per promoter warp
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int col0 = ((warp - 4) >> 2) * kSpan;
        const int64_t mq_off = (int64_t)blockIdx.x * kXN * kXM + (int64_t)quarter * kXN * 32;
        int64_t J = 0;
        bool stop = false;
        for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
            const int64_t r = it / per_real, rem = it - r * per_real;
            const int64_t mp = rem / g.n_nb, nb = rem - mp * g.n_nb;
            const int64_t xi = (2 * mp + rank) * kXM + row;
            const int64_t orow = g.r0 + r;
            for (int64_t j = 0; j < n_seg; ++j, ++J) {
                const int b = (int)(J & 1);
                if (!sm100::mbar_wait(&seg_full[b], (uint32_t)((J >> 1) & 1), abort_flag, kXWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                sm100::tc_fence_after();
                promote_red<PC>(g.master, (int64_t)gridDim.x * kXN * kXM, mq_off, tmem_base + (uint32_t)(b * kXN) + lane_off,
                                lane, j, j == n_seg - 1, col0, kSpan,
                                    [&](int c, float v) { store_node(g, orow, xi, nb * kXN + c, v); });
                sm100::tc_fence_before();
                __syncwarp();
                if (lane == 0) sm100::mbar_arrive(&seg_free[b]);
            }
        }
    } else if (warp >= 4 + kPPromoters) {
        // ------------------------------------------------------ producers
        const int t = (warp - 4 - kPPromoters) * 32 + lane;
        const int xrow = kPProducers == 8 ? (t < kXM ? t : -1) : (t < 2 * kXM ? (t & 127) : -1);
        const int yrow = kPProducers == 8 ? (t >= kXM ? t - kXM : -1) : (t >= 2 * kXM ? ((t - 2 * kXM) & 127) : -1);
        const FixedScales z = fixed_scales(g.fbound, *g.d_bound, true);
        int64_t gc = 0;
        bool stop = false;
        for (int64_t it = cluster; it < g.n_items && !stop; it += n_clusters) {
            const int64_t r = it / per_real, rem = it - r * per_real;
            const int64_t mp = rem / g.n_nb, nb = rem - mp * g.n_nb;
            const int64_t xi = (2 * mp + rank) * kXM + xrow, yj = nb * kXN + rank * kPHalfN + yrow;
            const float xa = (xrow >= 0 && xi < g.nx) ? *chk(g.x, xi, g.nx) : 0.0f;
            const float yb = (yrow >= 0 && yj < g.ny) ? *chk(g.y, yj, g.ny) : 0.0f;
            const int32_t XA = __float2int_rn(xa * z.xscale), YB = __float2int_rn(yb * z.xscale);
            for (int64_t i = 0; i < n_chunks; ++i, ++gc) {
                const int s = (int)(gc % kPStages);
                const uint32_t ph = (uint32_t)((gc / kPStages) & 1);
                if (*abort_flag ||
                    (gc >= kPStages && !sm100::mbar_wait(&empty[s], ph ^ 1u, abort_flag, kXWaitCycles)) ||
                    !sm100::mbar_wait(&fullR[gc % kXRecSlots], (uint32_t)((gc / kXRecSlots) & 1), abort_flag,
                                      kXWaitCycles)) {
                    if (!*abort_flag) timeout();
                    stop = true;
                    break;
                }
                const int4* rr = reinterpret_cast<const int4*>(ringR(gc));
                if (z.use_fixed)
                    produce_share_pair<PREC, true, kPProducers>(rr, stageA_hi(s), stageA_lo(s), stageB_hi(s), stageB_lo(s), t, XA,
                                                   xa, YB, yb, z.bias, z.shift);
                else
                    produce_share_pair<PREC, false, kPProducers>(rr, stageA_hi(s), stageA_lo(s), stageB_hi(s), stageB_lo(s), t, XA,
                                                    xa, YB, yb, z.bias, z.shift);
                sm100::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    sm100::mbar_arrive(&full[s]);
                    sm100::mbar_arrive(&freeR[gc % kXRecSlots]);
                }
            }
        }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0 && leader && *abort_flag && mma_segments > 0) {
        const int64_t Jl = mma_segments - 1;  // the pair's MMAs in flight finish first
        sm100::mbar_wait_cluster_for(&seg_full[Jl & 1], (uint32_t)((Jl >> 1) & 1), kXWaitCycles / 8);
    }
    __syncwarp();
    sm100::cluster_sync();  // neither CTA frees TMEM or exits while the pair still works on it
    if (warp == 1) {
        sm100::tc_fence_after();
        sm100::tmem_dealloc_pair(tmem_base, 512);
    }
}

// ------------------------------------------------------------------ host
static int64_t grid_terms_per_chunk(int mode)
{
    return mode == QRS_SYNTH_GEMM_3XTF32 ? GemmCfg<QRS_SYNTH_GEMM_3XTF32>::kTermsPerChunk
                                         : GemmCfg<QRS_SYNTH_GEMM_BF16X3>::kTermsPerChunk;
}

static int64_t grid_slab(int64_t nf_pad, int64_t n_real)
{
    int64_t s = (int64_t)(kXSlabBytes / ((size_t)nf_pad * sizeof(int4)));
    if (s < 1) s = 1;
    return s < n_real ? s : n_real;
}

static size_t grid_record_bytes(int64_t nf_pad, int64_t n_real)
{
    return ((size_t)grid_slab(nf_pad, n_real) * (size_t)nf_pad * sizeof(int4) + 255) / 256 * 256;
}

size_t grid_workspace_bytes(int mode, int64_t n_f, int64_t n_real, int num_sms)
{
    const int64_t T = grid_terms_per_chunk(mode);
    const int64_t nf_pad = (n_f + T - 1) / T * T;
    return 256 + grid_record_bytes(nf_pad, n_real) + (size_t)num_sms * kXN * kXM * sizeof(float);
}

int64_t grid_launch_count(int mode, int64_t n_f, int64_t n_real)
{
    const int64_t T = grid_terms_per_chunk(mode);
    const int64_t nf_pad = (n_f + T - 1) / T * T;
    const int64_t slab = grid_slab(nf_pad, n_real);
    return 1 + 2 * ((n_real + slab - 1) / slab);
}

static void pair_launch_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute (&at)[1], unsigned grid, int threads,
                               cudaStream_t s)
{
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = kPSmemBytes;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

// Clusters of two k_grid_pair CTAs the GPU holds at once (cached per handle
// and precision); 0 when pairs are switched off (QRS_GRID_PAIR=0 at
// qrs_create) or unavailable.
template <int PREC>
static int grid_pair_clusters(qrs_handle* h)
{
    int& c = h->grid_pair_clusters[PREC == QRS_SYNTH_GEMM_3XTF32 ? 0 : 1];
    if (!h->grid_pair) return 0;
    if (c == 0) {
        int n = 0;
        cudaError_t e =
            cudaFuncSetAttribute(k_grid_pair<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmemBytes);
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            pair_launch_config(cfg, at, (unsigned)(h->num_sms & ~1), PairShape<PREC>::kThreads, nullptr);
            e = cudaOccupancyMaxActiveClusters(&n, k_grid_pair<PREC>, &cfg);
        }
        if (e != cudaSuccess) cudaGetLastError();  // the single-SM kernel serves instead
        c = (e == cudaSuccess && n > 0) ? (n < h->num_sms / 2 ? n : h->num_sms / 2) : -1;
    }
    return c > 0 ? c : 0;
}

template <int PREC>
static cudaError_t launch_grid_t(qrs_handle* h, const DrawParams& p, const float* x, int64_t nx, const float* y,
                                 int64_t ny, const int32_t* index, int64_t P, int64_t n_real, float* out,
                                 cudaStream_t s)
{
    using Cfg = GemmCfg<PREC>;
    constexpr int T = Cfg::kTermsPerChunk;
    const int64_t nf_pad = (p.n_f + T - 1) / T * T;
    const int64_t slab = grid_slab(nf_pad, n_real);
    int4* rec = reinterpret_cast<int4*>(((uintptr_t)h->d_work + 255) & ~(uintptr_t)255);
    float* master = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(rec) + grid_record_bytes(nf_pad, n_real));

    k_grid_bound<<<1, 1024, 0, s>>>(x, nx, y, ny, h->d_xbound);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_grid_main<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kXSmemBytes);
    if (e != cudaSuccess) return e;
    GridArgs a;
    a.x = x;
    a.nx = nx;
    a.y = y;
    a.ny = ny;
    a.index = index;
    a.P = P;
    a.out = out;
    a.nf_pad = nf_pad;
    a.n_chunks = nf_pad / T;
    a.n_mt = (nx + kXM - 1) / kXM;
    a.n_nb = (ny + kXN - 1) / kXN;
    a.rec = rec;
    a.out_rows = n_real;
    a.master = master;
    a.d_bound = h->d_xbound;
    a.fbound = (float)freq_bound(p);
    a.err = h->d_err;
    // CTA pairs when there are x tiles to pair and the GPU can hold a pair
    const int clusters = a.n_mt >= 2 ? grid_pair_clusters<PREC>(h) : 0;
    for (int64_t r0 = 0; r0 < n_real; r0 += slab) {
        const int64_t nr = (n_real - r0 < slab) ? n_real - r0 : slab;
        DrawParams ps = p;
        ps.real_offset = p.real_offset + r0;
        const int64_t total = nr * nf_pad;
        const int64_t blocks = (total + 255) / 256;
        const unsigned gd = (unsigned)(blocks < 8LL * h->num_sms ? blocks : 8LL * h->num_sms);
        k_grid_draw<<<gd, 256, 0, s>>>(ps, nr, nf_pad, h->d_xbound, a.fbound, rec);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        a.r0 = r0;
        a.rec_rows = nr;
        if (clusters > 0) {
            a.n_items = nr * ((a.n_mt + 1) / 2) * a.n_nb;
            const int64_t nc = a.n_items < clusters ? a.n_items : clusters;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            pair_launch_config(cfg, at, (unsigned)(2 * nc), PairShape<PREC>::kThreads, s);
            e = cudaLaunchKernelEx(&cfg, k_grid_pair<PREC>, a);
        } else {
            a.n_items = nr * a.n_mt * a.n_nb;
            const int64_t ctas = a.n_items < h->num_sms ? a.n_items : h->num_sms;
            k_grid_main<PREC><<<(unsigned)ctas, kXThreads, kXSmemBytes, s>>>(a);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_synth_grid(qrs_handle* h, int mode, const DrawParams& p, const float* x, int64_t nx,
                              const float* y, int64_t ny, const int32_t* index, int64_t P, int64_t n_real, float* out,
                              cudaStream_t s)
{
    if (mode == QRS_SYNTH_GEMM_3XTF32)
        return launch_grid_t<QRS_SYNTH_GEMM_3XTF32>(h, p, x, nx, y, ny, index, P, n_real, out, s);
    return launch_grid_t<QRS_SYNTH_GEMM_BF16X3>(h, p, x, nx, y, ny, index, P, n_real, out, s);
}

}  // namespace qrs
