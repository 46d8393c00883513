// qrs_tc_split.cuh -- operand formats of the tensor-core products (split
// 3XTF32 and BF16X3, single-pass TF32) shared by the shared-draw GEMM
// (k_gemm.cu; all three) and the
// separable-grid form (k_grid.cu): per-format K-chunk geometry, accumulation
// segment lengths, and the hi/lo split of FP32 values into 16-byte pieces of
// a 128-byte-swizzled K-major operand row.
#pragma once

#include <cuda_bf16.h>

#include "qrs_internal.h"
#include "qrs_sm100.cuh"

#ifndef QRS_GEMM_SEG_TF32
#define QRS_GEMM_SEG_TF32 6   // K chunks per accumulation segment, 3XTF32 (72 accumulation steps)
#endif
#ifndef QRS_GEMM_SEG_TF32_SINGLE
#define QRS_GEMM_SEG_TF32_SINGLE 18  // K chunks per accumulation segment, single TF32 (72 accumulation steps)
#endif
// BF16X3's error is set by its 8-bit split (about 2^-17 per product), not by
// the accumulation drift: 16-chunk segments raise its largest measured error
// from 2.7e-5 to 3.1e-5 sigma (bar 5e-5) and halve the promotions.
#ifndef QRS_GEMM_SEG_BF16
#define QRS_GEMM_SEG_BF16 16  // K chunks per accumulation segment, BF16X3 (192 accumulation steps)
#endif
#ifndef QRS_GEMM_INTSPLIT
#define QRS_GEMM_INTSPLIT 1   // hi/lo splits by integer rounding (ALU) instead of conversions
#endif
#ifndef QRS_BF16_PACKED_CVT
#define QRS_BF16_PACKED_CVT 1 // BF16 halves by the paired conversion cvt.rn.bf16x2.f32
#endif

namespace qrs {

template <int PREC>
struct GemmCfg;
template <>
struct GemmCfg<QRS_SYNTH_GEMM_3XTF32> {
    static constexpr int kElemBytes = 4;
    static constexpr int kElemsPerRow = 32;    // one 128-byte row of a K chunk
    static constexpr int kTermsPerChunk = 16;  // cos and sin of 16 terms
    static constexpr int kTermsPer16B = 4;
    static constexpr uint32_t kFormat = 2;     // TF32
    static constexpr bool kTF32 = true;
    static constexpr bool kSplit = true;       // hi and lo halves, three products
    static constexpr int kSeg = QRS_GEMM_SEG_TF32;
};
// Single-pass TF32: each operand rounded once to TF32 (11 significant bits),
// one product per K step.
template <>
struct GemmCfg<QRS_SYNTH_GEMM_TF32> {
    static constexpr int kElemBytes = 4;
    static constexpr int kElemsPerRow = 32;
    static constexpr int kTermsPerChunk = 16;
    static constexpr int kTermsPer16B = 4;
    static constexpr uint32_t kFormat = 2;
    static constexpr bool kTF32 = true;
    static constexpr bool kSplit = false;
    static constexpr int kSeg = QRS_GEMM_SEG_TF32_SINGLE;
};
template <>
struct GemmCfg<QRS_SYNTH_GEMM_BF16X3> {
    static constexpr int kElemBytes = 2;
    static constexpr int kElemsPerRow = 64;
    static constexpr int kTermsPerChunk = 32;
    static constexpr int kTermsPer16B = 8;
    static constexpr uint32_t kFormat = 1;     // BF16
    static constexpr bool kTF32 = false;
    static constexpr bool kSplit = true;
    static constexpr int kSeg = QRS_GEMM_SEG_BF16;
};

// TF32 rounding to nearest, ties away from zero (as cvt.rna.tf32.f32): add half
// of the dropped 13-bit field to the magnitude bits, then clear the field.
__device__ __forceinline__ uint32_t tf32_rna_bits(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
// BF16 rounding to nearest, ties to even (as cvt.rn.bf16.f32), as FP32 bits.
__device__ __forceinline__ uint32_t bf16_rne_bits(float x)
{
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
}

// Split 16 bytes' worth of values into hi and lo halves in the operand format
// (TF32 in 32-bit words with the low 13 bits zero, or pairs of BF16); the
// residual x - hi is exact in FP32.
template <int PREC>
__device__ __forceinline__ void pack16(const float (&v)[GemmCfg<PREC>::kTermsPer16B], uint4& hi, uint4& lo)
{
    uint32_t* wh = reinterpret_cast<uint32_t*>(&hi);
    uint32_t* wl = reinterpret_cast<uint32_t*>(&lo);
    if (!GemmCfg<PREC>::kSplit) {  // one TF32 rounding per value, no low half
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            wh[e] = tf32_rna_bits(v[e]);
            wl[e] = 0u;
        }
    } else if (GemmCfg<PREC>::kTF32) {
#if QRS_GEMM_INTSPLIT
        // residuals x - hi two at a time, as fma(hi, -1, x) (exact, the same bits)
#pragma unroll
        for (int e = 0; e < 4; e += 2) {
            const uint32_t h0 = tf32_rna_bits(v[e]), h1 = tf32_rna_bits(v[e + 1]);
            const float2 r = __ffma2_rn(make_float2(__uint_as_float(h0), __uint_as_float(h1)), make_float2(-1.0f, -1.0f),
                                        make_float2(v[e], v[e + 1]));
            wh[e] = h0;
            wh[e + 1] = h1;
            wl[e] = tf32_rna_bits(r.x);
            wl[e + 1] = tf32_rna_bits(r.y);
        }
#else
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v[e]));
            const float r = v[e] - __uint_as_float(h);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
            wh[e] = h;
            wl[e] = l;
        }
#endif
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float x0 = v[2 * e], x1 = v[2 * e + 1];
#if QRS_BF16_PACKED_CVT
            // one conversion rounds both values (x1 to the high half); the
            // residuals x - hi are exact in FP32 and converted the same way
            uint32_t h, l;
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
            const float2 r = __ffma2_rn(make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xFFFF0000u)),
                                        make_float2(-1.0f, -1.0f), make_float2(x0, x1));  // x - hi, exact
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(r.y), "f"(r.x));
            wh[e] = h;
            wl[e] = l;
#elif QRS_GEMM_INTSPLIT
            const uint32_t h0 = bf16_rne_bits(x0), h1 = bf16_rne_bits(x1);
            const uint32_t l0 = bf16_rne_bits(x0 - __uint_as_float(h0));
            const uint32_t l1 = bf16_rne_bits(x1 - __uint_as_float(h1));
            wh[e] = __byte_perm(h0, h1, 0x7632);  // (h1 top half << 16) | h0 top half
            wl[e] = __byte_perm(l0, l1, 0x7632);
#else
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            wh[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            wl[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
#endif
        }
    }
}

// Segment promotion of a 128 x 256 TMEM accumulator slot into an FP32
// master held in global memory (L2), by one promoter warp: TMEM lanes of its
// quarter (slot_q carries the lane offset), columns [col0, col0 + span), PC
// columns per TMEM load.  The master of the CTA sits at master + mq_off (the
// quarter's base) as [column][32 lanes], so the warp's accesses to a column
// are one 128-byte run --
//   first segment:   master := slot;
//   later segments:  master += slot by FP32 reductions in L2 (red.global.add,
//                    one rounded add per element, the same as master + slot
//                    in registers), issued without waiting for a reply;
//   last segment:    value = slot + master (this thread's own reductions are
//                    ordered before its loads of the same addresses), or the
//                    slot alone when there is one segment, to store(column,
//                    value).
// (Four-wide vector reductions measured slower.)  The tensor core's FP32
// accumulation loses about 2^-26 per step with a consistent sign;
// restarting the slot each segment and adding segments in FP32 with round
// to nearest bounds that drift.
template <int PC, class Store>
__device__ __forceinline__ void promote_red(float* master, int64_t n_master, int64_t mq_off, uint32_t slot_q, int lane,
                                            int64_t j, bool last, int col0, int span, Store&& store)
{
    if (last && j > 0) __threadfence();
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
                                           *chk(master, mq_off + (int64_t)(c0 + q) * 32 + lane, n_master));
            }
#pragma unroll
            for (int q = 0; q < PC; ++q) store(c0 + q, __uint_as_float(v[q]));
        } else {
#pragma unroll
            for (int q = 0; q < PC; ++q) {
                float* a = chk(master, mq_off + (int64_t)(c0 + q) * 32 + lane, n_master);
                if (j == 0) *a = __uint_as_float(v[q]);
                else sm100::red_add_f32(a, __uint_as_float(v[q]));
            }
        }
    }
}

// The same promotion with the master in TMEM (a second 128 x 256 region,
// master_q with the lane offset): master := slot / master += slot through
// tcgen05.ld / tcgen05.st, value = slot + master at the last segment.  No
// memory traffic, but the slot and the master fill TMEM, so the MMAs of the
// next segment wait until the promotion has read the slot.
template <int PC, class Store>
__device__ __forceinline__ void promote_tmem(uint32_t master_q, uint32_t slot_q, int64_t j, bool last, int col0,
                                             int span, Store&& store)
{
#pragma unroll 1
    for (int c0 = col0; c0 < col0 + span; c0 += PC) {
        uint32_t v[PC], w[PC];
        sm100::tmem_ld_cols(slot_q + (uint32_t)c0, v);
        if (j > 0) sm100::tmem_ld_cols(master_q + (uint32_t)c0, w);
        sm100::tmem_ld_wait();
        if (j > 0) {
#pragma unroll
            for (int q = 0; q < PC; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(w[q]));
        }
        if (!last) {
            sm100::tmem_st_cols(master_q + (uint32_t)c0, v);
        } else {
#pragma unroll
            for (int q = 0; q < PC; ++q) store(c0 + q, __uint_as_float(v[q]));
        }
    }
    sm100::tmem_st_wait();
}

}  // namespace qrs
