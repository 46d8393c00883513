// k_draw.cu -- K1: the frequency draw exported as arrays (qrs_draw).
// One thread per (realisation, term); every output optional.  The same
// draw_term() feeds the fused synthesis and piston kernels, so what this
// kernel exports is exactly what those kernels sum.
#include "qrs_internal.h"

namespace qrs {

QRS_CHECK_HOOK(check_hook_draw)

__global__ void k_draw(DrawParams p, int64_t n_real, float* __restrict__ f_xy, float* __restrict__ amp,
                       float* __restrict__ coef, int32_t* __restrict__ cell, uint32_t* __restrict__ words,
                       uint64_t* __restrict__ r2)
{
    const int64_t total = n_real * p.n_f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / p.n_f, k = i - r * p.n_f;
        const uint64_t n = (uint64_t)(p.real_offset + r) * (uint64_t)p.n_f + (uint64_t)k;
        Words w;
        uint64_t Sx, Sy;
        const Term t = draw_term(p, n, k, &w, &Sx, &Sy);
        if (f_xy) *chk(reinterpret_cast<float2*>(f_xy), i, total) = make_float2(t.fx, t.fy);
        if (amp) *chk(amp, i, total) = t.F;
        if (coef) *chk(reinterpret_cast<float2*>(coef), i, total) = make_float2(t.a, t.b);
        if (cell) *chk(cell, i, total) = t.cell;
        if (words) *chk(reinterpret_cast<uint4*>(words), i, total) = make_uint4(w.w0, w.w1, w.w2, w.w3);
        if (r2) { *chk(r2, 2 * i, 2 * total) = Sx; *chk(r2, 2 * i + 1, 2 * total) = Sy; }
    }
}

cudaError_t launch_draw(const DrawParams& p, int64_t n_real, const qrs_draw_out& o, cudaStream_t s)
{
    const int64_t total = n_real * p.n_f;
    const int tpb = 256;
    int64_t blocks = (total + tpb - 1) / tpb;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    k_draw<<<(unsigned)blocks, tpb, 0, s>>>(p, n_real, o.f_xy, o.amp, o.coef, o.cell, o.words, o.r2);
    return cudaGetLastError();
}

}  // namespace qrs
