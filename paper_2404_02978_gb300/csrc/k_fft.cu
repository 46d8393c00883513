// k_fft.cu -- the spectrum of the FFT screen (Eq. 2), the paper's comparison
// method (Sec. 2.2): static sampling of the frequency plane on the grid of an
// n x n screen of pitch dx,
//   S[r][i][j] = (a + i b) sqrt(W(f)) A(|f|) df,  f = (j', i') df,  df = 1 / (n dx),
// j' the signed FFT index (j < (n + 1) / 2 ? j : j - n), a, b ~ N(0,1) by
// Box-Muller from words 2 and 3 of the Philox4x32-10 counter
// ((real_offset + r) n^2 + i n + j, stream 4), A the Eq. 7 filter of the PSD
// (1 without), and S = 0 at f = 0.  The screen itself is n^2 times the
// inverse DFT of S, left to an FFT library (cuFFT) by the caller: the method
// of the paper is the direct sum; this baseline shows what the static
// sampling it replaces does to the structure function.
//
// One thread per spectral sample, grid-stride; HBM-bound output (8 bytes per
// sample) over a Philox + Box-Muller + PSD computation per sample.
#include <algorithm>
#include <cmath>

#include "qrs_internal.h"

namespace qrs {

QRS_CHECK_HOOK(check_hook_fft)

constexpr uint32_t kStreamFft = 4u;

__global__ void k_fft_spectrum(float psd_c, float psd_a, float ap_D, float ap_d, float df, int64_t n, int64_t total,
                               uint64_t idx0, uint32_t key0, uint32_t key1, float2* __restrict__ spec)
{
    const int64_t half = (n + 1) / 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ij = e % (n * n);
        const int64_t i = ij / n, j = ij - i * n;
        float2 v = make_float2(0.0f, 0.0f);
        if (ij != 0) {
            const uint64_t c = idx0 + (uint64_t)e;
            const Words w = philox4x32_10((uint32_t)c, (uint32_t)(c >> 32), kStreamFft, 0u, key0, key1);
            const float U1 = (float)((w.w2 >> 8) + 1u) * 0x1p-24f;
            const float U2 = (float)(w.w3 >> 8) * 0x1p-24f;
            const float rad = sqrtf(-2.0f * logf(U1));
            float sb, cb;
            sincospif(2.0f * U2, &sb, &cb);
            const float fx = (float)(j < half ? j : j - n) * df;
            const float fy = (float)(i < half ? i : i - n) * df;
            const float f2 = fx * fx + fy * fy;
            float F = sqrtf(psd_w(psd_c, psd_a, f2)) * df;
            if (ap_D > 0.0f) F *= airy_filter(sqrtf(f2), ap_D, ap_d);
            v = make_float2(F * (rad * cb), F * (rad * sb));
        }
        *chk(spec, e, total) = v;
    }
}

}  // namespace qrs

using namespace qrs;

extern "C" qrs_status qrs_fft_spectrum(qrs_handle* h, const qrs_psd* psd, int64_t n, double dx, uint64_t seed,
                                       int64_t n_real, int64_t real_offset, float* spec, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_fft_spectrum");
    if (qrs::injected_launch_fault(h, "qrs_fft_spectrum") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (n < 2 || n > 32768) return fail(h, QRS_ERR_ARG, "n must be in [2, 32768]");
    if (!(std::isfinite(dx) && dx > 0.0)) return fail(h, QRS_ERR_ARG, "dx must be finite and > 0");
    if (n_real < 0 || real_offset < 0) return fail(h, QRS_ERR_ARG, "n_real and real_offset must be >= 0");
    // the PSD's checks and constants are those of a draw (a one-term SQUARE domain stands in for the grid)
    qrs_domain dom{};
    dom.kind = QRS_DOMAIN_SQUARE;
    dom.fmax = 0.5 / dx;
    qrs_sampler smp{};
    smp.kind = QRS_SAMPLER_R2;
    smp.n_rho = smp.n_theta = 1;
    smp.seed = seed;
    DrawParams p;
    if (psd && psd->kind == QRS_PSD_KOLMOGOROV) {
        // the Kolmogorov PSD is finite at every grid frequency but f = 0, whose sample is 0
        qrs_psd vk = *psd;
        vk.kind = QRS_PSD_VON_KARMAN;
        vk.L0_m = 1.0;
        qrs_status st = make_draw_params(h, &vk, &dom, &smp, 1, 0, &p);
        if (st != QRS_OK) return st;
        p.psd_a = 0.0f;
    } else {
        qrs_status st = make_draw_params(h, psd, &dom, &smp, 1, 0, &p);
        if (st != QRS_OK) return st;
    }
    const uint64_t nn = (uint64_t)n * (uint64_t)n;
    if (!counters_fit((int64_t)nn, real_offset, n_real)) return fail(h, QRS_ERR_ARG, "stream index overflows 2^64");
    if ((unsigned __int128)(uint64_t)n_real * nn >= ((unsigned __int128)1 << 62))
        return fail(h, QRS_ERR_ARG, "n_real n^2 spectral samples exceed 2^62");
    if (n_real == 0) return QRS_OK;
    if (!spec || ((uintptr_t)spec & 7)) return fail(h, QRS_ERR_ARG, "spec must be non-NULL and 8-byte aligned");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) {
        const int64_t total = n_real * (int64_t)nn;
        const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)h->num_sms * 8);
        k_fft_spectrum<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
            p.psd_c, p.psd_a, p.ap_D, p.ap_d, (float)(1.0 / ((double)n * dx)), n, total,
            (uint64_t)real_offset * nn, p.key0, p.key1, reinterpret_cast<float2*>(spec));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_fft_spectrum launch");
    ++h->launches;
    return QRS_OK;
}
