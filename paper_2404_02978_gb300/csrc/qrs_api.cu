// qrs_api.cu -- the C ABI of libqrs (include/qrs.h): handle, argument
// validation, draw parameters, dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "qrs_internal.h"
#include "qrs_piston.h"

namespace qrs {

QRS_CHECK_HOOK(check_hook_api)

qrs_status fail(qrs_handle* h, qrs_status st, const char* fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        h->last_error = buf;
    }
    return st;
}

qrs_status cuda_fail(qrs_handle* h, cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation) return fail(h, QRS_ERR_NOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(h, QRS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

qrs_status injected_launch_fault(qrs_handle* h, const char* where)
{
    if (h->fault & kFaultLaunch) return fail(h, QRS_ERR_CUDA, "%s: injected launch failure (QRS_FAULT=launch)", where);
    return QRS_OK;
}

qrs_status ensure_work(qrs_handle* h, size_t bytes)
{
    if (h->work_bytes >= bytes) return QRS_OK;
    if (h->fault & kFaultAlloc) return fail(h, QRS_ERR_NOMEM, "injected workspace allocation failure (QRS_FAULT=alloc)");
    if (h->d_work) {
        cudaError_t e = cudaDeviceSynchronize();  // workspace may be in use by earlier launches
        if (e != cudaSuccess) return cuda_fail(h, e, "workspace sync");
        cudaFree(h->d_work);
        h->d_work = nullptr;
        h->work_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&h->d_work, want);
    if (e != cudaSuccess) return cuda_fail(h, e, "workspace allocation");
    h->work_bytes = want;
    return QRS_OK;
}

// Von Karman constant c = Gamma(11/6)^2 / (2 pi^(11/3)) (24/5 Gamma(6/5))^(5/6), from tgamma.
static double vk_constant()
{
    const double pi = 3.14159265358979323846;
    return std::tgamma(11.0 / 6.0) * std::tgamma(11.0 / 6.0) / (2.0 * std::pow(pi, 11.0 / 3.0)) *
           std::pow(24.0 / 5.0 * std::tgamma(6.0 / 5.0), 5.0 / 6.0);
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

qrs_status make_draw_params(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, const qrs_sampler* smp,
                            int64_t n_f, int64_t real_offset, DrawParams* out)
{
    if (!psd || !dom || !smp) return fail(h, QRS_ERR_ARG, "psd, domain and sampler must be non-NULL");
    if (psd->kind != QRS_PSD_VON_KARMAN && psd->kind != QRS_PSD_KOLMOGOROV)
        return fail(h, QRS_ERR_ARG, "unknown psd kind %d", psd->kind);
    if (!finite_pos(psd->r0_m)) return fail(h, QRS_ERR_ARG, "r0 must be finite and > 0");
    if (psd->kind == QRS_PSD_VON_KARMAN && !finite_pos(psd->L0_m))
        return fail(h, QRS_ERR_ARG, "L0 must be finite and > 0 for the von Karman PSD");
    if (!(std::isfinite(psd->ap_D_m) && std::isfinite(psd->ap_d_m) && psd->ap_D_m >= 0.0 && psd->ap_d_m >= 0.0 &&
          (psd->ap_D_m > 0.0 ? psd->ap_d_m < psd->ap_D_m : psd->ap_d_m == 0.0)))
        return fail(h, QRS_ERR_ARG, "aperture filter: 0 <= ap_d < ap_D, or ap_D = ap_d = 0 for none");
    if (dom->kind < QRS_DOMAIN_SQUARE || dom->kind > QRS_DOMAIN_LOGPOLAR)
        return fail(h, QRS_ERR_ARG, "unknown domain kind %d", dom->kind);
    if (!finite_pos(dom->fmax)) return fail(h, QRS_ERR_ARG, "fmax must be finite and > 0");
    if (dom->kind == QRS_DOMAIN_LOGPOLAR && !(finite_pos(dom->fmin) && dom->fmin < dom->fmax))
        return fail(h, QRS_ERR_ARG, "LOGPOLAR needs 0 < fmin < fmax");
    if (psd->kind == QRS_PSD_KOLMOGOROV && dom->kind != QRS_DOMAIN_LOGPOLAR)
        return fail(h, QRS_ERR_ARG, "the Kolmogorov PSD is infinite at f = 0: use a LOGPOLAR domain (fmin > 0)");
    if (smp->kind < QRS_SAMPLER_R2 || smp->kind > QRS_SAMPLER_IMPORTANCE)
        return fail(h, QRS_ERR_ARG, "unknown sampler kind %d", smp->kind);
    if (smp->coef_kind != QRS_COEF_GAUSS && smp->coef_kind != QRS_COEF_EQ3)
        return fail(h, QRS_ERR_ARG, "unknown coefficient kind %d", smp->coef_kind);
    if (smp->n_rho < 1 || smp->n_theta < 1 || (int64_t)smp->n_rho * smp->n_theta > (1 << 24))
        return fail(h, QRS_ERR_ARG, "cell grid n_rho x n_theta must be in [1, 2^24]");
    if (n_f < 1 || n_f >= ((int64_t)1 << 31)) return fail(h, QRS_ERR_ARG, "n_f must be in [1, 2^31)");
    if (real_offset < 0) return fail(h, QRS_ERR_ARG, "real_offset must be >= 0");
    if (smp->kind == QRS_SAMPLER_JITTER && n_f != (int64_t)smp->n_rho * smp->n_theta)
        return fail(h, QRS_ERR_ARG, "JITTER needs n_f == n_rho * n_theta (one point per cell, Eq. 4)");
    if (smp->kind == QRS_SAMPLER_IMPORTANCE) {
        if (dom->kind != QRS_DOMAIN_LOGPOLAR) return fail(h, QRS_ERR_ARG, "IMPORTANCE cells need a LOGPOLAR domain");
        if (!smp->cell_cdf) return fail(h, QRS_ERR_ARG, "IMPORTANCE needs cell_cdf");
        if (((uintptr_t)smp->cell_cdf & 3) != 0) return fail(h, QRS_ERR_ARG, "cell_cdf must be 4-byte aligned");
        if (smp->fold != 0 && smp->fold != 1 && smp->fold != 2 && smp->fold != 4)
            return fail(h, QRS_ERR_ARG, "fold must be 0, 1, 2 or 4");
        if (!std::isfinite(smp->frame)) return fail(h, QRS_ERR_ARG, "frame must be finite");
    } else if ((smp->fold != 0 && smp->fold != 1) || smp->frame != 0.0) {
        return fail(h, QRS_ERR_ARG, "fold and frame apply to the IMPORTANCE sampler only");
    }
    DrawParams p;
    std::memset(&p, 0, sizeof(p));
    p.fmin = dom->kind == QRS_DOMAIN_LOGPOLAR ? dom->fmin : 0.0;
    p.fmax = dom->fmax;
    p.log_ratio = dom->kind == QRS_DOMAIN_LOGPOLAR ? std::log(dom->fmax / dom->fmin) : 0.0;
    p.n_f = n_f;
    p.real_offset = real_offset;
    p.psd_c = (float)(vk_constant() * std::pow(psd->r0_m, -5.0 / 3.0));
    p.psd_a = psd->kind == QRS_PSD_KOLMOGOROV ? 0.0f : (float)(1.0 / (psd->L0_m * psd->L0_m));
    p.ap_D = (float)psd->ap_D_m;
    p.ap_d = (float)psd->ap_d_m;
    if (dom->kind == QRS_DOMAIN_LOGPOLAR) {
        const double l2 = std::log2(dom->fmax / dom->fmin);
        p.l2_hi = (float)l2;
        p.l2_lo = (float)(l2 - (double)p.l2_hi);
        p.fmin_hi = (float)dom->fmin;
        p.fmin_lo = (float)(dom->fmin - (double)p.fmin_hi);
    }
    const double pi = 3.14159265358979323846;
    if (dom->kind == QRS_DOMAIN_SQUARE) p.jac_c = (float)(4.0 * dom->fmax * dom->fmax);
    else if (dom->kind == QRS_DOMAIN_DISC) p.jac_c = (float)(pi * dom->fmax * dom->fmax);
    else p.jac_c = (float)(2.0 * pi * p.log_ratio);
    p.inv_nf = (float)(1.0 / (double)n_f);
    p.key0 = (uint32_t)smp->seed;
    p.key1 = (uint32_t)(smp->seed >> 32);
    if (smp->use_fixed_s0) {
        p.s0x = smp->s0[0];
        p.s0y = smp->s0[1];
    } else {
        const Words w = philox4x32_10(0u, 0u, kStreamSeed, 0u, p.key0, p.key1);
        p.s0x = ((uint64_t)w.w1 << 32) | w.w0;
        p.s0y = ((uint64_t)w.w3 << 32) | w.w2;
    }
    p.cdf = smp->cell_cdf;
    p.dom = dom->kind;
    p.smp = smp->kind;
    p.coef = smp->coef_kind;
    p.n_rho = smp->n_rho;
    p.n_theta = smp->n_theta;
    if (smp->kind == QRS_SAMPLER_IMPORTANCE) {
        p.fold_sh = smp->fold == 4 ? 2 : smp->fold == 2 ? 1 : 0;
        p.frame = smp->frame;
    }
    *out = p;
    return QRS_OK;
}

double freq_bound(const DrawParams& p) { return p.fmax; }

bool counters_fit(int64_t n_f, int64_t real_offset, int64_t n_real)
{
    // every realisation index real_offset + r stays within int64 and every
    // stream index (real_offset + r) n_f + k below 2^64; the sum is formed in
    // 128-bit unsigned arithmetic, so no signed overflow
    if (n_f < 0 || real_offset < 0 || n_real < 0) return false;
    const unsigned __int128 sum = (unsigned __int128)(uint64_t)real_offset + (uint64_t)n_real;
    if (sum > (unsigned __int128)INT64_MAX) return false;
    const unsigned __int128 top = sum * (unsigned __int128)(uint64_t)n_f;
    return (top >> 64) == 0;
}

}  // namespace qrs

using namespace qrs;

extern "C" {

qrs_status qrs_create(qrs_handle** out, int32_t device)
{
    if (!out) return QRS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return QRS_ERR_CUDA;
    if (device < 0 || device >= ndev) return QRS_ERR_ARG;
    qrs_handle* h = new (std::nothrow) qrs_handle();
    if (!h) return QRS_ERR_NOMEM;
    h->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, 64);
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, 64);
    if (e == cudaSuccess) h->d_xbound = reinterpret_cast<float*>(reinterpret_cast<char*>(h->d_err) + 16);
    if (const char* f = std::getenv("QRS_FAULT")) {
        if (std::strstr(f, "alloc")) h->fault |= kFaultAlloc;
        if (std::strstr(f, "launch")) h->fault |= kFaultLaunch;
        if (std::strstr(f, "timeout")) h->fault |= kFaultTimeout;
    }
    if (const char* f = std::getenv("QRS_GRID_PAIR")) h->grid_pair = std::strcmp(f, "0") != 0;
    if (const char* f = std::getenv("QRS_GEMM_PAIR")) h->gemm_pair = std::strcmp(f, "0") != 0;
    if (const char* f = std::getenv("QRS_SYNTH_ANCHOR")) h->synth_anchor = std::strcmp(f, "0") != 0;
    if (e == cudaSuccess && qrs::kChecked) {  // the checked build reports into this handle's error word
        for (cudaError_t (*hook)(int*) : {check_hook_api, check_hook_draw, check_hook_fft, check_hook_gemm,
                                          check_hook_grid, check_hook_piston, check_hook_proposal, check_hook_sf,
                                          check_hook_stats, check_hook_synth})
            if (e == cudaSuccess) e = hook(h->d_err);
    }
    if (e != cudaSuccess) {
        if (h->d_err) cudaFree(h->d_err);
        delete h;
        return e == cudaErrorMemoryAllocation ? QRS_ERR_NOMEM : QRS_ERR_CUDA;
    }
    *out = h;
    return QRS_OK;
}

void qrs_destroy(qrs_handle* h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    destroy_piston_state(h);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_work) cudaFree(h->d_work);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    delete h;
}

const char* qrs_last_error(const qrs_handle* h) { return h ? h->last_error.c_str() : "null handle"; }

int64_t qrs_launch_count(const qrs_handle* h) { return h ? h->launches : 0; }

namespace qrs {

__global__ void k_check_selftest(float* scratch, int64_t i)
{
    *chk(scratch, i, (int64_t)8) = 1.0f;
}

}  // namespace qrs

int32_t qrs_checked_build(void) { return qrs::kChecked ? 1 : 0; }

qrs_status qrs_check_selftest(qrs_handle* h, int64_t i, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    h->last_error.clear();
    if (!qrs::kChecked) return fail(h, QRS_ERR_ARG, "qrs_check_selftest needs the bounds-checked library");
    float* scratch = reinterpret_cast<float*>(reinterpret_cast<char*>(h->d_err) + 32);  // 8 floats of the handle's 64 B
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) {
        qrs::k_check_selftest<<<1, 1, 0, (cudaStream_t)stream>>>(scratch, i);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_check_selftest launch");
    ++h->launches;
    return QRS_OK;
}

qrs_status qrs_sync(qrs_handle* h, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_sync");
    int word = 0;
    e = cudaMemcpy(&word, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_sync error word");
    if (word != 0) {
        cudaMemset(h->d_err, 0, sizeof(int));
        if (word == QRS_ERR_TIMEOUT) return fail(h, QRS_ERR_TIMEOUT, "a bounded device wait ran out");
        return fail(h, QRS_ERR_DEVICE_CHECK, "a device-side argument check failed (code %d)", word);
    }
    return QRS_OK;
}

qrs_status qrs_draw(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, const qrs_sampler* smp, int64_t n_f,
                    int64_t n_real, int64_t real_offset, const qrs_draw_out* out, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_draw");
    if (qrs::injected_launch_fault(h, "qrs_draw") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (!out) return fail(h, QRS_ERR_ARG, "out must be non-NULL");
    if (n_real < 0) return fail(h, QRS_ERR_ARG, "n_real must be >= 0");
    DrawParams p;
    qrs_status st = make_draw_params(h, psd, dom, smp, n_f, real_offset, &p);
    if (st != QRS_OK) return st;
    if (!counters_fit(n_f, real_offset, n_real)) return fail(h, QRS_ERR_ARG, "stream index overflows 2^64");
    if (((uintptr_t)out->f_xy & 7) || ((uintptr_t)out->coef & 7) || ((uintptr_t)out->words & 15) ||
        ((uintptr_t)out->r2 & 7) || ((uintptr_t)out->amp & 3) || ((uintptr_t)out->cell & 3))
        return fail(h, QRS_ERR_ARG, "misaligned output (f_xy/coef/r2 8 B, words 16 B, amp/cell 4 B)");
    if (n_real == 0) return QRS_OK;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = launch_draw(p, n_real, *out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_draw launch");
    ++h->launches;
    return QRS_OK;
}

qrs_status qrs_synthesize_points(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, const qrs_sampler* smp,
                                 int64_t n_f, int64_t n_real, int64_t real_offset, const float* xy, int64_t n_points,
                                 int32_t mode, const double* col_psd, float* out, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_synthesize_points");
    if (qrs::injected_launch_fault(h, "qrs_synthesize_points") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (n_real < 0 || n_points < 0) return fail(h, QRS_ERR_ARG, "n_real and n_points must be >= 0");
    DrawParams p;
    qrs_status st = make_draw_params(h, psd, dom, smp, n_f, real_offset, &p);
    if (st != QRS_OK) return st;
    if (!counters_fit(n_f, real_offset, n_real)) return fail(h, QRS_ERR_ARG, "stream index overflows 2^64");
    if (n_real == 0 || n_points == 0) return QRS_OK;
    if (!xy || !out) return fail(h, QRS_ERR_ARG, "xy and out must be non-NULL");
    if (((uintptr_t)xy & 7) || ((uintptr_t)out & 3)) return fail(h, QRS_ERR_ARG, "xy must be 8-byte, out 4-byte aligned");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (mode == QRS_SYNTH_FUSED) {
        if (col_psd) return fail(h, QRS_ERR_ARG, "col_psd applies to the shared-draw GEMM modes only");
        e = launch_synth_fused(h, p, xy, n_points, n_real, out, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "qrs_synthesize_points launch");
        ++h->launches;
        return QRS_OK;
    }
    if (mode == QRS_SYNTH_GEMM_3XTF32 || mode == QRS_SYNTH_GEMM_BF16X3 || mode == QRS_SYNTH_GEMM_TF32) {
        if (n_real > 65280) return fail(h, QRS_ERR_ARG, "GEMM modes take at most 65280 realisations per call");
        if (col_psd && ((uintptr_t)col_psd & 7)) return fail(h, QRS_ERR_ARG, "col_psd must be 8-byte aligned");
        st = ensure_work(h, gemm_workspace_bytes(mode, n_f, n_real, h->num_sms));
        if (st != QRS_OK) return st;
        e = launch_synth_gemm(h, mode, p, xy, n_points, n_real, col_psd, vk_constant(), out, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "qrs_synthesize_points GEMM launch");
        h->launches += 4;
        return QRS_OK;
    }
    return fail(h, QRS_ERR_ARG, "unknown synthesis mode %d", mode);
}

qrs_status qrs_synthesize_grid(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, const qrs_sampler* smp,
                               int64_t n_f, int64_t n_real, int64_t real_offset, const float* x, int64_t nx,
                               const float* y, int64_t ny, const int32_t* index, int64_t n_points, int32_t mode,
                               float* out, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_synthesize_grid");
    if (qrs::injected_launch_fault(h, "qrs_synthesize_grid") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (mode != QRS_SYNTH_GEMM_3XTF32 && mode != QRS_SYNTH_GEMM_BF16X3)
        return fail(h, QRS_ERR_ARG, "grid synthesis modes: QRS_SYNTH_GEMM_3XTF32 or QRS_SYNTH_GEMM_BF16X3");
    if (n_real < 0 || nx < 0 || ny < 0 || nx > (1 << 24) || ny > (1 << 24))
        return fail(h, QRS_ERR_ARG, "n_real >= 0 and nx, ny in [0, 2^24]");
    if (index && n_points < 0) return fail(h, QRS_ERR_ARG, "n_points must be >= 0");
    DrawParams p;
    qrs_status st = make_draw_params(h, psd, dom, smp, n_f, real_offset, &p);
    if (st != QRS_OK) return st;
    if (!counters_fit(n_f, real_offset, n_real)) return fail(h, QRS_ERR_ARG, "stream index overflows 2^64");
    if (n_real == 0 || nx == 0 || ny == 0 || (index && n_points == 0)) return QRS_OK;
    if (!x || !y || !out) return fail(h, QRS_ERR_ARG, "x, y and out must be non-NULL");
    if (((uintptr_t)x & 3) || ((uintptr_t)y & 3) || ((uintptr_t)out & 3) || ((uintptr_t)index & 3))
        return fail(h, QRS_ERR_ARG, "x, y, index and out must be 4-byte aligned");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    st = ensure_work(h, grid_workspace_bytes(mode, n_f, n_real, h->num_sms));
    if (st != QRS_OK) return st;
    e = launch_synth_grid(h, mode, p, x, nx, y, ny, index, index ? n_points : nx * ny, n_real, out,
                          (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_synthesize_grid launch");
    h->launches += grid_launch_count(mode, n_f, n_real);
    return QRS_OK;
}

static qrs_status build_piston_job(qrs_handle* h, const qrs_piston_job& j, PistonJobDev* d)
{
    qrs_status st = make_draw_params(h, &j.psd, &j.dom, &j.smp, j.n_f, j.real_offset, &d->p);
    if (st != QRS_OK) return st;
    if (j.psd.ap_D_m > 0.0)
        return fail(h, QRS_ERR_ARG, "piston jobs filter per aperture: the PSD's aperture filter must be off");
    if (j.n_real < 0) return fail(h, QRS_ERR_ARG, "n_real must be >= 0");
    if (!counters_fit(j.n_f, j.real_offset, j.n_real)) return fail(h, QRS_ERR_ARG, "stream index overflows 2^64");
    if (j.n_ap < 1 || j.n_ap > kPisMaxAp) return fail(h, QRS_ERR_ARG, "n_ap must be in [1, %d]", kPisMaxAp);
    if (j.n_pairs < 0) return fail(h, QRS_ERR_ARG, "n_pairs must be >= 0");
    if (!j.ap_xy || !j.ap_D) return fail(h, QRS_ERR_ARG, "ap_xy and ap_D must be non-NULL");
    if (j.n_pairs > 0 && j.delta && !j.pairs) return fail(h, QRS_ERR_ARG, "delta needs pairs");
    if (((uintptr_t)j.ap_xy & 7) || ((uintptr_t)j.pairs & 7) || ((uintptr_t)j.ap_D & 3) || ((uintptr_t)j.ap_d & 3))
        return fail(h, QRS_ERR_ARG, "misaligned aperture arrays (ap_xy, pairs 8 B; ap_D, ap_d 4 B)");
    d->ap_xy = reinterpret_cast<const float2*>(j.ap_xy);
    d->ap_D = j.ap_D;
    d->ap_d = j.ap_d;
    d->pairs = reinterpret_cast<const int2*>(j.pairs);
    d->piston = j.piston;
    d->delta = j.n_pairs > 0 ? j.delta : nullptr;
    d->n_real = j.n_real;
    d->item_begin = 0;
    d->n_ap = j.n_ap;
    d->n_pairs = j.n_pairs;
    return QRS_OK;
}

qrs_status qrs_diff_piston(qrs_handle* h, const qrs_piston_job* jobs, int32_t n_jobs, int32_t flags, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_diff_piston");
    if (qrs::injected_launch_fault(h, "qrs_diff_piston") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(h, QRS_ERR_ARG, "jobs must hold n_jobs >= 0 entries");
    if (flags & ~(QRS_PISTON_PERSISTENT | QRS_PISTON_GRAPH)) return fail(h, QRS_ERR_ARG, "unknown flags 0x%x", flags);
    std::vector<PistonJobDev> dev((size_t)n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        qrs_status st = build_piston_job(h, jobs[i], &dev[(size_t)i]);
        if (st != QRS_OK) return fail(h, st, "job %d: %s", i, h->last_error.c_str());
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (!(flags & (QRS_PISTON_PERSISTENT | QRS_PISTON_GRAPH))) {
        for (const PistonJobDev& J : dev) {
            if (J.n_real == 0) continue;
            e = launch_piston_single(J, h->num_sms, h->d_err, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "piston launch");
            ++h->launches;
        }
        return QRS_OK;
    }
    return run_piston_batch(h, dev, (flags & QRS_PISTON_GRAPH) != 0, s);
}

qrs_status qrs_pair_diff(qrs_handle* h, const float* values, int64_t n_real, int64_t n_points, const int32_t* pairs,
                         int64_t n_pairs, float* out, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_pair_diff");
    if (qrs::injected_launch_fault(h, "qrs_pair_diff") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (n_real < 0 || n_points < 0 || n_pairs < 0) return fail(h, QRS_ERR_ARG, "sizes must be >= 0");
    if (n_real == 0 || n_pairs == 0) return QRS_OK;
    if (!values || !pairs || !out) return fail(h, QRS_ERR_ARG, "values, pairs and out must be non-NULL");
    if (((uintptr_t)values & 3) || ((uintptr_t)pairs & 7) || ((uintptr_t)out & 3))
        return fail(h, QRS_ERR_ARG, "misaligned values/out (4 B) or pairs (8 B)");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess)
        e = launch_pair_diff(values, n_real, n_points, pairs, n_pairs, out, h->num_sms, h->d_err, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_pair_diff launch");
    ++h->launches;
    return QRS_OK;
}

static qrs_status stats_args(qrs_handle* h, const void* pts, int64_t n_sets, int64_t n, const void* out, int out_align)
{
    if (n_sets < 0 || n_sets > 65535 || n < 1 || n > 65536)
        return fail(h, QRS_ERR_ARG, "need 1 <= n <= 65536 and 0 <= n_sets <= 65535");
    if (n_sets > 0 && (!pts || !out)) return fail(h, QRS_ERR_ARG, "pts and out must be non-NULL");
    if (((uintptr_t)pts & 7) || ((uintptr_t)out & (uintptr_t)(out_align - 1)))
        return fail(h, QRS_ERR_ARG, "pts must be 8-byte aligned, out %d-byte", out_align);
    return QRS_OK;
}

qrs_status qrs_nearest_neighbour(qrs_handle* h, const float* pts, int64_t n_sets, int64_t n, float* out, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_nearest_neighbour");
    if (qrs::injected_launch_fault(h, "qrs_nearest_neighbour") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    qrs_status st = stats_args(h, pts, n_sets, n, out, 4);
    if (st != QRS_OK || n_sets == 0) return st;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = launch_nearest_neighbour(pts, n_sets, n, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_nearest_neighbour launch");
    ++h->launches;
    return QRS_OK;
}

qrs_status qrs_star_discrepancy(qrs_handle* h, const float* pts, int64_t n_sets, int64_t n, double* out, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_star_discrepancy");
    if (qrs::injected_launch_fault(h, "qrs_star_discrepancy") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    qrs_status st = stats_args(h, pts, n_sets, n, out, 8);
    if (st != QRS_OK || n_sets == 0) return st;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = launch_star_discrepancy(pts, n_sets, n, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_star_discrepancy launch");
    ++h->launches;
    return QRS_OK;
}

qrs_status qrs_structure_fn(qrs_handle* h, const float* delta, int64_t n_real, int64_t n_series, int64_t T,
                            const int32_t* lags, int32_t n_lags, double* acc, void* stream)
{
    if (!h) return QRS_ERR_ARG;
    qrs::NvtxRange nvtx_range("qrs_structure_fn");
    if (qrs::injected_launch_fault(h, "qrs_structure_fn") != QRS_OK) return QRS_ERR_CUDA;
    h->last_error.clear();
    if (n_real < 0 || n_series < 0 || T < 0 || n_lags < 0) return fail(h, QRS_ERR_ARG, "sizes must be >= 0");
    if (n_real == 0 || n_series == 0 || T == 0 || n_lags == 0) return QRS_OK;
    if (!delta || !lags || !acc) return fail(h, QRS_ERR_ARG, "delta, lags and acc must be non-NULL");
    if (((uintptr_t)delta & 3) || ((uintptr_t)lags & 3) || ((uintptr_t)acc & 7))
        return fail(h, QRS_ERR_ARG, "misaligned delta/lags (4 B) or acc (8 B)");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess)
        e = launch_structure_fn(delta, n_real, n_series, T, lags, n_lags, acc, h->num_sms, h->d_err, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qrs_structure_fn launch");
    ++h->launches;
    return QRS_OK;
}

}  // extern "C"
