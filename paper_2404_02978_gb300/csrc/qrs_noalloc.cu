// qrs_noalloc.cu -- qrs_synthesize_points_noalloc: the fused synthesis for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a framework which
// owns every byte of device memory through its own pool allocator, or a
// latency-bound loop in which an allocation could block or synchronise the
// device.  Creating a qrs_handle allocates its workspace, so those callers
// use this entry point instead: it takes no handle, allocates nothing, and
// keeps its only scratch -- the two-float point and anchor bounds that pick
// the phase path of the fused kernel -- in the file-scope device array below, which
// every GPU that loads the library holds until the process exits.
#include <cuda.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "qrs_internal.h"

namespace qrs {
cudaError_t launch_synth_fused_raw(int num_sms, float* d_bound, const DrawParams& p, const float* xy,
                                   int64_t n_points, int64_t n_real, float* out, int allow_anchor, cudaStream_t s);
}

namespace {

constexpr int kNoAllocScratchBytes = 256;  // QRS_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
bool g_noalloc_ready[kNoAllocMaxDevices];
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices];  // id of the context the address belongs to
float* g_noalloc_bound[kNoAllocMaxDevices];  // device address of the scratch, per device
int g_noalloc_sms[kNoAllocMaxDevices];

// Driver entry points, taken through the runtime (the library does not link
// the driver library, so it still loads on a machine without one).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the calling thread's current context (0 if there is none);
// called with g_noalloc_mu held.
unsigned long long current_context_id()
{
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = q0;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return 0;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// With device `dev` current: resolve the device address of the scratch array
// (its name in host code is only a host-side stand-in).  Done on the first
// call on each device, and again after the device's context has been
// replaced (cudaDeviceReset reloads the module, so the old address is stale);
// context ids are unique for the life of the process, so a replaced context
// is never mistaken for the old one.
qrs_status noalloc_setup(int dev)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long id = current_context_id();
    if (g_noalloc_ready[dev] && id != 0 && id == g_noalloc_ctx[dev]) return QRS_OK;
    void* addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);  // makes the primary context current
    if (e != cudaSuccess || addr == nullptr) return QRS_ERR_CUDA;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1) return QRS_ERR_CUDA;
    const unsigned long long now = current_context_id();
    if (now == 0) return QRS_ERR_CUDA;
    g_noalloc_bound[dev] = static_cast<float*>(addr);
    g_noalloc_sms[dev] = sms;
    g_noalloc_ctx[dev] = now;
    g_noalloc_ready[dev] = true;
    return QRS_OK;
}

}  // namespace

extern "C" qrs_status qrs_synthesize_points_noalloc(const qrs_psd* psd, const qrs_domain* dom,
                                                    const qrs_sampler* smp, int64_t n_f, int64_t n_real,
                                                    int64_t real_offset, const float* xy, int64_t n_points,
                                                    float* out, void* stream)
{
    using namespace qrs;
    if (n_real < 0 || n_points < 0) return QRS_ERR_ARG;
    DrawParams p;
    qrs_status st = make_draw_params(nullptr, psd, dom, smp, n_f, real_offset, &p);  // no message: no handle
    if (st != QRS_OK) return st;
    if (!counters_fit(n_f, real_offset, n_real)) return QRS_ERR_ARG;  // the limits of qrs_synthesize_points
    if (n_real == 0 || n_points == 0) return QRS_OK;
    if (!xy || !out || ((uintptr_t)xy & 7) || ((uintptr_t)out & 3)) return QRS_ERR_ARG;
    // the fused path needs two floats of scratch, whatever the problem size
    static_assert(2 * sizeof(float) <= kNoAllocScratchBytes, "scratch holds the point and anchor bounds");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return QRS_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return QRS_ERR_UNSUPPORTED;
    st = noalloc_setup(dev);
    if (st != QRS_OK) return st;
    // the phase path follows the same QRS_SYNTH_ANCHOR switch as a handle, so the outputs stay identical
    const char* anchor_env = std::getenv("QRS_SYNTH_ANCHOR");
    const int allow_anchor = (anchor_env && std::strcmp(anchor_env, "0") == 0) ? 0 : 1;
    cudaError_t e = launch_synth_fused_raw(g_noalloc_sms[dev], g_noalloc_bound[dev], p, xy, n_points, n_real, out,
                                           allow_anchor, (cudaStream_t)stream);
    return e == cudaSuccess ? QRS_OK : QRS_ERR_CUDA;
}
