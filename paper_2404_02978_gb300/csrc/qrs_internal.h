// qrs_internal.h -- handle layout and kernel launchers shared by the libqrs
// translation units (not installed; the public ABI is include/qrs.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>

#include "../../include/qrs.h"
#include "qrs_check.cuh"
#include "qrs_device.cuh"

struct qrs_handle {
    int device = 0;
    int num_sms = 0;
    int smem_optin = 0;
    int64_t launches = 0;
    std::string last_error;
    // Device workspace owned by the handle (allocated once in qrs_create).
    int* d_err = nullptr;          // device error word (0 = fine)
    float* d_xbound = nullptr;     // per-call point bound max(|x|, |y|) of a synthesis, then the anchor bound
    // Growing device workspace for the GEMM form and batched pistons.
    void* d_work = nullptr;
    size_t work_bytes = 0;
    // Pinned host staging for launch descriptors.
    void* h_stage = nullptr;
    size_t stage_bytes = 0;
    // Batched-piston state (persistent launch, CUDA graph cache).
    void* piston_state = nullptr;
    // Host-side fault injection, from QRS_FAULT at qrs_create ("alloc",
    // "launch", "timeout", separated by commas): workspace allocations and
    // launches then fail with their error status without touching the GPU;
    // "timeout" makes the next GEMM-form launch wait out a bounded wait on a
    // barrier that nothing arrives at (QRS_ERR_TIMEOUT at the next qrs_sync).
    int fault = 0;
    // Grid form: CTA pairs (k_grid_pair) allowed (QRS_GRID_PAIR=0 at
    // qrs_create switches them off), and the clusters of two the GPU holds
    // per precision (0: not yet queried, -1: unavailable).
    int grid_pair = 1;
    int grid_pair_clusters[2] = {0, 0};
    // Shared-draw GEMM form: the same for k_gemm_pair (QRS_GEMM_PAIR=0 at
    // qrs_create), per mode (3XTF32, BF16X3, TF32).
    int gemm_pair = 1;
    int gemm_pair_clusters[3] = {0, 0, 0};
    // Fused form: the anchored phase path allowed where the point groups
    // permit it (QRS_SYNTH_ANCHOR=0 at qrs_create keeps the exact paths).
    int synth_anchor = 1;
};

namespace qrs {

constexpr int kFaultAlloc = 1;
constexpr int kFaultLaunch = 2;
constexpr int kFaultTimeout = 4;  // the next tensor-core GEMM launch runs out a bounded wait (one-shot)

// An NVTX range over a C-ABI call (seen by profilers, free otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Error plumbing: set message, return status.
qrs_status fail(qrs_handle* h, qrs_status st, const char* fmt, ...);
qrs_status cuda_fail(qrs_handle* h, cudaError_t e, const char* where);
qrs_status ensure_work(qrs_handle* h, size_t bytes);
// QRS_ERR_CUDA with a message when launch-fault injection is on, else QRS_OK.
qrs_status injected_launch_fault(qrs_handle* h, const char* where);

// Host-side construction of the draw parameters from the public structs.
qrs_status make_draw_params(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, const qrs_sampler* smp,
                            int64_t n_f, int64_t real_offset, DrawParams* out);

// True when every stream index (real_offset + r) n_f + k of a call stays below
// 2^64 (all three arguments non-negative).
bool counters_fit(int64_t n_f, int64_t real_offset, int64_t n_real);

// Largest |f| component a draw can produce (for fixed-point scaling).
double freq_bound(const DrawParams& p);

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_draw(const DrawParams& p, int64_t n_real, const qrs_draw_out& o, cudaStream_t s);
cudaError_t launch_point_bound(const float* xy, int64_t n_points, float* d_bound, cudaStream_t s);
cudaError_t launch_synth_fused(qrs_handle* h, const DrawParams& p, const float* xy, int64_t n_points,
                               int64_t n_real, float* out, cudaStream_t s);
cudaError_t launch_pair_diff(const float* v, int64_t n_real, int64_t n_points, const int32_t* pairs, int64_t n_pairs,
                             float* out, int num_sms, int* err, cudaStream_t s);
cudaError_t launch_nearest_neighbour(const float* pts, int64_t n_sets, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_star_discrepancy(const float* pts, int64_t n_sets, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_structure_fn(const float* delta, int64_t n_real, int64_t n_series, int64_t T,
                                const int32_t* lags, int32_t n_lags, double* acc, int num_sms, int* err,
                                cudaStream_t s);

// Bounds-checked build: one hook per translation unit with kernels (each
// points that unit's check word at `err`; no-ops in the default build).
cudaError_t check_hook_draw(int* err);
cudaError_t check_hook_fft(int* err);
cudaError_t check_hook_gemm(int* err);
cudaError_t check_hook_grid(int* err);
cudaError_t check_hook_piston(int* err);
cudaError_t check_hook_proposal(int* err);
cudaError_t check_hook_sf(int* err);
cudaError_t check_hook_stats(int* err);
cudaError_t check_hook_synth(int* err);
cudaError_t check_hook_api(int* err);

struct PistonJobDev;
void destroy_piston_state(qrs_handle* h);

size_t gemm_workspace_bytes(int mode, int64_t n_f, int64_t n_real, int num_sms);
cudaError_t launch_synth_gemm(qrs_handle* h, int mode, const DrawParams& p, const float* xy, int64_t P,
                              int64_t n_real, const double* col_psd, double c_vk, float* out, cudaStream_t s);

size_t grid_workspace_bytes(int mode, int64_t n_f, int64_t n_real, int num_sms);
int64_t grid_launch_count(int mode, int64_t n_f, int64_t n_real);
cudaError_t launch_synth_grid(qrs_handle* h, int mode, const DrawParams& p, const float* x, int64_t nx,
                              const float* y, int64_t ny, const int32_t* index, int64_t P, int64_t n_real, float* out,
                              cudaStream_t s);

}  // namespace qrs
