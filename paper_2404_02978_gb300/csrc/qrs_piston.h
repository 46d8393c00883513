// qrs_piston.h -- device-side job descriptor of the piston kernels.
#pragma once

#include <vector>

#include "qrs_internal.h"

namespace qrs {

constexpr int kPisMaxAp = 64;  // apertures per job

struct PistonJobDev {
    DrawParams p;
    const float2* ap_xy;
    const float* ap_D;
    const float* ap_d;     // may be NULL (no obstruction)
    const int2* pairs;
    float* piston;         // [n_real][n_ap] or NULL
    float* delta;          // [n_real][n_pairs] or NULL
    int64_t n_real;
    int64_t item_begin;    // first global item of this job (batched launch)
    int32_t n_ap;
    int32_t n_pairs;
};

size_t piston_smem_bytes();
cudaError_t launch_piston_single(const PistonJobDev& J, int num_sms, int* err, cudaStream_t s);
qrs_status run_piston_batch(qrs_handle* h, std::vector<PistonJobDev>& jobs, bool graph, cudaStream_t s);
int piston_shape_count();
const char* piston_shape_name(int shape);
cudaError_t launch_piston_persistent(int shape, const PistonJobDev* d_jobs, int n_jobs, int64_t n_items,
                                     unsigned long long* d_counter, int num_sms, int* err, cudaStream_t s);

}  // namespace qrs
