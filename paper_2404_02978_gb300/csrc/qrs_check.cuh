// qrs_check.cuh -- the bounds-checked build of libqrs (QRS_CHECKED=1, built
// as libqrs_checked.so beside the library).
//
// Accesses written as chk(base, i, n) are tested against the extent n of
// their buffer in that build: an index outside [0, n) is not used -- the
// access goes to a 256-byte sink of the translation unit instead -- and
// QRS_ERR_DEVICE_CHECK is recorded in the device error word of the handle
// created last, which qrs_sync reports and clears.  chk_ok(i, n) is the same
// test for accesses made in inline PTX (bulk copies, shared-memory offsets
// of the tensor-core tiles): false means "skip it", with the error recorded.
// In the default build chk(base, i, n) is base + i and chk_ok is true, so
// the checks cost nothing there.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qrs.h"

#ifndef QRS_CHECKED
#define QRS_CHECKED 0
#endif

namespace qrs {

#if QRS_CHECKED
static __constant__ int* g_check_err = nullptr;               // this translation unit's copy
static __device__ __align__(16) unsigned char g_check_sink[256];  // out-of-range accesses land here

static __device__ __noinline__ void check_failed()
{
    int* e = g_check_err;
    if (e) atomicExch(e, (int)QRS_ERR_DEVICE_CHECK);
}
#endif

template <class T>
__device__ __forceinline__ T* chk(T* base, int64_t i, int64_t n)
{
#if QRS_CHECKED
    if (i < 0 || i >= n) {
        check_failed();
        return reinterpret_cast<T*>(g_check_sink);
    }
#endif
    return base + i;
}

// [i, i + len) inside [0, n)?
__device__ __forceinline__ bool chk_ok(int64_t i, int64_t len, int64_t n)
{
#if QRS_CHECKED
    if (i < 0 || len < 0 || i + len > n) {
        check_failed();
        return false;
    }
#endif
    (void)i;
    (void)len;
    (void)n;
    return true;
}

// Checked element of a fixed-size array (its own extent), e.g. shared tables.
template <class T, size_t N>
__device__ __forceinline__ T& el(T (&a)[N], int64_t i)
{
    return *chk(a, i, (int64_t)N);
}

template <class T, size_t R, size_t C>
__device__ __forceinline__ T& el(T (&a)[R][C], int64_t i, int64_t j)
{
#if QRS_CHECKED
    if (j < 0 || j >= (int64_t)C) {
        check_failed();
        return *reinterpret_cast<T*>(g_check_sink);
    }
#endif
    return *chk(&a[0][0], i * (int64_t)C + j, (int64_t)(R * C));
}

constexpr bool kChecked = QRS_CHECKED != 0;

}  // namespace qrs

// Each translation unit with kernels defines one hook (host) that points its
// copy of the error-word pointer at a handle's error word; qrs_create calls
// them all in the checked build.
#if QRS_CHECKED
#define QRS_CHECK_HOOK(name)                                                       \
    cudaError_t name(int* err) { return cudaMemcpyToSymbol(qrs::g_check_err, &err, sizeof(err)); }
#else
#define QRS_CHECK_HOOK(name) \
    cudaError_t name(int*) { return cudaSuccess; }
#endif
