// check.cuh -- optional bounds checking of the kernels' shared-memory accesses
// (build with -DCWT_BOUNDS_CHECK; build.py's check variant).
//
// CWT_SMEM(p): p is the address of a dynamic shared-memory element about to
// be read or written.  In a checked build, an address outside the CTA's
// dynamic shared memory (%dynamic_smem_size bytes from its start) is not
// accessed: the first such event of the launch is recorded in a device word
// of the translation unit (source line and byte offset) and the access is
// redirected to the start of the buffer.  CWT_IDX(i, n) does the same for an
// index i that must lie in [0, n) (static arrays, spectrum bins).  The host
// collects the words after every entry point (check_collect) and returns
// CWT_EDEVICE with the site in cwt_plan_last_error.  In an ordinary build
// both macros are the identity and cost nothing.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

#ifdef CWT_BOUNDS_CHECK

namespace cwtk {

// Register a translation unit's reader of its violation word (alloc.cu).
void check_register(cudaError_t (*take)(unsigned long long *), const char *unit);

namespace {

__device__ unsigned long long g_cwt_violation;  // (line << 32) | offset; 0 = none

__device__ __forceinline__ void cwt_record(int line, unsigned value) {
    atomicCAS(&g_cwt_violation, 0ull, ((unsigned long long)(unsigned)line << 32) | value);
}

template <typename T>
__device__ __forceinline__ T *cwt_smem_checked(T *p, int line) {
    extern __shared__ float2 cwt_dyn_smem[];
    unsigned size;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
    const unsigned base = (unsigned)__cvta_generic_to_shared(cwt_dyn_smem);
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    if (a < base || a - base + sizeof(T) > size) {
        cwt_record(line, a - base);
        return reinterpret_cast<T *>(cwt_dyn_smem);
    }
    return p;
}

__device__ __forceinline__ int cwt_idx_checked(int i, int n, int line) {
    if ((unsigned)i >= (unsigned)n) {
        cwt_record(line, (unsigned)i);
        return 0;
    }
    return i;
}

cudaError_t cwt_check_take(unsigned long long *v) {
    cudaError_t e = cudaMemcpyFromSymbol(v, g_cwt_violation, sizeof(*v));
    if (e == cudaSuccess && *v) {
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(g_cwt_violation, &zero, sizeof(zero));
    }
    return e;
}

struct CwtCheckRegistration {
    CwtCheckRegistration() { check_register(cwt_check_take, __BASE_FILE__); }
} g_cwt_check_registration;

}  // namespace
}  // namespace cwtk

#define CWT_SMEM(p) (::cwtk::cwt_smem_checked((p), __LINE__))
#define CWT_IDX(i, n) (::cwtk::cwt_idx_checked((i), (n), __LINE__))

#else

#define CWT_SMEM(p) (p)
#define CWT_IDX(i, n) (i)

#endif
