// alloc.cu -- every device and pinned-host allocation of the library goes
// through dev_alloc / host_alloc, which can be made to fail on purpose so
// that the out-of-memory paths are tested without exhausting a GPU.
//
// Failure injection (host side only): when the environment variable
// CWT_FAULT_ALLOC_AT holds "k" or "k:tag" (k >= 1), the k-th allocation the
// library makes after the variable last changed value returns
// cudaErrorMemoryAllocation without calling CUDA; the entry point that made
// it then frees what it holds and returns CWT_ENOMEM.  Unset or empty: no
// injection.  The variable is read on every allocation (allocations are
// rare: plan creation, first host-buffer call, new batch shapes, stream
// admission).
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace cwtk {

namespace {

std::mutex g_fault_mu;
std::string g_fault_value;
long long g_fault_count = 0;

bool inject_failure() {
    const char *v = std::getenv("CWT_FAULT_ALLOC_AT");
    std::lock_guard<std::mutex> lk(g_fault_mu);
    const std::string cur = v ? v : "";
    if (cur != g_fault_value) {
        g_fault_value = cur;
        g_fault_count = 0;
    }
    if (cur.empty()) return false;
    const long long k = std::atoll(cur.c_str());
    return k >= 1 && ++g_fault_count == k;
}

}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes) {
    if (inject_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t host_alloc(void **p, size_t bytes) {
    if (inject_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

}  // namespace cwtk

// ---- bounds-check builds (check.cuh): the translation units' violation words ----

namespace cwtk {

namespace {

struct CheckUnit {
    cudaError_t (*take)(unsigned long long *);
    const char *unit;
};

std::mutex &check_mu() {
    static std::mutex m;
    return m;
}
std::vector<CheckUnit> &check_units() {
    static std::vector<CheckUnit> v;
    return v;
}

}  // namespace

void check_register(cudaError_t (*take)(unsigned long long *), const char *unit) {
    std::lock_guard<std::mutex> lk(check_mu());
    check_units().push_back({take, unit});
}

bool check_collect(std::string *where) {
    std::lock_guard<std::mutex> lk(check_mu());
    bool hit = false;
    for (const CheckUnit &u : check_units()) {
        unsigned long long v = 0;
        if (u.take(&v) != cudaSuccess || !v) continue;
        if (!hit && where) {
            *where = std::string("bounds check: ") + u.unit + " line " + std::to_string(v >> 32) +
                     ", offset/index " + std::to_string(v & 0xffffffffu);
        }
        hit = true;
    }
    return hit;
}

}  // namespace cwtk
