// jit.cu -- plan-time specialization of the smooth-length kernels (Section
// "Fast Fourier transform": the paper pads to 2,3,5,7-smooth lengths).
//
// The fixed-length kernels of smooth_device.cuh run a radix schedule whose
// every stride, butterfly count and divisor is a compile-time constant; the
// library ships them for 27 whole-second EEG lengths (CWT_MR_FIXED) and three
// cluster local lengths (CWT_CL_MR_FIXED), and every other smooth length runs
// the runtime-schedule kernels.  A plan created with cwt_options.specialize =
// 1 gets the fixed form for its own length instead: NVRTC compiles
// smooth_device.cuh, or smooth_cluster_device.cuh for a row on a cluster of
// CL CTAs (their text is embedded in the library at build time,
// jit_headers.cpp), for the scheduler's schedule of N (of N / CL) into a
// cubin for the device's architecture, the driver loads it, and the plan
// launches those kernels.  Modules are cached per (device, schedule) for the
// life of the process; a failed compile or load leaves the plan on the
// runtime-schedule kernels (cwt_plan_info.specialized reports which ran).
//
// Rows per CTA are the runtime-schedule kernels' choice for the plan's row
// count (up to 256 threads, at least two CTAs per SM when rows are few);
// CTAs per SM as many as shared memory, 2048 threads and 64 registers a
// thread allow, at most 4 (the rules the shipped fixed kernels were measured
// with).
#include <cuda.h>
#include <nvrtc.h>
#include <unistd.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "smooth_cluster.cuh"

// The headers the plan-time compiler needs, embedded by build.py.
extern "C" const int cwt_jit_header_count;
extern "C" const char *const cwt_jit_header_names[];
extern "C" const char *const cwt_jit_header_texts[];

namespace cwtk {

struct JitKernels {
    CUmodule mod = nullptr;
    CUfunction sb = nullptr, fwd = nullptr;
    int rows = 1, threads = 32, smem = 0;
    int cl = 1;  // CTAs per row: 1, or the cluster of the cluster kernels
};

namespace {

// The driver calls, fetched through the runtime (the library links no driver
// library, so that it loads on a machine without one).
struct Driver {
    CUresult (*module_load_data)(CUmodule *, const void *) = nullptr;
    CUresult (*module_get_function)(CUfunction *, CUmodule, const char *) = nullptr;
    CUresult (*module_unload)(CUmodule) = nullptr;
    CUresult (*func_set_attribute)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*launch_kernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                              CUstream, void **, void **) = nullptr;
    bool ok = false;
};

template <typename F>
bool entry(const char *name, F *fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    *fn = reinterpret_cast<F>(p);
    return true;
}

const Driver &driver() {
    static const Driver d = [] {
        Driver x;
        x.ok = entry("cuModuleLoadData", &x.module_load_data) &&
               entry("cuModuleGetFunction", &x.module_get_function) && entry("cuModuleUnload", &x.module_unload) &&
               entry("cuFuncSetAttribute", &x.func_set_attribute) && entry("cuLaunchKernel", &x.launch_kernel);
        return x;
    }();
    return d;
}

struct JitBinary {
    std::vector<char> cubin;
    std::string sb_name, fwd_name;  // the kernels' lowered names
};

std::mutex g_jit_mu;
std::map<std::string, JitBinary> g_cubins;     // (arch, schedule) -> compiled module
std::map<std::string, JitKernels *> g_modules;  // (device, schedule) -> loaded kernels

struct JitShape {
    int rows, minb, threads, smem;
};

JitShape jit_shape(const MrSchedule &s, int rows) {
    JitShape j;
    const int row_smem = (s.N + (s.N >> 4)) * 8;
    j.rows = rows;
    j.threads = (j.rows * s.T + 31) / 32 * 32;
    j.smem = j.rows * row_smem;
    const int by_smem = (227 * 1024) / (j.smem + 1024);
    const int by_threads = 2048 / j.threads;
    const int by_regs = 65536 / (j.threads * 64);
    j.minb = by_smem < by_threads ? by_smem : by_threads;
    if (by_regs < j.minb) j.minb = by_regs;
    if (j.minb > 4) j.minb = 4;
    if (j.minb < 1) j.minb = 1;
    return j;
}

// MrFixed<N, T, ROWS, MINB, R0, R1, ...> for schedule s (the local row of a
// cluster kernel when cl > 1).
std::string fixed_type(const MrSchedule &s, const JitShape &j) {
    std::string t = "cwtk::MrFixed<" + std::to_string(s.N) + ", " + std::to_string(s.T) + ", " +
                    std::to_string(j.rows) + ", " + std::to_string(j.minb);
    for (int q = 0; q < s.np; ++q) t += ", " + std::to_string(s.p[q].R);
    return t + ">";
}

// Compile the two kernels of schedule s for `arch` (e.g. "sm_103a"); on
// failure *log holds the compiler's message.
bool compile(const MrSchedule &s, int rows, int cl, const std::string &arch, std::vector<char> *cubin,
             std::string *sb_name, std::string *fwd_name, std::string *log) {
    const JitShape j = jit_shape(s, rows);
    const std::string fx = fixed_type(s, j);
    const std::string cls = std::to_string(cl);
    const std::string sb_expr = cl > 1 ? "&cwtk::cl_mr::scale_block_kernel<" + cls + ", " + fx + ">"
                                       : "&cwtk::mr_fixed_scale_block_kernel<" + fx + ">";
    const std::string fwd_expr = cl > 1 ? "&cwtk::cl_mr::forward_kernel<" + cls + ", " + fx + ">"
                                        : "&cwtk::mr_fixed_forward_kernel<" + fx + ">";
    const char *src = cl > 1 ? "#include \"smooth_cluster_device.cuh\"\n" : "#include \"smooth_device.cuh\"\n";
    nvrtcProgram prog = nullptr;
    if (nvrtcCreateProgram(&prog, src, "cwt_specialized.cu", cwt_jit_header_count, cwt_jit_header_texts,
                           cwt_jit_header_names) != NVRTC_SUCCESS) {
        *log = "nvrtcCreateProgram failed";
        return false;
    }
    nvrtcAddNameExpression(prog, sb_expr.c_str());
    nvrtcAddNameExpression(prog, fwd_expr.c_str());
    const std::string arch_opt = "--gpu-architecture=" + arch;
    // -default-device: the kernels' lambdas (no execution-space annotation) are device code
    const char *opts[] = {arch_opt.c_str(), "-std=c++17", "-lineinfo", "-default-device"};
    const nvrtcResult r = nvrtcCompileProgram(prog, 4, opts);
    size_t log_size = 0;
    nvrtcGetProgramLogSize(prog, &log_size);
    std::string lg(log_size, '\0');
    if (log_size) nvrtcGetProgramLog(prog, &lg[0]);
    bool ok = r == NVRTC_SUCCESS;
    if (ok) {
        const char *lowered = nullptr;
        ok = nvrtcGetLoweredName(prog, sb_expr.c_str(), &lowered) == NVRTC_SUCCESS && lowered;
        if (ok) *sb_name = lowered;
        ok = ok && nvrtcGetLoweredName(prog, fwd_expr.c_str(), &lowered) == NVRTC_SUCCESS && lowered;
        if (ok) *fwd_name = lowered;
        size_t n = 0;
        ok = ok && nvrtcGetCUBINSize(prog, &n) == NVRTC_SUCCESS && n > 0;
        if (ok) {
            cubin->resize(n);
            ok = nvrtcGetCUBIN(prog, cubin->data()) == NVRTC_SUCCESS;
        }
    }
    if (!ok) *log = std::string("plan-time compile of ") + fx + " failed: " + nvrtcGetErrorString(r) + "\n" + lg;
    nvrtcDestroyProgram(&prog);
    return ok;
}

std::string schedule_key(const MrSchedule &s, int rows, int cl) {
    std::string k = std::to_string(s.N) + "/" + std::to_string(s.T) + "/" + std::to_string(rows) + "/" +
                    std::to_string(cl);
    for (int q = 0; q < s.np; ++q) k += "x" + std::to_string(s.p[q].R);
    return k;
}

}  // namespace

namespace {

// The compiled module of (s, rows, cl) for arch in g_cubins, compiling it
// (without holding the lock, so that several compile at once) when absent.
// ---- the on-disk cache (CWT_JIT_CACHE_DIR) ------------------------------------
// With CWT_JIT_CACHE_DIR naming a writable directory, every compiled module is
// also kept there, one file per (architecture, schedule, rows, cluster,
// embedded source, NVRTC version), and a later process loads it instead of
// compiling.  A file holds a magic line, the full key (checked on load, so a
// hash collision or a truncated file reads as a miss), the two lowered kernel
// names, the cubin's size and the cubin; it is written to a temporary name and
// renamed into place, so readers never see half a file.

uint64_t fnv1a(const char *p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) h = (h ^ (unsigned char)p[i]) * 1099511628211ull;
    return h;
}

// The embedded headers' digest and the compiler's version: a rebuilt library
// or another toolkit never reads an older file.
const std::string &source_tag() {
    static const std::string tag = [] {
        uint64_t h = fnv1a("", 0);
        for (int i = 0; i < cwt_jit_header_count; ++i) {
            h = fnv1a(cwt_jit_header_names[i], std::strlen(cwt_jit_header_names[i]), h);
            h = fnv1a(cwt_jit_header_texts[i], std::strlen(cwt_jit_header_texts[i]), h);
        }
        int major = 0, minor = 0;
        nvrtcVersion(&major, &minor);
        char b[64];
        std::snprintf(b, sizeof b, "%016llx/nvrtc%d.%d", (unsigned long long)h, major, minor);
        return std::string(b);
    }();
    return tag;
}

std::string cache_path(const std::string &key) {
    const char *dir = std::getenv("CWT_JIT_CACHE_DIR");
    if (!dir || !*dir) return std::string();
    char name[40];
    std::snprintf(name, sizeof name, "/cwt_jit_%016llx.bin", (unsigned long long)fnv1a(key.data(), key.size()));
    return std::string(dir) + name;
}

constexpr const char *kCacheMagic = "cwt-jit-module 1";

bool cache_load(const std::string &key, JitBinary *b) {
    const std::string path = cache_path(key);
    if (path.empty()) return false;
    std::FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return false;
    std::string data;
    char buf[1 << 16];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) data.append(buf, n);
    std::fclose(f);
    // magic \n key \n sb_name \n fwd_name \n size \n cubin
    size_t pos = 0;
    std::string fields[5];
    for (std::string &fl : fields) {
        const size_t e = data.find('\n', pos);
        if (e == std::string::npos) return false;
        fl = data.substr(pos, e - pos);
        pos = e + 1;
    }
    if (fields[0] != kCacheMagic || fields[1] != key || fields[2].empty() || fields[3].empty()) return false;
    char *end = nullptr;
    const unsigned long long size = std::strtoull(fields[4].c_str(), &end, 10);
    if (!end || *end || size == 0 || size != data.size() - pos) return false;
    b->sb_name = fields[2];
    b->fwd_name = fields[3];
    b->cubin.assign(data.begin() + (std::ptrdiff_t)pos, data.end());
    return true;
}

void cache_store(const std::string &key, const JitBinary &b) {
    const std::string path = cache_path(key);
    if (path.empty()) return;
    const std::string tmp = path + ".tmp" + std::to_string((long long)getpid()) + "." +
                            std::to_string((unsigned long long)std::hash<std::thread::id>()(std::this_thread::get_id()));
    std::FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;  // an unwritable cache is no error: the module stays in memory
    const std::string head = std::string(kCacheMagic) + "\n" + key + "\n" + b.sb_name + "\n" + b.fwd_name + "\n" +
                             std::to_string(b.cubin.size()) + "\n";
    const bool ok = std::fwrite(head.data(), 1, head.size(), f) == head.size() &&
                    std::fwrite(b.cubin.data(), 1, b.cubin.size(), f) == b.cubin.size();
    if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
}

// The module of (s, rows, cl) for arch: from the cache on disk, else compiled
// (and stored there).
bool load_or_compile(const MrSchedule &s, int rows, int cl, const std::string &arch, JitBinary *b,
                     std::string *log) {
    const std::string disk_key = arch + ":" + schedule_key(s, rows, cl) + ":" + source_tag();
    if (cache_load(disk_key, b)) return true;
    if (!compile(s, rows, cl, arch, &b->cubin, &b->sb_name, &b->fwd_name, log)) return false;
    cache_store(disk_key, *b);
    return true;
}

bool jit_binary(const MrSchedule &s, int rows, int cl, const std::string &arch, std::string *log) {
    const std::string key = arch + ":" + schedule_key(s, rows, cl);
    {
        std::lock_guard<std::mutex> lock(g_jit_mu);
        if (g_cubins.count(key)) return true;
    }
    JitBinary b;
    if (!load_or_compile(s, rows, cl, arch, &b, log)) return false;
    std::lock_guard<std::mutex> lock(g_jit_mu);
    g_cubins.emplace(key, std::move(b));
    return true;
}

}  // namespace

bool jit_compile_check(const MrSchedule &s, int rows, int cl, std::string *log) {
    JitBinary b;
    return load_or_compile(s, rows, cl, "sm_103a", &b, log);
}

JitKernels *jit_kernels(const MrSchedule &s, int rows, int cl, int device, std::string *log) {
#ifdef CWT_BOUNDS_CHECK
    // the bounds-checked build runs the runtime-schedule kernels, whose checks it collects
    (void)s;
    (void)rows;
    (void)cl;
    (void)device;
    *log = "plan-time specialization is off in the bounds-checked build";
    return nullptr;
#else
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) {
        *log = "compute capability query failed";
        return nullptr;
    }
    const std::string arch = "sm_" + std::to_string(major * 10 + minor) + "a";
    const std::string skey = schedule_key(s, rows, cl);
    const std::string mkey = std::to_string(device) + ":" + skey;
    {
        std::lock_guard<std::mutex> lock(g_jit_mu);
        auto it = g_modules.find(mkey);
        if (it != g_modules.end()) return it->second;
    }
    if (!jit_binary(s, rows, cl, arch, log)) return nullptr;
    std::lock_guard<std::mutex> lock(g_jit_mu);
    auto it = g_modules.find(mkey);
    if (it != g_modules.end()) return it->second;
    const JitBinary &b = g_cubins.find(arch + ":" + skey)->second;
    // the runtime API has made the device's primary context current
    const Driver &drv = driver();
    if (!drv.ok) {
        *log = "the driver's module calls are not available";
        return nullptr;
    }
    JitKernels *k = new (std::nothrow) JitKernels();
    if (!k) return nullptr;
    const JitShape j = jit_shape(s, rows);
    k->rows = j.rows;
    k->threads = j.threads;
    k->smem = j.smem;
    k->cl = cl;
    CUresult r = drv.module_load_data(&k->mod, b.cubin.data());
    if (r == CUDA_SUCCESS) r = drv.module_get_function(&k->sb, k->mod, b.sb_name.c_str());
    if (r == CUDA_SUCCESS) r = drv.module_get_function(&k->fwd, k->mod, b.fwd_name.c_str());
    if (r == CUDA_SUCCESS) r = drv.func_set_attribute(k->sb, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, k->smem);
    if (r == CUDA_SUCCESS) r = drv.func_set_attribute(k->fwd, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, k->smem);
    if (r == CUDA_SUCCESS && cl > 8)  // clusters above the portable 8 CTAs
        r = drv.func_set_attribute(k->sb, CU_FUNC_ATTRIBUTE_NON_PORTABLE_CLUSTER_SIZE_ALLOWED, 1);
    if (r == CUDA_SUCCESS && cl > 8)
        r = drv.func_set_attribute(k->fwd, CU_FUNC_ATTRIBUTE_NON_PORTABLE_CLUSTER_SIZE_ALLOWED, 1);
    if (r != CUDA_SUCCESS) {
        *log = "loading the specialized kernels failed: driver error " + std::to_string((int)r);
        if (k->mod) drv.module_unload(k->mod);
        delete k;
        return nullptr;
    }
    g_modules[mkey] = k;
    return k;
#endif
}

namespace {

cudaError_t sb_launch_k(const JitKernels *k, const MrArgs &a, cudaStream_t st) {
    MrArgs args = a;
    void *params[] = {&args};
    const unsigned grid = (unsigned)((a.total_rows + k->rows - 1) / k->rows);
    const CUresult r = driver().launch_kernel(k->sb, grid, 1, 1, (unsigned)k->threads, 1, 1, (unsigned)k->smem,
                                              (CUstream)st, params, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

}  // namespace

cudaError_t jit_sb_launch(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st) {
    return sb_launch_k(p->jit, a, st);
}

cudaError_t jit_fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    const JitKernels *k = p->jit;
    const void *x = signal;
    int f64 = p->io == CWT_DTYPE_F64, n = p->n, C = p->C;
    float2 *spec = p->spec;
    const float2 *twN = p->twN, *twL = p->twL;
    MrSchedule sch = p->sch;
    CUresult r;
    if (k->cl > 1) {  // forward_kernel<CL, FX>(x, f64, n, spec, twL, twN, sch), C rows of CL CTAs
        void *params[] = {&x, &f64, &n, &spec, &twL, &twN, &sch};
        r = driver().launch_kernel(k->fwd, (unsigned)(C * k->cl), 1, 1, (unsigned)k->threads, 1, 1,
                                   (unsigned)k->smem, (CUstream)st, params, nullptr);
    } else {  // mr_fixed_forward_kernel<FX>(x, f64, n, spec, twN, C)
        void *params[] = {&x, &f64, &n, &spec, &twN, &C};
        const unsigned grid = (unsigned)((C + k->rows - 1) / k->rows);
        r = driver().launch_kernel(k->fwd, grid, 1, 1, (unsigned)k->threads, 1, 1, (unsigned)k->smem,
                                   (CUstream)st, params, nullptr);
    }
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

// scale_block_kernel<CL, FX>(ClMrArgs, MrSchedule): rows of CL CTAs each.
cudaError_t jit_cl_sb_launch(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st) {
    const JitKernels *k = p->jit;
    ClMrArgs args = a;
    MrSchedule sch = p->sch;
    void *params[] = {&args, &sch};
    const unsigned grid = (unsigned)(p->C * p->S * k->cl);
    const CUresult r = driver().launch_kernel(k->sb, grid, 1, 1, (unsigned)k->threads, 1, 1, (unsigned)k->smem,
                                              (CUstream)st, params, nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

JitKernels *jit_tune(cwt_plan_s *p, cudaStream_t st, std::string *log) {
#ifdef CWT_BOUNDS_CHECK
    (void)p;
    (void)st;
    *log = "plan-time specialization is off in the bounds-checked build";
    return nullptr;
#else
    // one-CTA rows: candidates of N; cluster rows: candidates of the local length NL
    const int cl = p->cl;
    const int NL = p->N / cl;
    constexpr int kMaxCandidates = 8;
    MrSchedule cand[kMaxCandidates];
    const int n = mr_schedule_candidates(NL, cand, kMaxCandidates);
    if (n < 1) {
        *log = "no schedule to tune";
        return nullptr;
    }
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, p->device) != cudaSuccess) {
        *log = "compute capability query failed";
        return nullptr;
    }
    const std::string arch = "sm_" + std::to_string(major * 10 + minor) + "a";
    const int total = p->C * p->S;
    int rows[kMaxCandidates];
    for (int i = 0; i < n; ++i) rows[i] = cl == 1 ? mr_launch_rows(cand[i], total) : 1;
    // compile the candidates at once (NVRTC is thread-safe), then load them
    {
        std::vector<std::thread> pool;
        std::vector<std::string> logs((size_t)n);
        for (int i = 0; i < n; ++i)
            pool.emplace_back([&, i] { jit_binary(cand[i], rows[i], cl, arch, &logs[(size_t)i]); });
        for (auto &t : pool) t.join();
    }
    JitKernels *k[kMaxCandidates] = {};
    for (int i = 0; i < n; ++i) {
        std::string lg;
        k[i] = jit_kernels(cand[i], rows[i], cl, p->device, &lg);
        if (!k[i] && log->empty()) *log = lg;
    }
    // time each on the plan's own rows (all of them, or as many as 256 MB of
    // scratch outputs hold)
    const size_t esz = p->io == CWT_DTYPE_F64 ? 8 : 4;
    const size_t row_bytes = (size_t)p->n_out * esz *
                             (((p->outputs & CWT_OUT_COMPLEX) ? 2 : 0) + ((p->outputs & CWT_OUT_POWER) ? 1 : 0) +
                              ((p->outputs & CWT_OUT_PHASE) ? 1 : 0));
    const size_t cap = row_bytes ? ((size_t)256 << 20) / row_bytes : (size_t)total;
    const int trows = (int)std::max<size_t>(1, std::min<size_t>((size_t)total, cap));
    const size_t cells = (size_t)trows * (size_t)p->n_out;
    void *oc = nullptr, *op = nullptr, *oph = nullptr;
    cudaError_t e = cudaSuccess;
    if (p->outputs & CWT_OUT_COMPLEX) e = dmalloc(&oc, cells * 2 * esz);
    if (e == cudaSuccess && (p->outputs & CWT_OUT_POWER)) e = dmalloc(&op, cells * esz);
    if (e == cudaSuccess && (p->outputs & CWT_OUT_PHASE)) e = dmalloc(&oph, cells * esz);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->spec, 0, sizeof(float2) * (size_t)p->C * p->N, st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    MrArgs a;  // one-CTA rows
    a.spec = p->spec;
    a.bank = p->bank;
    a.band = p->band;
    a.twN = p->twN;
    a.out_c = oc;
    a.out_p = op;
    a.out_ph = oph;
    a.S = p->S;
    a.n_out = p->n_out;
    a.sub = p->d;
    a.total_rows = trows;
    a.f64 = p->io == CWT_DTYPE_F64;
    ClMrArgs ca;  // cluster rows: the first trows rows (the grid is trows clusters)
    ca.spec = p->spec;
    ca.bank = p->bank;
    ca.band = p->band;
    ca.twL = p->twL;
    ca.twN = p->twN;
    ca.out_c = oc;
    ca.out_p = op;
    ca.out_ph = oph;
    ca.S = p->S;
    ca.n_out = p->n_out;
    ca.sub = p->d;
    ca.f64 = p->io == CWT_DTYPE_F64;
    const bool compiled_in = cl == 1 ? p->sch.fixed >= 0 : p->sch.fixed_cl >= 0;
    auto launch = [&](int i) -> cudaError_t {
        if (cl == 1) return i >= 0 ? sb_launch_k(k[i], a, st) : mr_fixed_sb_launch(p, a, st);
        const JitKernels *kk = i >= 0 ? k[i] : nullptr;
        if (!kk) return cl_mr_fixed_sb(p, ca, st, trows);
        ClMrArgs args = ca;
        MrSchedule sch = cand[i];
        void *params[] = {&args, &sch};
        const CUresult r = driver().launch_kernel(kk->sb, (unsigned)(trows * cl), 1, 1, (unsigned)kk->threads, 1,
                                                  1, (unsigned)kk->smem, (CUstream)st, params, nullptr);
        return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
    };
    // candidate -1: the length's compiled-in kernel, when it has one
    int best = -2;
    float best_ms = 0.f;
    for (int i = compiled_in ? -1 : 0; i < n && e == cudaSuccess; ++i) {
        if (i >= 0 && !k[i]) continue;
        float ms = 0.f, lo = -1.f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // rep 0 warms up
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = launch(i);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (lo < 0.f || ms < lo)) lo = ms;
        }
        // a candidate displaces the compiled-in kernel only when 2% faster
        const float margin = best == -1 ? 0.98f : 1.0f;
        if (e == cudaSuccess && (best == -2 || lo < margin * best_ms)) {
            best = i;
            best_ms = lo;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(oc);
    cudaFree(op);
    cudaFree(oph);
    if (e != cudaSuccess) {
        *log = std::string("timing the tuning candidates failed: ") + cudaGetErrorString(e);
        return nullptr;
    }
    if (best == -1) {  // the compiled-in kernel is the fastest: the plan keeps it
        log->clear();
        return nullptr;
    }
    if (best < 0) return nullptr;
    p->sch = cand[best];  // fixed / fixed_cl -1: the plan runs k[best]
    return k[best];
#endif
}

}  // namespace cwtk

extern "C" cwt_status cwt_specialize_check(int n_fft, char *log, size_t log_len) {
    cwtk::MrSchedule s;
    int cl = 1;
    if (n_fft < cwtk::kMinFft || n_fft > cwtk::kMaxClusterFft || (n_fft & (n_fft - 1)) == 0) return CWT_EUNSUPPORTED;
    if (!(n_fft <= cwtk::kMaxFft && cwtk::mr_schedule(n_fft, &s)) && !cwtk::mr_cluster_split(n_fft, &cl, &s, true))
        return CWT_EUNSUPPORTED;
    std::string lg;
    const int rows = cl == 1 && s.T < 128 ? 256 / s.T : 1;
    const bool ok = cwtk::jit_compile_check(s, rows, cl, &lg);
    if (log && log_len) std::snprintf(log, log_len, "%s", lg.c_str());
    return ok ? CWT_OK : CWT_ECUDA;
}
