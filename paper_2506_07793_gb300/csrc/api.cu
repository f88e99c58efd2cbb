// api.cu -- the library's C ABI (include/cwt.h): argument validation, plan
// lifecycle, execution entry points and profiling counters.
//
// Plan creation follows Section "Optimizing performance" of arXiv 2506.07793:
// the Fourier-transformed wavelets are generated in GPU memory once, then data
// are transformed there, and results leave the GPU only when asked for.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>

#include "fft_core.cuh"
#include "internal.h"
#include "smooth_kernel.cuh"

using cwtk::ilog2c;

namespace {

constexpr double kPi = 3.14159265358979323846;

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

cwt_status fail_cuda(cwt_plan_s *p, cudaError_t e) {
    if (p) p->last_error = cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return CWT_ENOMEM;
    return CWT_ECUDA;
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// Device pointer of the given device, 16-byte aligned.
bool device_ptr_ok(const void *ptr, int dev) {
    if (!ptr || (reinterpret_cast<uintptr_t>(ptr) & 15u)) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();  // clear the non-sticky error
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

cudaError_t prof_begin(cwt_plan_s *p, int kernel, cudaStream_t st, cwtk::ProfEvent *ev) {
    if (!p->profiling) return cudaSuccess;
    if (p->prof_pool.empty()) {
        cwtk::ProfEvent e{};
        cudaError_t r = cudaEventCreate(&e.start);
        if (r == cudaSuccess) r = cudaEventCreate(&e.stop);
        if (r != cudaSuccess) return r;
        p->prof_pool.push_back(e);
    }
    *ev = p->prof_pool.back();
    p->prof_pool.pop_back();
    ev->kernel = kernel;
    return cudaEventRecord(ev->start, st);
}

cudaError_t prof_end(cwt_plan_s *p, cudaStream_t st, cwtk::ProfEvent *ev) {
    if (!p->profiling) return cudaSuccess;
    cudaError_t r = cudaEventRecord(ev->stop, st);
    p->prof.push_back(*ev);
    return r;
}

size_t out_elem_bytes(const cwt_plan_s *p) { return p->io == CWT_DTYPE_F64 ? 8 : 4; }

// Bounds-check builds: wait for the launches on `st` and report a recorded
// out-of-range access as CWT_EDEVICE.  Ordinary builds: nothing.
cwt_status check_after(cwt_plan_s *p, cudaStream_t st) {
#ifdef CWT_BOUNDS_CHECK
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(p, e);
    std::string where;
    if (cwtk::check_collect(&where)) {
        if (p) p->last_error = where;
        return CWT_EDEVICE;
    }
#else
    (void)p;
    (void)st;
#endif
    return CWT_OK;
}

cwt_status run_execute(cwt_plan_s *p, const void *sig, void *oc, void *op, void *oph,
                       cudaStream_t st) {
    cwtk::ProfEvent ev{};
    cudaError_t e = prof_begin(p, CWT_KERNEL_FORWARD_FFT, st, &ev);
    if (e == cudaSuccess) e = cwtk::launch_forward(p, sig, st);
    const bool tc = p->precision != CWT_PREC_FP32;
    if (e == cudaSuccess && tc) e = cwtk::launch_tc_row_bounds(p, st);
    if (e == cudaSuccess) e = prof_end(p, st, &ev);
    if (e == cudaSuccess) e = prof_begin(p, CWT_KERNEL_SCALE_BLOCK, st, &ev);
    if (e == cudaSuccess)
        e = tc ? cwtk::launch_scale_block_tc(p, oc, op, oph, st) : cwtk::launch_scale_block(p, oc, op, oph, st);
    if (e == cudaSuccess) e = prof_end(p, st, &ev);
    if (e != cudaSuccess) return fail_cuda(p, e);
    return check_after(p, st);
}

void free_plan_memory(cwt_plan_s *p) {
    cwtk::free_batch_state(p->batch);
    p->batch = nullptr;
    cudaFree(p->bank);
    cudaFree(p->band);
    cudaFree(p->spec);
    cudaFree(p->tc_chmax);
    cudaFree(p->tc_wl1);
    if (p->twL != p->twN) cudaFree(p->twL);
    cudaFree(p->twN);
    cudaFree(p->stage_in);
    cudaFree(p->stage_c);
    cudaFree(p->stage_p);
    cudaFree(p->stage_ph);
    for (auto &e : p->prof) {
        cudaEventDestroy(e.start);
        cudaEventDestroy(e.stop);
    }
    for (auto &e : p->prof_pool) {
        cudaEventDestroy(e.start);
        cudaEventDestroy(e.stop);
    }
    p->prof.clear();
    p->prof_pool.clear();
}

}  // namespace

extern "C" {

const char *cwt_status_str(cwt_status s) {
    switch (s) {
        case CWT_OK: return "CWT_OK";
        case CWT_EINVAL: return "CWT_EINVAL: invalid argument";
        case CWT_ENOMEM: return "CWT_ENOMEM: out of memory";
        case CWT_EUNSUPPORTED: return "CWT_EUNSUPPORTED: not supported by this build";
        case CWT_ECUDA: return "CWT_ECUDA: CUDA runtime error";
        case CWT_EAGAIN: return "CWT_EAGAIN: not ready";
        case CWT_EBUSY: return "CWT_EBUSY: admission refused";
        case CWT_EDEVICE: return "CWT_EDEVICE: device reported an error";
    }
    return "CWT_UNKNOWN_STATUS";
}

// the Python binding mirrors this layout
static_assert(sizeof(cwt_options) == 64 && offsetof(cwt_options, gmw_gamma) == 24 &&
                  offsetof(cwt_options, normalization) == 32 && offsetof(cwt_options, specialize) == 36,
              "cwt_options layout");
static_assert(sizeof(cwt_plan_info_t) == 120 && offsetof(cwt_plan_info_t, radices) == 64 &&
                  offsetof(cwt_plan_info_t, fixed_kernel) == 104 && offsetof(cwt_plan_info_t, cluster) == 112 &&
                  offsetof(cwt_plan_info_t, specialized) == 116,
              "cwt_plan_info_t layout");

cwt_status cwt_options_init(cwt_options *opt) {
    if (!opt) return CWT_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = CWT_PREC_FP32;
    opt->decimation = 1;
    opt->pad_policy = CWT_PAD_POW2;
    opt->fft_length = 0;
    opt->io_dtype = CWT_DTYPE_F32;
    opt->gmw_gamma = 3.0;
    return CWT_OK;
}

cwt_status cwt_fft_length(int samples, int pad_policy, int *n_fft) {
    if (!n_fft || samples < 1) return CWT_EINVAL;
    if (pad_policy == CWT_PAD_SMOOTH) {
        // smallest 2,3,5,7-smooth length >= max(samples, 32) that the kernels
        // run: one CTA per row, else a cluster split N = CL NL (passed over:
        // the 43 lengths with neither, e.g. 5^7)
        for (int m = samples < cwtk::kMinFft ? cwtk::kMinFft : samples; m <= cwtk::kMaxClusterFft; ++m) {
            int x = m;
            for (int f : {2, 3, 5, 7})
                while (x % f == 0) x /= f;
            if (x != 1) continue;
            cwtk::MrSchedule sch;
            int cl = 1;
            if (!is_pow2(m) && !(m <= cwtk::kMaxFft && cwtk::mr_schedule(m, &sch)) &&
                !cwtk::mr_cluster_split(m, &cl, &sch))
                continue;
            *n_fft = m;
            return CWT_OK;
        }
        return CWT_EUNSUPPORTED;
    }
    if (pad_policy != CWT_PAD_POW2) return CWT_EINVAL;
    if (samples > cwtk::kMaxClusterFft) return CWT_EUNSUPPORTED;
    int N = cwtk::kMinFft;
    while (N < samples) N <<= 1;
    *n_fft = N;
    return CWT_OK;
}

cwt_status cwt_plan_create(cwt_plan *out, int channels, int samples, double fs,
                           const double *freqs_hz, int n_freqs, const double *n_cycles,
                           int wavelet, unsigned output_kinds, const cwt_options *opt) {
    // ---- host-side validation (no CUDA call before this block ends) ----
    if (!out || channels < 1 || samples < 1 || !(fs > 0.0) || !std::isfinite(fs) || !freqs_hz ||
        !n_cycles || n_freqs < 1)
        return CWT_EINVAL;
    for (int i = 0; i < n_freqs; ++i) {
        if (!(freqs_hz[i] > 0.0) || !(freqs_hz[i] < 0.5 * fs) || !std::isfinite(freqs_hz[i]))
            return CWT_EINVAL;
        if (!(n_cycles[i] > 0.0) || !std::isfinite(n_cycles[i])) return CWT_EINVAL;
    }
    const unsigned all = CWT_OUT_COMPLEX | CWT_OUT_POWER | CWT_OUT_PHASE;
    if (output_kinds == 0 || (output_kinds & ~all)) return CWT_EINVAL;
    cwt_options o;
    cwt_options_init(&o);
    if (opt) o = *opt;
    if (!cwtk::wavelet_params_ok(wavelet, n_cycles, n_freqs, o.gmw_gamma)) return CWT_EINVAL;
    if (o.decimation < 1) return CWT_EINVAL;
    if (o.io_dtype != CWT_DTYPE_F32 && o.io_dtype != CWT_DTYPE_F64) return CWT_EINVAL;
    const bool tc = o.precision == CWT_PREC_TC_FP16 || o.precision == CWT_PREC_TC_BF16;
    if (o.precision != CWT_PREC_FP32 && !tc) return CWT_EINVAL;
    if (o.edge_mode != CWT_EDGE_CYCLIC && o.edge_mode != CWT_EDGE_LINEAR) return CWT_EINVAL;
    if (o.normalization != CWT_NORM_UNIT_ENERGY && o.normalization != CWT_NORM_MNE) return CWT_EINVAL;
    if (o.specialize < 0 || o.specialize > 2) return CWT_EINVAL;
    // linear edges: pad by the widest wavelet's support radius R (envelope
    // below 1e-9 of its peak beyond R samples, support.cu) so that nothing wraps
    int pad_extra = 0;
    if (o.edge_mode == CWT_EDGE_LINEAR) {
        int R = 0;
        for (int i = 0; i < n_freqs; ++i) {
            const int r = cwtk::support_radius(wavelet, freqs_hz[i], n_cycles[i], o.gmw_gamma, fs);
            if (r < 0) return CWT_EUNSUPPORTED;
            R = std::max(R, r);
        }
        if (!((double)R + 1.0 + samples <= (double)cwtk::kMaxClusterFft)) return CWT_EUNSUPPORTED;
        pad_extra = R + 1;
    }
    const int min_len = samples + pad_extra;
    int N = 0;
    if (o.fft_length != 0) {
        if (o.fft_length < min_len || o.fft_length < cwtk::kMinFft) return CWT_EINVAL;
        if (!is_pow2(o.fft_length)) {
            cwtk::MrSchedule sch;
            int x = o.fft_length;
            for (int f : {2, 3, 5, 7})
                while (x % f == 0) x /= f;
            if (x != 1) return CWT_EINVAL;  // not 2,3,5,7-smooth
            int cl = 1;
            if (!(o.fft_length <= cwtk::kMaxFft && cwtk::mr_schedule(o.fft_length, &sch)) &&
                !cwtk::mr_cluster_split(o.fft_length, &cl, &sch))
                return CWT_EUNSUPPORTED;
        }
        if (o.fft_length > cwtk::kMaxClusterFft) return CWT_EUNSUPPORTED;
        N = o.fft_length;
    } else {
        cwt_status st = cwt_fft_length(min_len, o.pad_policy, &N);
        if (st != CWT_OK) return st;
    }
    if ((long long)channels * n_freqs > (1ll << 30)) return CWT_EUNSUPPORTED;
    // tensor-core inverse FFTs: power-of-two rows of 16384 .. 131072 points
    if (tc && (!is_pow2(N) || N < cwtk::kMaxFft || N > cwtk::kMaxClusterFft)) return CWT_EUNSUPPORTED;
    if (!cwtk::scales_on_grid(wavelet, freqs_hz, n_cycles, n_freqs, o.gmw_gamma, fs, N))
        return CWT_EINVAL;

    cwt_plan_s *p = new (std::nothrow) cwt_plan_s();
    if (!p) return CWT_ENOMEM;
    p->C = channels;
    p->n = samples;
    p->S = n_freqs;
    p->N = N;
    p->d = o.decimation;
    p->mr = !is_pow2(N);
    if (p->mr) {
        // one CTA per row where a schedule covers N, else a cluster (checked above)
        if (!(N <= cwtk::kMaxFft && cwtk::mr_schedule(N, &p->sch)))
            cwtk::mr_cluster_split(N, &p->cl, &p->sch, o.specialize != 0);
    }
    p->precision = o.precision;
    int f = 1;  // no spectral fold on the cluster and tensor-core paths
    while (!p->mr && !tc && (p->d % (2 * f)) == 0 && N / (2 * f) >= cwtk::kMinFft) f *= 2;
    p->fold = f;
    p->M = N / f;
    p->sub = p->d / f;
    p->n_out = (samples + p->d - 1) / p->d;
    p->fs = fs;
    p->wavelet = wavelet;
    p->gmw_gamma = o.gmw_gamma;
    p->pad_extra = pad_extra;
    p->norm2 = o.normalization == CWT_NORM_MNE ? 2.0 : 1.0;
    p->outputs = output_kinds;
    p->io = o.io_dtype;
    p->freqs.assign(freqs_hz, freqs_hz + n_freqs);
    p->cycles.assign(n_cycles, n_cycles + n_freqs);

    // ---- device side ----
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cwtk::device_twiddles(&p->tw);
    const size_t bank_b = sizeof(float) * (size_t)n_freqs * N;
    const size_t band_b = sizeof(int) * 2 * (size_t)n_freqs;
    const size_t spec_b = sizeof(float2) * (size_t)channels * N;
    if (e == cudaSuccess) e = cwtk::dmalloc(&p->bank, bank_b);
    if (e == cudaSuccess) e = cwtk::dmalloc(&p->band, band_b);
    if (e == cudaSuccess) e = cwtk::dmalloc(&p->spec, spec_b);
    p->bytes = bank_b + band_b + spec_b;
    cudaStream_t st = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess && p->mr) {
        e = cwtk::dmalloc(&p->twN, sizeof(float2) * (size_t)N);
        if (e == cudaSuccess) e = cwtk::make_twiddles_n(N, p->twN, st);
        p->bytes += sizeof(float2) * (size_t)N;
        p->twL = p->twN;
        if (e == cudaSuccess && p->cl > 1) {
            const int NL = N / p->cl;
            e = cwtk::dmalloc(&p->twL, sizeof(float2) * (size_t)NL);
            if (e == cudaSuccess) e = cwtk::make_twiddles_n(NL, p->twL, st);
            p->bytes += sizeof(float2) * (size_t)NL;
        }
    }
    const bool tune = o.specialize == 2 && p->mr;
    // a split above 8 CTAs with no kernel compiled in compiles the scheduler's
    // schedule now, also before tuning (which then has a kernel to fall back on)
    const bool wide = p->cl > 8 && p->sch.fixed_cl < 0;
    if (e == cudaSuccess && o.specialize && (!tune || wide) && p->mr &&
        (p->cl == 1 ? p->sch.fixed < 0 : p->sch.fixed_cl < 0)) {
        // a failed compile or load is not a plan error: the runtime-schedule kernels run
        std::string log;
        const int rows = p->cl == 1 ? cwtk::mr_launch_rows(p->sch, channels * n_freqs) : 1;
        p->jit = cwtk::jit_kernels(p->sch, rows, p->cl, p->device, &log);
        if (!p->jit) p->last_error = log;
        if (!p->jit && wide) {
            // no kernel for that cluster size: the portable split and its table
            p->bytes -= sizeof(float2) * (size_t)(N / p->cl);
            cwtk::mr_cluster_split(N, &p->cl, &p->sch, false);
            e = cudaStreamSynchronize(st);  // the old table's fill has finished
            cudaFree(p->twL);
            p->twL = nullptr;
            const int NL = N / p->cl;
            if (e == cudaSuccess) e = cwtk::dmalloc(&p->twL, sizeof(float2) * (size_t)NL);
            if (e == cudaSuccess) e = cwtk::make_twiddles_n(NL, p->twL, st);
            p->bytes += sizeof(float2) * (size_t)NL;
        }
    }
    if (e == cudaSuccess) e = cwtk::launch_bank(p, st);
    if (e == cudaSuccess && tc) {
        e = cwtk::dmalloc(&p->tc_chmax, sizeof(float) * (size_t)channels);
        if (e == cudaSuccess) e = cwtk::dmalloc(&p->tc_wl1, sizeof(float) * (size_t)n_freqs);
        p->bytes += sizeof(float) * ((size_t)channels + n_freqs);
        if (e == cudaSuccess) e = cwtk::launch_tc_wl1(p, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess && tune) {
        // candidates timed on the plan's rows once the bank is in place; a
        // failure leaves the plan on the runtime-schedule kernels
        e = cudaStreamSynchronize(st);
        std::string log;
        cwtk::JitKernels *k = e == cudaSuccess ? cwtk::jit_tune(p, st, &log) : nullptr;
        p->tuned = k != nullptr;
        if (k) p->jit = k;
        else if (!p->jit) p->last_error = log;
    }
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cwt_status s = fail_cuda(p, e);
        free_plan_memory(p);
        delete p;
        return s;
    }
    *out = p;
    return CWT_OK;
}

cwt_status cwt_plan_destroy(cwt_plan p) {
    if (!p) return CWT_OK;
    {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        free_plan_memory(p);
    }
    delete p;
    return CWT_OK;
}

namespace {

// radices[8] (0-terminated), the inlined pair (0, 0: generic) and the
// fixed-kernel flag of a mixed-radix schedule; radices and pair pre-zeroed.
// As the local row of a cluster (cl > 1) the schedule runs on the cluster
// kernels: no inlined pair, fixed when its local length is compiled in.
void describe_schedule(const cwtk::MrSchedule &sch, int cl, int *radices, int *pair, int *fixed) {
    for (int q = 0; q < sch.np && q < 7; ++q) radices[q] = sch.p[q].R;
    if (cl > 1) {
        *fixed = sch.fixed_cl >= 0;
        return;
    }
#define CWT_MR_CASE(I, A, B) \
    if (sch.fast == I) pair[0] = A, pair[1] = B;
    CWT_MR_FAST_PAIRS(CWT_MR_CASE)
#undef CWT_MR_CASE
    *fixed = sch.fixed >= 0;
}

}  // namespace

cwt_status cwt_plan_info(cwt_plan p, cwt_plan_info_t *info) {
    if (!p || !info) return CWT_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->channels = p->C;
    info->samples = p->n;
    info->scales = p->S;
    info->fft_length = p->N;
    info->n_out = p->n_out;
    info->decimation = p->d;
    info->fold = p->fold;
    info->inverse_length = p->M;
    info->device = p->device;
    info->io_dtype = p->io;
    info->output_kinds = p->outputs;
    info->workspace_bytes = p->bytes + p->stage_bytes;
    info->bank_ms = p->bank_ms;
    info->precision = p->precision;
    info->cluster = p->mr ? p->cl : (p->M > cwtk::kMaxFft ? p->M / cwtk::kMaxFft : 1);
    if (p->mr) describe_schedule(p->sch, p->cl, info->radices, info->inlined_pair, &info->fixed_kernel);
    info->specialized = p->jit == nullptr ? 0 : p->tuned ? 2 : 1;
    if (p->jit) {  // the compiled-at-creation kernels are fixed-length ones
        info->fixed_kernel = 1;
        info->inlined_pair[0] = info->inlined_pair[1] = 0;
    }
    return CWT_OK;
}

cwt_status cwt_smooth_schedule(int n_fft, int *radices, int *threads, int *inlined_pair,
                               int *fixed_kernel) {
    if (!radices || !threads || !inlined_pair || !fixed_kernel) return CWT_EINVAL;
    cwtk::MrSchedule sch;
    if (is_pow2(n_fft) || !cwtk::mr_schedule(n_fft, &sch)) return CWT_EUNSUPPORTED;
    for (int q = 0; q < 8; ++q) radices[q] = 0;
    inlined_pair[0] = inlined_pair[1] = 0;
    describe_schedule(sch, 1, radices, inlined_pair, fixed_kernel);
    *threads = sch.T;
    return CWT_OK;
}

cwt_status cwt_smooth_cluster(int n_fft, int specialize, int *cluster, int *radices, int *fixed_kernel) {
    if (!cluster || !radices || !fixed_kernel || specialize < 0 || specialize > 2) return CWT_EINVAL;
    cwtk::MrSchedule sch;
    int cl = 1;
    if (is_pow2(n_fft) || n_fft < cwtk::kMinFft || n_fft > cwtk::kMaxClusterFft) return CWT_EUNSUPPORTED;
    if (!(n_fft <= cwtk::kMaxFft && cwtk::mr_schedule(n_fft, &sch)) &&
        !cwtk::mr_cluster_split(n_fft, &cl, &sch, specialize != 0))
        return CWT_EUNSUPPORTED;
    int pair[2] = {0, 0};
    for (int q = 0; q < 8; ++q) radices[q] = 0;
    describe_schedule(sch, cl, radices, pair, fixed_kernel);
    *cluster = cl;
    return CWT_OK;
}

size_t cwt_plan_workspace_bytes(cwt_plan p) { return p ? p->bytes + p->stage_bytes : 0; }

const char *cwt_plan_last_error(cwt_plan p) { return p ? p->last_error.c_str() : ""; }

cwt_status cwt_execute(cwt_plan p, const void *d_signal, void *d_complex, void *d_power,
                       void *d_phase, void *stream) {
    if (!p) return CWT_EINVAL;
    const bool wc = p->outputs & CWT_OUT_COMPLEX, wp = p->outputs & CWT_OUT_POWER,
               wph = p->outputs & CWT_OUT_PHASE;
    if (wc != (d_complex != nullptr) || wp != (d_power != nullptr) || wph != (d_phase != nullptr))
        return CWT_EINVAL;
    DeviceGuard g(p->device);
    if (!g.ok) return CWT_ECUDA;
    if (!device_ptr_ok(d_signal, p->device)) return CWT_EINVAL;
    if (wc && !device_ptr_ok(d_complex, p->device)) return CWT_EINVAL;
    if (wp && !device_ptr_ok(d_power, p->device)) return CWT_EINVAL;
    if (wph && !device_ptr_ok(d_phase, p->device)) return CWT_EINVAL;
    return run_execute(p, d_signal, d_complex, d_power, d_phase, (cudaStream_t)stream);
}

// Device address of page-locked host memory that the device can write
// directly (cudaHostAlloc, cudaHostRegister with mapping), or nullptr.
void *mapped_host_ptr(void *ptr) {
    if (!ptr || (reinterpret_cast<uintptr_t>(ptr) & 15u)) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();  // clear the non-sticky error
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    if (reinterpret_cast<uintptr_t>(at.devicePointer) & 15u) return nullptr;
    return at.devicePointer;
}

cwt_status cwt_execute_host(cwt_plan p, const void *h_signal, void *h_complex, void *h_power,
                            void *h_phase, void *stream) {
    if (!p || !h_signal) return CWT_EINVAL;
    const bool wc = p->outputs & CWT_OUT_COMPLEX, wp = p->outputs & CWT_OUT_POWER,
               wph = p->outputs & CWT_OUT_PHASE;
    if (wc != (h_complex != nullptr) || wp != (h_power != nullptr) || wph != (h_phase != nullptr))
        return CWT_EINVAL;
    DeviceGuard g(p->device);
    if (!g.ok) return CWT_ECUDA;
    const size_t eb = out_elem_bytes(p);
    const size_t in_b = eb * (size_t)p->C * p->n;
    const size_t out_b = eb * (size_t)p->C * p->S * p->n_out;
    cudaError_t e = cudaSuccess;
    if (!p->stage_in) {
        e = cwtk::dmalloc(&p->stage_in, in_b);
        if (e == cudaSuccess && wc) e = cwtk::dmalloc(&p->stage_c, 2 * out_b);
        if (e == cudaSuccess && wp) e = cwtk::dmalloc(&p->stage_p, out_b);
        if (e == cudaSuccess && wph) e = cwtk::dmalloc(&p->stage_ph, out_b);
        if (e != cudaSuccess) {
            cudaFree(p->stage_in);
            cudaFree(p->stage_c);
            cudaFree(p->stage_p);
            cudaFree(p->stage_ph);
            p->stage_in = p->stage_c = p->stage_p = p->stage_ph = nullptr;
            return fail_cuda(p, e);
        }
        p->stage_bytes = in_b + (wc ? 2 * out_b : 0) + (wp ? out_b : 0) + (wph ? out_b : 0);
    }
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemcpyAsync(p->stage_in, h_signal, in_b, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail_cuda(p, e);
    // outputs the device can address in host memory are written there by the
    // kernels' epilogues (one pass over the host link); the rest are staged
    void *mc = wc ? mapped_host_ptr(h_complex) : nullptr;
    void *mp = wp ? mapped_host_ptr(h_power) : nullptr;
    void *mph = wph ? mapped_host_ptr(h_phase) : nullptr;
    cwt_status s = run_execute(p, p->stage_in, wc ? (mc ? mc : p->stage_c) : nullptr,
                               wp ? (mp ? mp : p->stage_p) : nullptr,
                               wph ? (mph ? mph : p->stage_ph) : nullptr, st);
    if (s != CWT_OK) return s;
    if (wc && !mc) e = cudaMemcpyAsync(h_complex, p->stage_c, 2 * out_b, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && wp && !mp)
        e = cudaMemcpyAsync(h_power, p->stage_p, out_b, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && wph && !mph)
        e = cudaMemcpyAsync(h_phase, p->stage_ph, out_b, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? CWT_OK : fail_cuda(p, e);
}

cwt_status cwt_execute_batch(cwt_plan p, const cwt_epoch *epochs, int n_epochs, const void *d_in,
                             void *d_complex, void *d_power, void *d_phase, void *stream) {
    if (!p || n_epochs < 0 || (n_epochs > 0 && !epochs)) return CWT_EINVAL;
    const bool wc = p->outputs & CWT_OUT_COMPLEX, wp = p->outputs & CWT_OUT_POWER,
               wph = p->outputs & CWT_OUT_PHASE;
    if (wc != (d_complex != nullptr) || wp != (d_power != nullptr) || wph != (d_phase != nullptr))
        return CWT_EINVAL;
    // batches pad each epoch to pow2 and run FP32 inverse FFTs
    if (p->io != CWT_DTYPE_F32 || p->mr || p->precision != CWT_PREC_FP32) return CWT_EUNSUPPORTED;
    for (int i = 0; i < n_epochs; ++i) {
        const cwt_epoch &e = epochs[i];
        if (e.samples < 1 || e.samples > p->n || e.in_offset < 0 || e.out_offset < 0) return CWT_EINVAL;
        if (e.samples + p->pad_extra > 8192) return CWT_EUNSUPPORTED;
        // each epoch's own length N_e must represent every scale (checked once
        // per length and remembered)
        int Ne = 0;
        cwt_fft_length(e.samples + p->pad_extra, CWT_PAD_POW2, &Ne);
        const unsigned bit = 1u << ilog2c(Ne);
        if (!(p->grid_ok_lengths & bit)) {
            if (!cwtk::scales_on_grid(p->wavelet, p->freqs.data(), p->cycles.data(), p->S, p->gmw_gamma,
                                      p->fs, Ne))
                return CWT_EINVAL;
            p->grid_ok_lengths |= bit;
        }
    }
    if (n_epochs == 0) return CWT_OK;
    DeviceGuard g(p->device);
    if (!g.ok) return CWT_ECUDA;
    if (!device_ptr_ok(d_in, p->device)) return CWT_EINVAL;
    if (wc && !device_ptr_ok(d_complex, p->device)) return CWT_EINVAL;
    if (wp && !device_ptr_ok(d_power, p->device)) return CWT_EINVAL;
    if (wph && !device_ptr_ok(d_phase, p->device)) return CWT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // prepare (banks, work items, autotuning on a new shape), then one timed launch
    cudaError_t e = cwtk::batch_execute(p, epochs, n_epochs, (const float *)d_in, (float2 *)d_complex,
                                        (float *)d_power, (float *)d_phase, st, true);
    cwtk::ProfEvent ev{};
    if (e == cudaSuccess) e = prof_begin(p, CWT_KERNEL_BATCH, st, &ev);
    if (e == cudaSuccess)
        e = cwtk::batch_execute(p, epochs, n_epochs, (const float *)d_in, (float2 *)d_complex,
                                (float *)d_power, (float *)d_phase, st, false);
    if (e == cudaSuccess) e = prof_end(p, st, &ev);
    if (e != cudaSuccess) return fail_cuda(p, e);
    return check_after(p, st);
}

cwt_status cwt_plan_batch_stats(cwt_plan p, cwt_batch_stats *stats) {
    if (!p || !stats) return CWT_EINVAL;
    cwtk::batch_stats(p, stats);
    return CWT_OK;
}

cwt_status cwt_plan_bank(cwt_plan p, float *h_bank, int *h_band_start, int *h_band_len) {
    if (!p) return CWT_EINVAL;
    DeviceGuard g(p->device);
    if (!g.ok) return CWT_ECUDA;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && h_bank)
        e = cudaMemcpy(h_bank, p->bank, sizeof(float) * (size_t)p->S * p->N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && (h_band_start || h_band_len)) {
        int *tmp = new (std::nothrow) int[2 * (size_t)p->S];
        if (!tmp) return CWT_ENOMEM;
        e = cudaMemcpy(tmp, p->band, sizeof(int) * 2 * (size_t)p->S, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (int s = 0; s < p->S; ++s) {
                if (h_band_start) h_band_start[s] = tmp[2 * s];
                if (h_band_len) h_band_len[s] = tmp[2 * s + 1];
            }
        delete[] tmp;
    }
    return e == cudaSuccess ? CWT_OK : fail_cuda(p, e);
}

cwt_status cwt_fft(const void *d_in, void *d_out, int n, int batch, int direction, void *stream) {
    if (!d_in || !d_out || batch < 0 || !is_pow2(n) || (direction != 1 && direction != -1))
        return CWT_EINVAL;
    if (n < cwtk::kMinFft || n > cwtk::kMaxClusterFft) return CWT_EUNSUPPORTED;
    if (batch == 0) return CWT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CWT_ECUDA;
    if (!device_ptr_ok(d_in, dev) || !device_ptr_ok(d_out, dev)) return CWT_EINVAL;
    const float2 *tw = nullptr;
    cudaError_t e = cwtk::device_twiddles(&tw);
    if (e == cudaSuccess)
        e = cwtk::launch_fft((const float2 *)d_in, (float2 *)d_out, ilog2c(n), batch, direction, tw,
                             (cudaStream_t)stream);
    if (e == cudaErrorMemoryAllocation) return CWT_ENOMEM;
    if (e != cudaSuccess) return CWT_ECUDA;
    return check_after(nullptr, (cudaStream_t)stream);
}

cwt_status cwt_plan_set_profiling(cwt_plan p, int enable) {
    if (!p) return CWT_EINVAL;
    p->profiling = enable != 0;
    return CWT_OK;
}

cwt_status cwt_plan_profile_read(cwt_plan p, int kernel, int *launches, double *total_ms, int reset) {
    if (!p || kernel < 0 || kernel >= CWT_KERNEL_COUNT) return CWT_EINVAL;
    DeviceGuard g(p->device);
    if (!g.ok) return CWT_ECUDA;
    int cnt = 0;
    double ms = 0.0;
    if (kernel == CWT_KERNEL_BANK) {
        cnt = 1;
        ms = p->bank_ms;
    } else {
        for (auto &ev : p->prof) {
            if (ev.kernel != kernel) continue;
            cudaError_t e = cudaEventSynchronize(ev.stop);
            float f = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&f, ev.start, ev.stop);
            if (e != cudaSuccess) return fail_cuda(p, e);
            ms += f;
            ++cnt;
        }
        if (reset) {
            std::vector<cwtk::ProfEvent> keep;
            for (auto &ev : p->prof) {
                if (ev.kernel == kernel)
                    p->prof_pool.push_back(ev);
                else
                    keep.push_back(ev);
            }
            p->prof.swap(keep);
        }
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    return CWT_OK;
}

}  // extern "C"
