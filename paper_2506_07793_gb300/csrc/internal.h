// internal.h -- plan state and kernel launchers shared by the library's
// translation units (not part of the public ABI; see include/cwt.h).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include <string>
#include <vector>

#include "cwt.h"
#include "mixed_radix.cuh"

namespace cwtk {

struct JitKernels;  // jit.cu


constexpr int kMinFft = 32;        // smallest padded length (keeps radix passes >= 2)
constexpr int kMaxFftLog2 = 14;    // largest one-CTA length 16384 (shared-memory row)
constexpr int kMaxFft = 1 << kMaxFftLog2;
constexpr int kMaxClusterFftLog2 = 17;  // up to 131072 on a cluster of 8 CTAs
constexpr int kMaxClusterFft = 1 << kMaxClusterFftLog2;
constexpr double kBandRelThreshold = 1e-10;  // bins below this fraction of a scale's peak are skipped

// Device (cudaMalloc) and pinned host (cudaMallocHost) allocations of the
// library, with host-side failure injection (alloc.cu).
cudaError_t dev_alloc(void **p, size_t bytes);
cudaError_t host_alloc(void **p, size_t bytes);
template <class T>
cudaError_t dmalloc(T **p, size_t bytes) {
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}
template <class T>
cudaError_t hmalloc(T **p, size_t bytes) {
    return host_alloc(reinterpret_cast<void **>(p), bytes);
}

// Bounds-check builds (-DCWT_BOUNDS_CHECK, check.cuh): true when a kernel
// recorded an out-of-range shared-memory access or index since the last call
// (the words are cleared); *where names the first one.  Always false in an
// ordinary build.
bool check_collect(std::string *where);

// Per-device FP32 twiddle table exp(2 pi i m / 2^17), built in FP64 on first use.
cudaError_t device_twiddles(const float2 **out);

struct BatchState;
void free_batch_state(BatchState *b);

struct ProfEvent {
    int kernel;
    cudaEvent_t start, stop;
};

}  // namespace cwtk

struct cwt_plan_s {
    int device = 0;
    int C = 0, n = 0, S = 0;
    int N = 0;        // padded forward length
    int d = 1;        // decimation
    int fold = 1;     // spectral fold factor (power of two dividing d)
    int M = 0;        // inverse length N / fold
    int sub = 1;      // d / fold: remaining subsampling of the inverse output
    int n_out = 0;
    double fs = 0;
    int wavelet = 0;
    double gmw_gamma = 3.0;  // gamma of Eq. 5 (CWT_WAVELET_GMW only)
    double norm2 = 1.0;      // sum_m |w[m]|^2 of each scale (1: unit energy, 2: MNE's convention)
    int pad_extra = 0;       // linear edges: samples added before padding (R + 1)
    unsigned grid_ok_lengths = 0;  // batch: bit log2(N_e) set once every scale passed
                                   // the grid check at that epoch length
    unsigned outputs = 0;
    int io = CWT_DTYPE_F32;
    std::vector<double> freqs, cycles;

    bool mr = false;            // smooth (non power-of-two) N: mixed-radix kernels
    cwtk::MrSchedule sch{};     // their pass schedule (of N / cl points)
    int cl = 1;                 // smooth N above 16384: CTAs per row (a cluster), N = cl * sch.N
    cwtk::JitKernels *jit = nullptr;  // kernels compiled at plan creation for sch (jit.cu; shared, cached)
    bool tuned = false;               // jit chosen by timing candidate schedules (specialize = 2)
    float2 *twN = nullptr;      // exp(2 pi i m / N), m < N (mixed-radix plans only)
    float2 *twL = nullptr;      // cl > 1: exp(2 pi i m / NL), m < NL = N / cl
    float *bank = nullptr;    // [S][N] W_s[k] / N (real)
    int *band = nullptr;      // [S][2]: start, length
    float2 *spec = nullptr;   // [C][N] forward spectra (workspace)
    int precision = CWT_PREC_FP32;  // cwt_precision of the inverse FFTs
    float *tc_chmax = nullptr;  // tensor-core plans: [C] max |Re|, |Im| of each spectrum
    float *tc_wl1 = nullptr;    // tensor-core plans: [S] sum of |W_s| over the band
    const float2 *tw = nullptr;
    size_t bytes = 0;
    double bank_ms = 0;

    // host-buffer execution staging (allocated on first use)
    void *stage_in = nullptr, *stage_c = nullptr, *stage_p = nullptr, *stage_ph = nullptr;
    size_t stage_bytes = 0;

    cwtk::BatchState *batch = nullptr;  // batch path state (banks per length, graph, tuning)

    bool profiling = false;
    std::vector<cwtk::ProfEvent> prof, prof_pool;
    std::string last_error;
};

namespace cwtk {

// Opt a kernel into `bytes` of dynamic shared memory once per device
// (one bit of *done per device ordinal < 32; setting it twice is harmless).
template <typename K>
cudaError_t ensure_smem_attr(K *kernel, int bytes, std::atomic<unsigned> *done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // one bit per device; host threads may race here, and setting the
    // attribute twice is harmless
    if (dev < 32 && (done->load(std::memory_order_acquire) & (1u << dev))) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && dev < 32) done->fetch_or(1u << dev, std::memory_order_acq_rel);
    return e;
}

// Host-side check of the wavelet kind and its shape parameters (n_cycles
// already checked > 0 and finite): Morlet/Gabor take sigma = n_cycles; the
// generalized Morse wavelet takes beta = n_cycles <= 1000 and 0 < gamma <= 64.
inline bool wavelet_params_ok(int wavelet, const double *n_cycles, int n, double gamma) {
    if (wavelet == CWT_WAVELET_MORLET || wavelet == CWT_WAVELET_GABOR) return true;
    if (wavelet != CWT_WAVELET_GMW) return false;
    if (!(gamma > 0.0) || !(gamma <= 64.0)) return false;
    for (int i = 0; i < n; ++i)
        if (!(n_cycles[i] <= 1000.0)) return false;
    return true;
}

// Scales whose wavelet the N-point grid cannot represent are refused.  The
// spectrum sampled on the bins, P[k] = sum_q G((k/N + q) fs), is normalised
// to unit energy by sum_k P[k]^2; when every P[k] is below ~1e-154 that sum
// underflows in FP64 and the scale would come out as zeros.  This happens
// only when the carrier lies far below the first DFT bin (e.g. 1.5 Hz with
// sigma = 7 in a 32-point window at 500 Hz, where the first bin sits at ten
// times the carrier).  The library refuses (CWT_EINVAL) a scale whose largest
// |P[k]| is below kMinSpectrumPeak; every other scale, resolved or not, is
// the exact alias-summed closed form.
constexpr double kMinSpectrumPeak = 1e-150;

// Largest |P[k]| over the bins that can hold the maximum of a scale's
// alias-summed spectrum (Eq. 3/4 for Morlet/Gabor with sig = sigma, Eq. 5 for
// the GMW with sig = beta): the two bins around the carrier F and the bins
// 0, 1 and N - 1 around DC, with the aliases q = -2..2.  Host-only.
inline double spectrum_peak_on_grid(int wavelet, double F, double sig, double gamma, double fs,
                                    int N) {
    auto g = [&](double nu) -> double {
        if (wavelet == CWT_WAVELET_GMW) {
            if (!(nu > 0.0)) return 0.0;
            const double wp = std::pow(sig / gamma, 1.0 / gamma);
            const double w = wp * nu / F;
            const double la = std::log(2.0) + (sig / gamma) * (1.0 + std::log(gamma) - std::log(sig));
            return std::exp(la + sig * std::log(w) - std::pow(w, gamma));
        }
        const double kappa = wavelet == CWT_WAVELET_GABOR ? 0.0 : std::exp(-0.5 * sig * sig);
        const double u = nu / F;
        return std::exp(-0.5 * sig * sig * (u - 1.0) * (u - 1.0)) - kappa * std::exp(-0.5 * sig * sig * u * u);
    };
    const long long k0 = (long long)std::floor(F * (double)N / fs);
    const long long ks[5] = {0, 1, N - 1, k0, k0 + 1};
    double best = 0.0;
    for (long long k : ks) {
        const long long kk = ((k % N) + N) % N;
        double sum = 0.0;
        for (int q = -2; q <= 2; ++q) sum += g(((double)kk / (double)N + q) * fs);
        best = std::max(best, std::fabs(sum));
    }
    return best;
}

// True when every scale passes the check above at length N.
inline bool scales_on_grid(int wavelet, const double *F, const double *sig, int S, double gamma,
                           double fs, int N) {
    for (int s = 0; s < S; ++s)
        if (!(spectrum_peak_on_grid(wavelet, F[s], sig[s], gamma, fs, N) >= kMinSpectrumPeak)) return false;
    return true;
}

// Launchers (return the launch error, if any).
cudaError_t launch_bank(cwt_plan_s *p, cudaStream_t st);
// Bank and bands of the plan's scales for padded length N into the given
// buffers ([S][N] floats, [S][2] ints); synchronises `st`.
cudaError_t launch_bank_n(const cwt_plan_s *p, int N, float *bank, int *band, cudaStream_t st,
                          double *ms_out);
cudaError_t launch_forward(const cwt_plan_s *p, const void *signal, cudaStream_t st);
cudaError_t launch_scale_block(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                               cudaStream_t st);
cudaError_t launch_fft(const float2 *in, float2 *out, int log2n, int batch, int sign,
                       const float2 *tw, cudaStream_t st);
// Tensor-core inverse FFTs (tc_scale_block.cu): per-channel spectrum bounds
// after the forward FFT, per-scale band sums at plan creation, the scale block.
cudaError_t launch_tc_row_bounds(const cwt_plan_s *p, cudaStream_t st);
cudaError_t launch_tc_wl1(const cwt_plan_s *p, cudaStream_t st);
cudaError_t launch_scale_block_tc(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                  cudaStream_t st);
// Rows of 2^15..2^17 points on thread-block clusters (cluster.cu).
cudaError_t launch_forward_cluster(const cwt_plan_s *p, const void *signal, cudaStream_t st);
cudaError_t launch_scale_block_cluster(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                       cudaStream_t st);
cudaError_t launch_fft_cluster(const float2 *in, float2 *out, int log2n, int batch, int sign,
                               const float2 *tw, cudaStream_t st);
// prepare_only: build the work items, generate missing banks and autotune a
// new batch shape (its candidate runs write valid outputs); otherwise launch
// the chosen schedule's graph once.
// Smooth lengths (smooth.cu): schedule, per-N twiddles, kernels.
bool mr_schedule(int N, MrSchedule *out);
cudaError_t make_twiddles_n(int N, float2 *tw, cudaStream_t st);
cudaError_t launch_forward_mr(const cwt_plan_s *p, const void *signal, cudaStream_t st);
// Support radius in samples of one scale's wavelet (envelope below 1e-9 of its
// peak beyond it), or -1 past 2^17 samples (support.cu).
int support_radius(int wavelet, double F, double sig, double gamma, double fs);
// Plan-time specialization (jit.cu): the fixed-length kernels compiled for
// schedule s with `rows` rows per CTA (cl = 1), or as the local row of a
// cluster of cl CTAs, on `device` (cached), or nullptr with the reason in
// *log; the same compile for sm_103a without a device, as a check.
JitKernels *jit_kernels(const MrSchedule &s, int rows, int cl, int device, std::string *log);
bool jit_compile_check(const MrSchedule &s, int rows, int cl, std::string *log);
// cwt_options.specialize = 2: the fixed-length kernels of up to eight candidate
// schedules (mr_schedule_candidates), each timed on the plan's rows; the
// fastest, with p->sch set to its schedule (jit.cu).
JitKernels *jit_tune(cwt_plan_s *p, cudaStream_t st, std::string *log);
// The scheduler's schedule of N first, its passes on up to two other thread
// counts, then the cost model's two cheapest radix sets in each of their pass
// orders; returns how many (smooth.cu).
int mr_schedule_candidates(int N, MrSchedule *out, int max_out);
// Rows per CTA of the runtime-schedule kernels for total_rows rows (smooth.cu).
int mr_launch_rows(const MrSchedule &sch, int total_rows);
// Smooth lengths above 16384 on clusters: the split N = CL NL, preferring
// local rows two CTAs per SM hold; jit: the plan compiles its kernels at
// creation, so every local schedule and cluster sizes up to 16 are open
// (smooth_cluster.cu).
bool mr_cluster_split(int N, int *cl, MrSchedule *sch, bool jit = false);
cudaError_t launch_forward_mr_cluster(const cwt_plan_s *p, const void *signal, cudaStream_t st);
cudaError_t launch_scale_block_mr_cluster(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                          cudaStream_t st);
cudaError_t launch_scale_block_mr(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                  cudaStream_t st);
cudaError_t batch_execute(cwt_plan_s *p, const cwt_epoch *epochs, int n_epochs, const float *in,
                          float2 *oc, float *op, float *oph, cudaStream_t st, bool prepare_only);
void batch_stats(const cwt_plan_s *p, cwt_batch_stats *s);

}  // namespace cwtk
