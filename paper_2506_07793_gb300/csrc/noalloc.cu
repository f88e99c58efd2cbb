// noalloc.cu -- cwt_execute_noalloc: the whole transform with no allocation.
//
// Some callers may not allocate GPU memory once they are running: real-time
// EEG / brain-machine-interface processing loops that must not block (a
// cudaMalloc or cudaFree can synchronise the device and stall the loop past
// its deadline), and plug-ins hosted by an application that owns the GPU
// memory budget.  This entry point serves them: the caller passes the signal
// and the outputs, and everything else the transform needs (twiddle table,
// wavelet bank, band table, spectra) lives in one file-scope device array of
// fixed size that every GPU loading this library holds until process exit.
//
// The arithmetic is the plan path's (FP64 bank evaluated in the same order,
// the same Stockham kernels), so the results match cwt_execute.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "fft_core.cuh"
#include "internal.h"
#include "phase.cuh"

namespace cwtk {
namespace {

constexpr size_t kScratchBytes = CWT_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTwBytes = sizeof(float2) * (size_t)kTwN;  // twiddle table at offset 0
constexpr int kNaThreads = 256;

// The scratch.  Host code must not use this name as an address: it takes the
// device address from cudaGetSymbolAddress (per device) and passes pointers.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void na_twiddle_kernel(float2 *tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < kTwN) {
        double s, c;
        sincospi(2.0 * (double)m / (double)kTwN, &s, &c);
        tw[m] = make_float2((float)c, (float)s);
    }
}

// Eq. 3 (Morlet spectrum in Hz, alias-summed) in FP64, the same evaluation
// order as the plan's generator so that the FP32 bank is identical.
__device__ double na_alias_sum(int k, int N, double fs, double f, double sg) {
    const double kappa = exp(-0.5 * sg * sg);
    const double reach = 40.0 * f / sg;
    const double base = (double)k / (double)N;
    const double q_lo = ceil(-reach / fs - base), q_hi = floor((f + reach) / fs - base);
    double v = 0.0;
    for (double q = q_lo; q <= q_hi; q += 1.0) {
        const double u = (base + q) * fs / f;
        const double a = u - 1.0;
        double g = exp(-0.5 * sg * sg * a * a);
        g -= kappa * exp(-0.5 * sg * sg * u * u);
        v += g;
    }
    return v;
}

// grid (nblk, S): per-block partial sums of the squared alias sums.
__global__ void __launch_bounds__(kNaThreads)
na_bank_energy_kernel(int N, double fs, const double *__restrict__ F, const double *__restrict__ sig,
                      double *__restrict__ partial) {
    __shared__ double red[kNaThreads];
    const int s = blockIdx.y;
    const int k = blockIdx.x * kNaThreads + threadIdx.x;
    const double v = k < N ? na_alias_sum(k, N, fs, F[s], sig[s]) : 0.0;
    red[threadIdx.x] = v * v;
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = red[0];
}

// One CTA per scale: normalise to unit energy (1/N folded in), FP32 bank, band.
__global__ void __launch_bounds__(kNaThreads)
na_bank_finish_kernel(int N, int nblk, double fs, const double *__restrict__ F,
                      const double *__restrict__ sig, const double *__restrict__ partial,
                      float *__restrict__ bank, int *__restrict__ band) {
    __shared__ double sd[kNaThreads];
    __shared__ int smin[kNaThreads], smax[kNaThreads];
    const int s = blockIdx.x;
    float *b = bank + (size_t)s * N;
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int i = 0; i < nblk; ++i) e += partial[(size_t)s * nblk + i];
        sd[0] = e;
    }
    __syncthreads();
    const double energy = sd[0];
    const double scale = energy > 0.0 ? 1.0 / sqrt((double)N * energy) : 0.0;
    __syncthreads();
    double mx = 0.0;
    for (int k = threadIdx.x; k < N; k += kNaThreads) {
        const double v = na_alias_sum(k, N, fs, F[s], sig[s]);
        b[k] = (float)(v * scale);
        mx = fmax(mx, fabs(v));
    }
    sd[threadIdx.x] = mx;
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + w]);
        __syncthreads();
    }
    const double thr = sd[0] * kBandRelThreshold;
    int lo = N, hi = -N;
    for (int k = threadIdx.x; k < N; k += kNaThreads) {
        if (fabs(na_alias_sum(k, N, fs, F[s], sig[s])) > thr) {
            const int ks = k < N / 2 ? k : k - N;
            lo = min(lo, ks);
            hi = max(hi, ks);
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            smin[threadIdx.x] = min(smin[threadIdx.x], smin[threadIdx.x + w]);
            smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int start = 0, len = 0;
        if (smax[0] >= smin[0]) {
            start = smin[0] < 0 ? smin[0] + N : smin[0];
            len = smax[0] - smin[0] + 1;
        }
        band[2 * s] = start;
        band[2 * s + 1] = len;
    }
}

template <int N>
__global__ void __launch_bounds__(RowConfig<N>::THREADS)
na_forward_kernel(const float *__restrict__ x, int C, int n, float2 *__restrict__ spec,
                  const float2 *__restrict__ tw) {
    using RC = RowConfig<N>;
    extern __shared__ float2 na_smem[];
    const int rl = threadIdx.x / RC::T, j = threadIdx.x % RC::T;
    const int row = blockIdx.x * RC::ROWS + rl;
    const bool act = row < C;
    float2 *sm = na_smem + rl * FftShape<N, RC::R>::SMEM_F2;
    const float *xr = x + (size_t)(act ? row : 0) * (size_t)n;
    float2 *out = spec + (size_t)(act ? row : 0) * (size_t)N;
    auto load = [&](int i) -> float2 { return make_float2((act && i < n) ? xr[i] : 0.f, 0.f); };
    auto store = [&](int t, float2 v) {
        if (act) out[t] = v;
    };
    fft_row<N, RC::R, -1>(sm, tw, j, load, store);
}

__device__ __noinline__ void na_store_phase(float *dst, float2 v) { *dst = phase_atan2(v.y, v.x); }

template <int N>
__global__ void __launch_bounds__(RowConfig<N>::THREADS)
na_scale_block_kernel(const float2 *__restrict__ spec, const float *__restrict__ bank,
                      const int *__restrict__ band, const float2 *__restrict__ tw, int S, int rows,
                      int n, float2 *oc, float *op, float *oph) {
    using RC = RowConfig<N>;
    extern __shared__ float2 na_smem[];
    const int rl = threadIdx.x / RC::T, j = threadIdx.x % RC::T;
    const int row = blockIdx.x * RC::ROWS + rl;
    const bool act = row < rows;
    const int c = act ? row / S : 0;
    const int s = act ? row - c * S : 0;
    float2 *sm = na_smem + rl * FftShape<N, RC::R>::SMEM_F2;
    const float2 *X = spec + (size_t)c * N;
    const float *W = bank + (size_t)s * N;
    const int b0 = band[2 * s], B = act ? band[2 * s + 1] : 0;
    auto load = [&](int k) -> float2 {
        if (((k - b0) & (N - 1)) < B) {
            const float2 xv = X[k];
            const float w = W[k];
            return make_float2(xv.x * w, xv.y * w);
        }
        return make_float2(0.f, 0.f);
    };
    const size_t obase = (size_t)row * (size_t)n;
    auto store = [&](int t, float2 v) {
        if (!act || t >= n) return;
        if (oc) oc[obase + t] = v;
        if (op) op[obase + t] = fmaf(v.x, v.x, v.y * v.y);
        if (oph) na_store_phase(oph + obase + t, v);
    };
    fft_row<N, RC::R, +1>(sm, tw, j, load, store);
}

template <int N>
cudaError_t na_run(const float *x, int C, int n, int S, char *base, size_t off_par, size_t off_part,
                   size_t off_band, size_t off_bank, size_t off_spec, double fs, float2 *oc,
                   float *op, float *oph, cudaStream_t st) {
    using RC = RowConfig<N>;
    static std::atomic<unsigned> attr_f{0}, attr_s{0};
    cudaError_t e = ensure_smem_attr(na_forward_kernel<N>, RC::SMEM_BYTES, &attr_f);
    if (e == cudaSuccess) e = ensure_smem_attr(na_scale_block_kernel<N>, RC::SMEM_BYTES, &attr_s);
    if (e != cudaSuccess) return e;
    const float2 *tw = (const float2 *)base;
    const double *F = (const double *)(base + off_par);
    const double *sig = F + S;
    double *partial = (double *)(base + off_part);
    int *band = (int *)(base + off_band);
    float *bank = (float *)(base + off_bank);
    float2 *spec = (float2 *)(base + off_spec);
    const int nblk = (N + kNaThreads - 1) / kNaThreads;
    na_bank_energy_kernel<<<dim3(nblk, S), kNaThreads, 0, st>>>(N, fs, F, sig, partial);
    na_bank_finish_kernel<<<S, kNaThreads, 0, st>>>(N, nblk, fs, F, sig, partial, bank, band);
    na_forward_kernel<N><<<(C + RC::ROWS - 1) / RC::ROWS, RC::THREADS, RC::SMEM_BYTES, st>>>(
        x, C, n, spec, tw);
    const int rows = C * S;
    na_scale_block_kernel<N><<<(rows + RC::ROWS - 1) / RC::ROWS, RC::THREADS, RC::SMEM_BYTES, st>>>(
        spec, bank, band, tw, S, rows, n, oc, op, oph);
    return cudaGetLastError();
}

std::mutex g_na_mutex;
char *g_na_base[64] = {};

// Once per device, with that device current: resolve the scratch's device
// address and write the twiddle table into it.
cudaError_t na_setup(int dev, cudaStream_t st, char **base) {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_base[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        na_twiddle_kernel<<<kTwN / 256, 256, 0, st>>>((float2 *)ptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        g_na_base[dev] = (char *)ptr;
    }
    *base = g_na_base[dev];
    return cudaSuccess;
}

bool na_dev_ptr(const void *p, int dev) {
    if (!p || (reinterpret_cast<uintptr_t>(p) & 15u)) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

}  // namespace
}  // namespace cwtk

extern "C" cwt_status cwt_execute_noalloc(const float *d_signal, int channels, int samples,
                                          double fs, const double *freqs_hz,
                                          const double *n_cycles, int n_freqs, void *d_complex,
                                          float *d_power, float *d_phase, void *stream) {
    using namespace cwtk;
    // ---- host-side validation, before any CUDA call ----
    if (channels < 1 || samples < 1 || !(fs > 0.0) || !std::isfinite(fs) || !freqs_hz ||
        !n_cycles || n_freqs < 1 || (!d_complex && !d_power && !d_phase))
        return CWT_EINVAL;
    for (int i = 0; i < n_freqs; ++i) {
        if (!(freqs_hz[i] > 0.0) || !(freqs_hz[i] < 0.5 * fs) || !std::isfinite(freqs_hz[i]))
            return CWT_EINVAL;
        if (!(n_cycles[i] > 0.0) || !std::isfinite(n_cycles[i])) return CWT_EINVAL;
    }
    int N = 0;
    cwt_status stt = cwt_fft_length(samples, CWT_PAD_POW2, &N);
    if (stt != CWT_OK) return stt;
    if (!scales_on_grid(CWT_WAVELET_MORLET, freqs_hz, n_cycles, n_freqs, 3.0, fs, N)) return CWT_EINVAL;
    const int nblk = (N + kNaThreads - 1) / kNaThreads;
    const size_t off_par = align256(kTwBytes);
    const size_t off_part = off_par + align256(sizeof(double) * 2 * (size_t)n_freqs);
    const size_t off_band = off_part + align256(sizeof(double) * (size_t)n_freqs * nblk);
    const size_t off_bank = off_band + align256(sizeof(int) * 2 * (size_t)n_freqs);
    const size_t off_spec = off_bank + align256(sizeof(float) * (size_t)n_freqs * N);
    const size_t need = off_spec + sizeof(float2) * (size_t)channels * N;
    if (need > kScratchBytes || (long long)channels * n_freqs > (1ll << 30)) return CWT_EINVAL;

    // ---- device side ----
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CWT_ECUDA;
    if (!na_dev_ptr(d_signal, dev) || (d_complex && !na_dev_ptr(d_complex, dev)) ||
        (d_power && !na_dev_ptr(d_power, dev)) || (d_phase && !na_dev_ptr(d_phase, dev)))
        return CWT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    char *base = nullptr;
    cudaError_t e = na_setup(dev, st, &base);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + off_par, freqs_hz, sizeof(double) * n_freqs,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + off_par + sizeof(double) * n_freqs, n_cycles,
                            sizeof(double) * n_freqs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        float2 *oc = (float2 *)d_complex;
        const int S = n_freqs;
        switch (ilog2c(N)) {
#define CWT_NA_CASE(L)                                                                             \
    case L:                                                                                        \
        e = na_run<1 << L>(d_signal, channels, samples, S, base, off_par, off_part, off_band,     \
                           off_bank, off_spec, fs, oc, d_power, d_phase, st);                      \
        break;
            CWT_NA_CASE(5) CWT_NA_CASE(6) CWT_NA_CASE(7) CWT_NA_CASE(8) CWT_NA_CASE(9)
            CWT_NA_CASE(10) CWT_NA_CASE(11) CWT_NA_CASE(12) CWT_NA_CASE(13) CWT_NA_CASE(14)
#undef CWT_NA_CASE
            default: return CWT_EUNSUPPORTED;
        }
    }
    if (e == cudaErrorMemoryAllocation) return CWT_ENOMEM;
#ifdef CWT_BOUNDS_CHECK
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && check_collect(nullptr)) return CWT_EDEVICE;
#endif
    return e == cudaSuccess ? CWT_OK : CWT_ECUDA;
}
