// tables.cu -- FP64 generation of the twiddle table and the wavelet bank.
//
// Section "Optimizing performance" of arXiv 2506.07793 generates the
// Fourier-transformed wavelets in GPU memory before the data arrive, and
// Table 2 / the Discussion note that generation is cheap enough to redo when
// the analysis is reconfigured.  Here every table is computed in FP64 on the
// GPU and rounded once to FP32 for the hot kernels.
//
// Wavelet bank.  Eq. 3 gives the Morlet spectrum in the dimensionless
// frequency omega = sigma * nu / F (nu in Hz, F the carrier, sigma = n_cycles):
//     G(nu) = exp(-sigma^2 (nu/F - 1)^2 / 2) - kappa exp(-sigma^2 (nu/F)^2 / 2),
// kappa = exp(-sigma^2 / 2) (zero mean); kappa = 0 is the Gabor wavelet (Eq. 4).
// Sampling the spectrum on the N bins of a length-N DFT is exact for the
// N-periodised sampled wavelet once all aliases are summed (Poisson summation):
//     P[k] = sum_q G((k/N + q) fs).
// Each scale is normalised to unit discrete energy through Parseval,
// sum_m |w[m]|^2 = (1/N) sum_k |P[k]|^2, and the 1/N of the inverse FFT is
// folded in:  bank[k] = P[k] / sqrt(N * sum_k P[k]^2) (times sqrt(2) under
// MNE-python's convention, sum_m |w[m]|^2 = 2).
// The constant prefactors of Eq. 3 (c_sigma, pi^(-1/4)) cancel in the
// normalisation.  The spectrum is real because psi(-t) = conj(psi(t)).
//
// Generalized Morse wavelet (Eq. 5, Section "Fourier transformed formula"),
// with the Heaviside step U in place of the printed sign() so that the
// wavelet stays analytic:  G(nu) = U(nu) alpha w^beta exp(-w^gamma) with
// w = w_p nu / F, w_p = (beta/gamma)^(1/gamma) the peak of w^beta exp(-w^gamma)
// (so the spectrum peaks at nu = F) and alpha = 2 (e gamma / beta)^(beta/gamma)
// (peak value 2).  beta comes in the sigma slot, gamma per plan; the same
// alias sum and normalisation follow.
//
// Band.  Bins whose |P| is below kBandRelThreshold of the scale's peak are
// skipped by the hot kernel; the band is the signed-frequency interval
// [kmin, kmax] holding every bin above it (it wraps modulo N).
#include <cuda_runtime.h>

#include <mutex>

#include "fft_core.cuh"
#include "internal.h"

namespace cwtk {

namespace {

__global__ void twiddle_kernel(float2 *tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < kTwN) {
        double s, c;
        sincospi(2.0 * (double)m / (double)kTwN, &s, &c);
        tw[m] = make_float2((float)c, (float)s);
    }
}

constexpr int kBankThreads = 256;

// Eq. 3 / Eq. 4 evaluated at nu (Hz).
__device__ __forceinline__ double spectrum_g(double nu, double F, double sigma, double kappa) {
    const double u = nu / F;
    const double a = u - 1.0;
    double g = exp(-0.5 * sigma * sigma * a * a);
    if (kappa != 0.0) g -= kappa * exp(-0.5 * sigma * sigma * u * u);
    return g;
}

// Eq. 5 at nu (Hz) with U(nu); wp = w_p, la = ln(alpha).
__device__ __forceinline__ double spectrum_gmw(double nu, double F, double beta, double gamma,
                                               double wp, double la) {
    if (!(nu > 0.0)) return 0.0;
    const double w = wp * nu / F;
    return exp(la + beta * log(w) - pow(w, gamma));
}

// grid (ceil(N / 256), S): raw[s][k] = sum_q G((k/N + q) fs) and per-block
// partial sums of raw^2 (fixed-order tree, so the result is deterministic).
// kind: CWT_WAVELET_MORLET / _GABOR (sig = sigma) or _GMW (sig = beta).
__global__ void __launch_bounds__(kBankThreads)
bank_raw_kernel(int N, double fs, const double *__restrict__ F, const double *__restrict__ sig,
                int kind, double gamma, double *__restrict__ raw, double *__restrict__ partial) {
    __shared__ double red[kBankThreads];
    const int s = blockIdx.y;
    const int k = blockIdx.x * kBankThreads + threadIdx.x;
    double v = 0.0;
    if (k < N) {
        const double f = F[s], sg = sig[s];
        const double base = (double)k / (double)N;
        if (kind == CWT_WAVELET_GMW) {
            const double beta = sg;
            const double wp = pow(beta / gamma, 1.0 / gamma);
            const double la = log(2.0) + (beta / gamma) * (1.0 + log(gamma) - log(beta));
            // past the peak G decreases; G/2 < exp(-760) (zero in double) once
            // w^gamma - wp^gamma - beta ln(w / wp) > 760: fixed-point iteration
            // from the right of the peak
            const double wpg = pow(wp, gamma);
            double w = 2.0 * wp;
            for (int it = 0; it < 12; ++it) w = pow(wpg + 760.0 + beta * log(w / wp), 1.0 / gamma);
            const double nu_hi = f * w / wp;
            const double q_hi = floor(nu_hi / fs - base);
            for (double q = 0.0; q <= q_hi; q += 1.0) v += spectrum_gmw((base + q) * fs, f, beta, gamma, wp, la);
        } else {
            const double kappa = kind == CWT_WAVELET_GABOR ? 0.0 : exp(-0.5 * sg * sg);
            const double reach = 40.0 * f / sg;  // exp(-x) underflows past x ~ 745
            const double nu_lo = -reach, nu_hi = f + reach;
            const double q_lo = ceil(nu_lo / fs - base), q_hi = floor(nu_hi / fs - base);
            for (double q = q_lo; q <= q_hi; q += 1.0) v += spectrum_g((base + q) * fs, f, sg, kappa);
        }
        raw[(size_t)s * N + k] = v;
    }
    red[threadIdx.x] = v * v;
    __syncthreads();
    for (int w = kBankThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = red[0];
}

// One CTA per scale: normalise, round to FP32, find the band.
__global__ void __launch_bounds__(kBankThreads)
bank_finish_kernel(int N, int nblk, double norm2, const double *__restrict__ raw,
                   const double *__restrict__ partial, float *__restrict__ bank,
                   int *__restrict__ band) {
    __shared__ double sd[kBankThreads];
    __shared__ int smin[kBankThreads], smax[kBankThreads];
    const int s = blockIdx.x;
    const double *r = raw + (size_t)s * N;
    float *b = bank + (size_t)s * N;
    // energy: fixed-order sum of the partials
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int i = 0; i < nblk; ++i) e += partial[(size_t)s * nblk + i];
        sd[0] = e;
    }
    __syncthreads();
    const double energy = sd[0];
    // sum_m |w[m]|^2 = norm2: Parseval over the N bins, 1/N of the inverse FFT folded in
    const double scale = energy > 0.0 ? sqrt(norm2 / ((double)N * energy)) : 0.0;
    __syncthreads();
    double mx = 0.0;
    for (int k = threadIdx.x; k < N; k += kBankThreads) {
        const double v = r[k];
        b[k] = (float)(v * scale);
        mx = fmax(mx, fabs(v));
    }
    sd[threadIdx.x] = mx;
    __syncthreads();
    for (int w = kBankThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + w]);
        __syncthreads();
    }
    const double thr = sd[0] * kBandRelThreshold;
    int lo = N, hi = -N;
    for (int k = threadIdx.x; k < N; k += kBankThreads) {
        if (fabs(r[k]) > thr) {
            const int ks = k < N / 2 ? k : k - N;  // signed frequency bin
            lo = min(lo, ks);
            hi = max(hi, ks);
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int w = kBankThreads / 2; w > 0; w >>= 1) {
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

std::mutex g_tw_mutex;
const float2 *g_tw[64] = {};

}  // namespace

cudaError_t device_twiddles(const float2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_tw_mutex);
    if (!g_tw[dev]) {
        float2 *tw = nullptr;
        e = cwtk::dmalloc(&tw, sizeof(float2) * kTwN);
        if (e != cudaSuccess) return e;
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaFree(tw);
            return e;
        }
        twiddle_kernel<<<kTwN / 256, 256, 0, st>>>(tw);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        if (e != cudaSuccess) {
            cudaFree(tw);
            return e;
        }
        g_tw[dev] = tw;  // kept until process exit, shared by every plan on this device
    }
    *out = g_tw[dev];
    return cudaSuccess;
}

cudaError_t launch_bank(cwt_plan_s *p, cudaStream_t st) {
    return launch_bank_n(p, p->N, p->bank, p->band, st, &p->bank_ms);
}

cudaError_t launch_bank_n(const cwt_plan_s *p, int N, float *bank, int *band, cudaStream_t st,
                          double *ms_out) {
    const int S = p->S;
    const int nblk = (N + kBankThreads - 1) / kBankThreads;
    double *raw = nullptr, *partial = nullptr, *dF = nullptr, *dsig = nullptr;
    cudaError_t e = cwtk::dmalloc(&raw, sizeof(double) * (size_t)S * N);
    if (e == cudaSuccess) e = cwtk::dmalloc(&partial, sizeof(double) * (size_t)S * nblk);
    if (e == cudaSuccess) e = cwtk::dmalloc(&dF, sizeof(double) * S);
    if (e == cudaSuccess) e = cwtk::dmalloc(&dsig, sizeof(double) * S);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dF, p->freqs.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dsig, p->cycles.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = cudaEventRecord(t0, st);
    if (e == cudaSuccess) {
        bank_raw_kernel<<<dim3(nblk, S), kBankThreads, 0, st>>>(N, p->fs, dF, dsig, p->wavelet,
                                                                p->gmw_gamma, raw, partial);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        bank_finish_kernel<<<S, kBankThreads, 0, st>>>(N, nblk, p->norm2, raw, partial, bank, band);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && ms_out) *ms_out = ms;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(raw);
    cudaFree(partial);
    cudaFree(dF);
    cudaFree(dsig);
    return e;
}

}  // namespace cwtk
