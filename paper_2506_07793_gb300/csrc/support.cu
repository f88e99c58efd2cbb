// support.cu -- the time support of a scale's wavelet, which sets the padding
// of linear ("same"-mode) edges (Section "Fourier transformed formula": the
// FFT gives a cyclic convolution, equal to the simple one once no wavelet
// wraps around).  Host code only; it runs at plan creation.
//
// The support radius is the time beyond which the wavelet's envelope stays
// below 1e-9 of its peak.  Morlet and Gabor (Eq. 3, Eq. 4) have the Gaussian
// envelope exp(-t^2 / (2 a^2)), a = n_cycles / (2 pi F): 1e-9 at
// a sqrt(2 ln 1e9) = 6.44 a, taken as 6.5 a.  The generalized Morse wavelet
// (Eq. 5) has no closed form in time; its spectrum depends on nu / F only,
// so psi_F(t) = F psi_1(F t), and the radius is R_1 / F with R_1 that of
// F = 1 Hz.  R_1 is measured: the spectrum sampled at M points of a band
// fs_ref that holds all of it, one inverse FFT (FP64) -- the wavelet
// periodised over M / fs_ref seconds -- and the last sample above 1e-9 of the
// peak on either side of t = 0, accepted once it lies within a quarter of
// the period (the periodic replicas then add nothing above the floor), else
// M doubles.
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace cwtk {

namespace {

constexpr double kEnvelopeFloor = 1e-9;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// In-place radix-2 FFT, a[k] <- sum_m a[m] exp(sign 2 pi i k m / M), M a
// power of two (iterative Cooley-Tukey, bit-reversed input order).
void fft_pow2(std::vector<std::complex<double>> &a, int sign) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = sign * kTwoPi / (double)len;
        for (size_t k = 0; k < len / 2; ++k) {
            const std::complex<double> w(std::cos(ang * (double)k), std::sin(ang * (double)k));
            for (size_t i = 0; i < n; i += len) {
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

// Eq. 5 with U(nu) at F = 1 Hz, up to its constant: (w_p nu)^beta exp(-(w_p nu)^gamma),
// w_p = (beta / gamma)^(1 / gamma) (the peak at nu = 1).
double gmw_shape(double nu, double beta, double gamma, double wp) {
    if (!(nu > 0.0)) return 0.0;
    const double w = wp * nu;
    return std::exp(beta * std::log(w) - std::pow(w, gamma) - (beta / gamma) * (std::log(beta / gamma) - 1.0));
}

// R_1 of the GMW (seconds at F = 1 Hz), or -1 when it exceeds max_seconds.
double gmw_radius_1hz(double beta, double gamma, double max_seconds) {
    const double wp = std::pow(beta / gamma, 1.0 / gamma);
    // the band: past the peak the shape falls below 1e-20 of it by nu_hi
    double nu_hi = 1.0;
    while (gmw_shape(nu_hi, beta, gamma, wp) > 1e-20) nu_hi *= 1.25;
    const double fs_ref = std::max(64.0, 4.0 * nu_hi);
    for (int M = 4096; M <= (1 << 21); M *= 2) {
        std::vector<std::complex<double>> a((size_t)M);
        for (int k = 1; k < M / 2; ++k) a[(size_t)k] = gmw_shape(k * fs_ref / M, beta, gamma, wp);
        fft_pow2(a, +1);
        double peak = 0.0;
        for (const auto &v : a) peak = std::max(peak, std::abs(v));
        const double floor = kEnvelopeFloor * peak;
        int r = 0;
        for (int m = 0; m < M / 2; ++m) {
            if (std::abs(a[(size_t)m]) > floor) r = std::max(r, m);
            if (m > 0 && std::abs(a[(size_t)(M - m)]) > floor) r = std::max(r, m);
        }
        if (r + 1 < M / 4) return (r + 1) / fs_ref;
        if (M / fs_ref > 4.0 * max_seconds) break;
    }
    return -1.0;
}

std::mutex g_support_mu;
std::map<std::pair<double, double>, double> g_gmw_r1;  // (beta, gamma) -> R_1

}  // namespace

int support_radius(int wavelet, double F, double sig, double gamma, double fs) {
    if (wavelet != CWT_WAVELET_GMW) {
        const double a = sig / (kTwoPi * F);
        const double R = std::ceil(6.5 * a * fs);
        return R <= (double)kMaxClusterFft ? (int)R : -1;
    }
    const double max_seconds = (double)kMaxClusterFft * F / fs;  // R_1 past this cannot fit
    double r1 = -1.0;
    {
        std::lock_guard<std::mutex> lock(g_support_mu);
        auto it = g_gmw_r1.find({sig, gamma});
        if (it != g_gmw_r1.end()) {
            r1 = it->second;
        } else {
            r1 = gmw_radius_1hz(sig, gamma, max_seconds);
            if (r1 >= 0.0) g_gmw_r1[{sig, gamma}] = r1;  // successes only: a bound depends on F / fs
        }
    }
    if (r1 < 0.0) return -1;
    const double R = std::ceil(r1 * fs / F);
    return R <= (double)kMaxClusterFft ? (int)R : -1;
}

}  // namespace cwtk

extern "C" cwt_status cwt_support_radius(int wavelet, double freq_hz, double n_cycles, double gmw_gamma, double fs,
                                         int *radius) {
    if (!radius || !(fs > 0.0) || !(freq_hz > 0.0) || !(freq_hz < 0.5 * fs) || !(n_cycles > 0.0) ||
        !std::isfinite(n_cycles))
        return CWT_EINVAL;
    if (wavelet != CWT_WAVELET_MORLET && wavelet != CWT_WAVELET_GABOR && wavelet != CWT_WAVELET_GMW)
        return CWT_EINVAL;
    if (wavelet == CWT_WAVELET_GMW && !(gmw_gamma > 0.0 && gmw_gamma <= 64.0)) return CWT_EINVAL;
    const int R = cwtk::support_radius(wavelet, freq_hz, n_cycles, gmw_gamma, fs);
    if (R < 0) return CWT_EUNSUPPORTED;
    *radius = R;
    return CWT_OK;
}
