"""Pins for the oracle's generalized Morse wavelet (Eq. 5, with the Heaviside
step U(omega) in place of the printed sign(omega)).

The GMW is defined by its spectrum, Psi(nu) = U(nu) alpha w^beta exp(-w^gamma)
with w = w_p nu / F.  The oracle turns it into the N-periodised sampled
wavelet through the alias-summed spectrum and an O(N^2) inverse DFT.  These
tests tie that to mathematics other than the oracle's own formula:
  * the normalisation constant alpha and the peak frequency w_p: the spectrum
    peaks at nu = F with value 2 (the convention of Lilly and Olhede);
  * analyticity: nothing at negative frequencies;
  * gamma = 1 (the Cauchy wavelet): the inverse Fourier transform is known in
    closed form, alpha Gamma(beta+1) / (c (1 - 2 pi i tau / c)^(beta+1)), so the
    periodised sampled closed form must equal the oracle's wavelet -- this
    checks the frequency mapping, the alias sum and the IDFT's sign;
  * any gamma: w[0] of the unit-energy wavelet is a ratio of the moments
    int w^beta exp(-w^gamma) dw = Gamma((beta+1)/gamma) / gamma and
    int w^(2 beta) exp(-2 w^gamma) dw, which checks where beta and gamma enter.
"""
from math import gamma as Gamma

import numpy as np
import pytest

import oracle

PI = np.pi
SHAPES = [(20.0, 3.0), (3.0, 1.0), (8.0, 2.0), (60.0, 3.0), (1.5, 0.7), (6.5, 1.5)]


@pytest.mark.parametrize("beta,gam", SHAPES)
def test_gmw_peak_is_two_at_F(beta, gam):
    F = 12.5
    assert abs(oracle.gmw_spectrum(F, F, beta, gam) - 2.0) < 1e-13
    grid = F * (1.0 + np.linspace(-0.2, 0.2, 4001))
    vals = np.array([oracle.gmw_spectrum(v, F, beta, gam) for v in grid])
    assert abs(grid[np.argmax(vals)] - F) <= F * 1e-4 + 1e-12
    assert vals.max() <= 2.0 + 1e-13


@pytest.mark.parametrize("beta,gam", SHAPES)
def test_gmw_is_analytic(beta, gam):
    for nu in (0.0, -1e-9, -3.0, -1e3):
        assert oracle.gmw_spectrum(nu, 10.0, beta, gam) == 0.0
    # a low-frequency scale: the DFT of the periodised wavelet vanishes on the
    # negative-frequency bins k > N/2 (up to rounding of the O(N^2) sums)
    N, fs = 256, 256.0
    W = np.fft.fft(oracle.wavelet(8.0, beta, fs, N, wavelet="gmw", gamma=gam))
    if beta >= 3.0:
        assert np.abs(W[N // 2 + 1:]).max() < 1e-12 * np.abs(W).max()
    # the spectrum is real and non-negative (Psi >= 0), so w[-m] = conj(w[m])
    assert np.abs(W.imag).max() < 1e-12 * np.abs(W).max()
    assert W.real.min() > -1e-12 * np.abs(W).max()


@pytest.mark.parametrize("beta,F,fs,N", [(6.5, 20.0, 256.0, 256), (12.0, 5.0, 128.0, 512),
                                         (30.0, 40.0, 500.0, 200),
                                         (3.0, 100.0, 256.0, 256)])  # broad, aliased past fs
def test_gmw_gamma_one_matches_cauchy_closed_form(beta, F, fs, N):
    """gamma = 1: psi(tau) = int_0^inf Psi(nu) e^{+2 pi i nu tau} dnu
    = (alpha / c) Gamma(beta + 1) (1 - 2 pi i tau / c)^-(beta+1), c = w_p / F = beta / F;
    the oracle's wavelet must equal its N-periodised samples (unit energy)."""
    c = beta / F
    m = np.arange(N)
    p = np.zeros(N, dtype=np.complex128)
    R = 400
    for r in range(-R, R + 1):
        tau = (m + r * N) / fs
        p += (1.0 - 2j * PI * tau / c) ** (-(beta + 1.0))
    p /= np.sqrt(np.sum(np.abs(p) ** 2))
    w = oracle.wavelet(F, beta, fs, N, wavelet="gmw", gamma=1.0)
    assert np.abs(w - p).max() < 1e-11


@pytest.mark.parametrize("beta,gam", [(20.0, 3.0), (4.0, 2.0), (8.0, 1.5), (3.0, 1.0)])
def test_gmw_moment_identity(beta, gam):
    """w[0] = sum_k P[k] / sqrt(N sum_k P[k]^2) for the unit-energy wavelet;
    with fine bins and no aliasing the sums are Riemann sums of
    int Psi = (F / w_p) alpha Gamma((beta+1)/gamma) / gamma and
    int Psi^2 = (F / w_p) alpha^2 Gamma((2 beta+1)/gamma) / (gamma 2^((2 beta+1)/gamma)),
    so w[0] = sqrt(F / (w_p fs)) I1 / sqrt(I2)."""
    F, fs, N = 16.0, 256.0, 4096
    wp = (beta / gam) ** (1.0 / gam)
    I1 = Gamma((beta + 1.0) / gam) / gam
    I2 = Gamma((2.0 * beta + 1.0) / gam) / (gam * 2.0 ** ((2.0 * beta + 1.0) / gam))
    expected = np.sqrt(F / (wp * fs)) * I1 / np.sqrt(I2)
    w = oracle.wavelet(F, beta, fs, N, wavelet="gmw", gamma=gam)
    assert abs(w[0].imag) < 1e-13
    assert abs(w[0].real - expected) < 1e-9 * expected


def test_gmw_unit_energy_and_bad_arguments():
    w = oracle.wavelet(10.0, 20.0, 200.0, 300, wavelet="gmw", gamma=3.0)
    assert abs(np.sum(np.abs(w) ** 2) - 1.0) < 1e-13
    with pytest.raises(ValueError):
        oracle.wavelet(10.0, 20.0, 200.0, 300, wavelet="gmw", gamma=0.0)
