"""Pins for the FP64 oracle: each test ties it to something other than itself.

The checks come from the paper's own statements and from mathematics:
  * the cyclic convolution theorem (Eq. 1 / Eq. 2), evaluated with a library
    FFT, and a brute-force DFT on tiny inputs;
  * the closed-form Morlet spectrum of Eq. 3 (and Gabor, Eq. 4), whose
    Poisson-summed samples must equal the DFT of the oracle's time-domain,
    periodised wavelet;
  * admissibility (zero mean) of the Morlet wavelet (the kappa term of Eq. 3);
  * the CWT of a pure sinusoid in closed form, linearity, shift equivariance;
  * decimation as plain subsampling, and agreement with a library linear
    convolution where the wavelet fits inside the zero padding ("cyclic
    convolution approximates simple convolution, except around the edge").
Each is chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle

PI = np.pi


def morlet_closed_form(freq, sigma, fs, N, kappa_on=True):
    """Eq. 3 in Hz: G(nu) = exp(-sigma^2 (nu/F - 1)^2 / 2) - kappa exp(-sigma^2 (nu/F)^2 / 2),
    sampled on the N DFT bins and summed over all aliases q (Poisson summation)."""
    kappa = np.exp(-0.5 * sigma * sigma) if kappa_on else 0.0
    k = np.arange(N)
    reach = 40.0 * freq / sigma + freq
    qmax = int(np.ceil(reach / fs)) + 2
    P = np.zeros(N)
    for q in range(-qmax, qmax + 1):
        nu = (k / N + q) * fs
        P += np.exp(-0.5 * sigma**2 * (nu / freq - 1.0) ** 2) - kappa * np.exp(-0.5 * sigma**2 * (nu / freq) ** 2)
    return P


CASES = [
    # (F, sigma, fs, N)
    (10.0, 7.0, 500.0, 512),      # typical
    (1.0, 3.0, 1000.0, 1024),     # small sigma: kappa = e^-4.5 is large
    (230.0, 3.0, 500.0, 256),     # near Nyquist: aliasing matters
    (2.0, 7.0, 64.0, 64),         # wavelet much longer than N: many replicas
    (40.0, 10.0, 250.0, 2048),
]


@pytest.mark.parametrize("F,sigma,fs,N", CASES)
def test_spectrum_matches_eq3_closed_form(F, sigma, fs, N):
    """DFT of the time-domain periodised wavelet == Poisson-summed Eq. 3."""
    p = oracle.periodised_wavelet(F, sigma, fs, N)
    P = np.fft.fft(p)
    G = morlet_closed_form(F, sigma, fs, N)
    # absolute constant of the Gaussian transform: int exp(-t^2/2a^2) e^{-2pi i nu t} dt = a sqrt(2 pi) ...
    a = sigma / (2 * PI * F)
    expected = fs * a * np.sqrt(2 * PI) * G
    scale = np.abs(expected).max()
    assert np.abs(P - expected).max() <= 1e-11 * scale
    # and after unit-energy normalisation
    w = oracle.wavelet(F, sigma, fs, N)
    W = np.fft.fft(w)
    Gn = G / np.sqrt(np.sum(G * G) / N)
    assert np.abs(W - Gn).max() <= 1e-11 * np.abs(Gn).max()


@pytest.mark.parametrize("F,sigma,fs,N", CASES[:3])
def test_gabor_spectrum_matches_eq4(F, sigma, fs, N):
    p = oracle.periodised_wavelet(F, sigma, fs, N, wavelet="gabor")
    G = morlet_closed_form(F, sigma, fs, N, kappa_on=False)
    a = sigma / (2 * PI * F)
    expected = fs * a * np.sqrt(2 * PI) * G
    assert np.abs(np.fft.fft(p) - expected).max() <= 1e-11 * np.abs(expected).max()


@pytest.mark.parametrize("F,sigma,fs,N", CASES)
def test_admissibility_zero_mean(F, sigma, fs, N):
    """Morlet's kappa term makes the continuous spectrum vanish at 0; the
    discrete mean equals the alias sum of G at multiples of fs (closed form)."""
    p = oracle.periodised_wavelet(F, sigma, fs, N)
    a = sigma / (2 * PI * F)
    kappa = np.exp(-0.5 * sigma * sigma)
    alias = 0.0
    for q in range(-50, 51):
        if q == 0:
            continue
        nu = q * fs
        alias += np.exp(-0.5 * sigma**2 * (nu / F - 1) ** 2) - kappa * np.exp(-0.5 * sigma**2 * (nu / F) ** 2)
    expected = fs * a * np.sqrt(2 * PI) * alias
    scale = fs * a * np.sqrt(2 * PI)
    assert abs(p.sum() - expected) <= 1e-11 * scale
    # the Gabor wavelet (kappa = 0) is not zero-mean: its mean is the sampled
    # Gaussian at nu = 0, exp(-sigma^2/2) (times the same constant).
    pg = oracle.periodised_wavelet(F, sigma, fs, N, wavelet="gabor")
    g0 = fs * a * np.sqrt(2 * PI) * (np.exp(-0.5 * sigma**2) + sum(
        np.exp(-0.5 * sigma**2 * (q * fs / F - 1) ** 2) for q in range(-50, 51) if q != 0))
    assert abs(pg.sum() - g0) <= 1e-11 * scale


@pytest.mark.parametrize("F,sigma,fs,N", CASES)
def test_unit_energy_and_hermitian_symmetry(F, sigma, fs, N):
    w = oracle.wavelet(F, sigma, fs, N)
    assert abs(np.sum(np.abs(w) ** 2) - 1.0) < 1e-13
    # psi(-tau) = conj(psi(tau)) => w[-m mod N] = conj(w[m]) => real spectrum
    mirrored = w[(-np.arange(N)) % N]
    assert np.abs(mirrored - np.conj(w)).max() < 1e-15 * 10
    assert np.abs(np.fft.fft(w).imag).max() < 1e-12 * np.abs(np.fft.fft(w)).max()


def test_peak_at_carrier_frequency():
    """F is the carrier: for sigma = 7 the spectral peak lies at bin F N / fs."""
    for F in (5.0, 12.5, 40.0):
        N, fs = 1024, 256.0
        W = np.fft.fft(oracle.wavelet(F, 7.0, fs, N)).real
        assert abs(int(np.argmax(W)) - F * N / fs) <= 1


def test_brute_force_dft_matches_library():
    rng = np.random.default_rng(11)
    for N in (1, 2, 3, 8, 15, 32):
        z = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        assert np.allclose(oracle.dft(z, -1), np.fft.fft(z), atol=1e-12)
        assert np.allclose(oracle.dft(z, +1), np.fft.ifft(z) * N, atol=1e-12)


@pytest.mark.parametrize("N,n", [(8, 8), (16, 11), (32, 20), (32, 1)])
def test_convolution_theorem_tiny(N, n):
    """Direct cyclic convolution == IDFT(DFT(x_pad) * DFT(w)) (Eq. 1), by
    brute-force DFT and by the library FFT."""
    rng = np.random.default_rng(N * 100 + n)
    x = rng.standard_normal(n)
    F, sigma, fs = 3.0, 4.0, 16.0
    w = oracle.wavelet(F, sigma, fs, N)
    c = oracle.cwt(x, N, fs, [F], [sigma])[0, 0]
    xp = np.zeros(N)
    xp[:n] = x
    ref_lib = np.fft.ifft(np.fft.fft(xp) * np.fft.fft(w))[:n]
    ref_bf = oracle.dft(oracle.dft(xp, -1) * oracle.dft(w, -1), +1)[:n] / N
    assert np.abs(c - ref_lib).max() < 1e-13
    assert np.abs(c - ref_bf).max() < 1e-12


def test_impulse_response():
    N, n, m0 = 64, 50, 7
    x = np.zeros(n)
    x[m0] = 1.0
    F, sigma, fs = 8.0, 5.0, 64.0
    w = oracle.wavelet(F, sigma, fs, N)
    c = oracle.cwt(x, N, fs, [F], [sigma])[0, 0]
    t = np.arange(n)
    assert np.array_equal(c, w[(t - m0) % N])


def test_sinusoid_closed_form():
    """x = A cos(2 pi k0 m / N + phi) with n = N:
    c[t] = A/2 (W[k0] e^{i(2 pi k0 t/N + phi)} + W[N-k0] e^{-i(...)}), W = DFT(w)."""
    N, fs = 1024, 256.0
    k0 = 40
    F = k0 * fs / N
    A, phi = 17.0, 0.3
    m = np.arange(N)
    x = A * np.cos(2 * PI * k0 * m / N + phi)
    c = oracle.cwt(x, N, fs, [F], [7.0])[0, 0]
    W = np.fft.fft(oracle.wavelet(F, 7.0, fs, N))
    arg = 2 * PI * k0 * m / N + phi
    expected = 0.5 * A * (W[k0] * np.exp(1j * arg) + W[N - k0] * np.exp(-1j * arg))
    assert np.abs(c - expected).max() < 1e-11 * A
    # at its own scale the magnitude is A/2 |W[k0]| up to the negative-frequency ripple
    mag = np.abs(c)
    assert mag.max() <= 0.5 * A * (abs(W[k0]) + abs(W[N - k0])) * (1 + 1e-12)
    assert mag.min() >= 0.5 * A * (abs(W[k0]) - abs(W[N - k0])) * (1 - 1e-12)


def test_linearity():
    rng = np.random.default_rng(5)
    n, N, fs = 300, 512, 250.0
    x, y = rng.standard_normal((2, n))
    freqs, cyc = [4.0, 11.0, 60.0], [3.0, 7.0, 9.0]
    cx = oracle.cwt(x, N, fs, freqs, cyc)
    cy = oracle.cwt(y, N, fs, freqs, cyc)
    cz = oracle.cwt(2.5 * x - 0.75 * y, N, fs, freqs, cyc)
    assert np.abs(cz - (2.5 * cx - 0.75 * cy)).max() < 1e-12 * np.abs(cz).max()


def test_shift_equivariance():
    rng = np.random.default_rng(6)
    N = 256
    x = rng.standard_normal(N)
    s = 37
    c = oracle.cwt(x, N, 128.0, [9.0], [6.0])[0, 0]
    cs = oracle.cwt(np.roll(x, s), N, 128.0, [9.0], [6.0])[0, 0]
    assert np.abs(cs - np.roll(c, s)).max() < 1e-12 * np.abs(c).max()


def test_decimation_is_subsampling():
    rng = np.random.default_rng(7)
    n, N = 203, 256
    x = rng.standard_normal((2, n))
    full = oracle.cwt(x, N, 200.0, [5.0, 30.0], [5.0, 7.0])
    for d in (2, 3, 4, 7):
        dec = oracle.cwt(x, N, 200.0, [5.0, 30.0], [5.0, 7.0], decimation=d)
        assert np.array_equal(dec, full[..., ::d])


def test_interior_equals_linear_convolution():
    """With padding wider than the wavelet's support, the cyclic result equals
    a plain linear convolution with the (unperiodised) sampled wavelet."""
    rng = np.random.default_rng(8)
    fs, F, sigma = 200.0, 20.0, 7.0
    n = 300
    a = sigma / (2 * PI * F)
    R = int(np.ceil(40 * a * fs))          # support radius in samples (envelope == 0 beyond)
    N = 1
    while N < n + R + 1:
        N *= 2
    x = rng.standard_normal(n)
    c = oracle.cwt(x, N, fs, [F], [sigma])[0, 0]
    tau = np.arange(-R, R + 1) / fs
    kappa = np.exp(-0.5 * sigma**2)
    psi = np.exp(-tau**2 / (2 * a * a)) * (np.exp(2j * PI * F * tau) - kappa)
    psi /= np.sqrt(np.sum(np.abs(oracle.periodised_wavelet(F, sigma, fs, N)) ** 2))
    lin = np.convolve(x, psi)[R:R + n]
    assert np.abs(c - lin).max() < 1e-12 * np.abs(c).max()


def test_row_subset_and_threads_consistent():
    rng = np.random.default_rng(9)
    x = rng.standard_normal((3, 120))
    freqs, cyc = [2.0, 10.0, 33.0], [3.0, 7.0, 10.0]
    full = oracle.cwt(x, 128, 100.0, freqs, cyc, threads=1)
    rows = [(2, 1), (0, 2), (1, 0)]
    sub = oracle.cwt_rows(x, 128, 100.0, freqs, cyc, rows, threads=3)
    for i, (c, s) in enumerate(rows):
        assert np.array_equal(sub[i], full[c, s])
    assert np.array_equal(oracle.cwt(x, 128, 100.0, freqs, cyc, threads=4), full)


def test_power_and_phase_definitions():
    c = np.array([3 + 4j, -1 - 0j, -1 + 1e-300j, 0j, -2j])
    assert np.array_equal(oracle.power(c), np.abs(c) ** 2)
    ph = oracle.phase(c)
    assert np.all(ph <= PI) and np.all(ph > -PI - 1e-15)
    assert np.allclose(np.exp(1j * ph[[0, 1, 4]]), c[[0, 1, 4]] / np.abs(c[[0, 1, 4]]))


def test_bad_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.wavelet(-1.0, 7.0, 100.0, 64)
    with pytest.raises(ValueError):
        oracle.wavelet(10.0, 0.0, 100.0, 64)
    with pytest.raises(ValueError):
        oracle.cwt(np.zeros((1, 10)), 8, 100.0, [10.0], [7.0])  # N < n


def test_golden_fixture_regression():
    """tests/golden/oracle_tiny.txt was written by tests/golden/make_golden.py,
    which calls only oracle/.  It guards the oracle against silent changes."""
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny.txt")
    from tests.golden.make_golden import TINY, compute
    rows = np.loadtxt(path, comments="#")
    got = compute(**TINY)
    assert rows.shape == got.shape
    assert np.abs(rows - got).max() <= 1e-12 * np.abs(rows).max()


# Unresolved wavelets: the carrier lies below the first DFT bins of N, so the
# replicas of the periodised wavelet cancel almost completely (to 1e-11 .. 1e-20
# of their amplitude here).  The oracle then takes the spectral side of Poisson
# summation; the pin is the time-domain definition
# p[m] = sum_r psi((m + r N) / fs) evaluated in 60-digit arithmetic.
UNRESOLVED = [
    # (kind, F, sigma, fs, N)
    ("morlet", 7.8, 7.0, 500.0, 32),    # 0.5 bin: first bin at 2 F
    ("morlet", 1.0, 7.0, 125.0, 64),    # 0.51 bin (the 1 Hz scale of a 2048-point window at 4 kHz)
    ("gabor", 5.0, 7.0, 500.0, 32),     # Gabor, 0.32 bin: no zero-mean term, DC bin dominates
    ("morlet", 3.0, 12.0, 250.0, 64),   # 0.77 bin, large sigma
    ("morlet", 6.0, 5.0, 500.0, 32),    # 0.38 bin, smaller sigma
]


def _mp_periodised(kind, F, sigma, fs, N, dps=60):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = dps
    Fm, sg, fsm = mp.mpf(F), mp.mpf(sigma), mp.mpf(fs)
    a = sg / (2 * mp.pi * Fm)
    kappa = mp.e ** (-sg * sg / 2) if kind == "morlet" else mp.mpf(0)
    reach = int(mpmath.ceil(40 * a * fsm))  # envelope below e^-800 beyond
    out = np.zeros(N, np.complex128)
    for m in range(N):
        s = mp.mpc(0)
        r_lo = -((reach + m) // N) - 1
        r_hi = (reach - m) // N + 1
        for r in range(r_lo, r_hi + 1):
            tau = (m + r * N) / fsm
            env = mp.e ** (-(tau * tau) / (2 * a * a))
            s += env * (mp.expj(2 * mp.pi * Fm * tau) - kappa)
        out[m] = complex(s)
    return out


@pytest.mark.parametrize("kind,F,sigma,fs,N", UNRESOLVED)
def test_unresolved_wavelet_matches_high_precision_periodisation(kind, F, sigma, fs, N):
    """The oracle's periodised wavelet equals the 60-digit time-domain sum to
    1e-11 of its peak, and so does the unit-energy wavelet."""
    ref = _mp_periodised(kind, F, sigma, fs, N)
    p = oracle.periodised_wavelet(F, sigma, fs, N, wavelet=kind)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(p - ref).max() <= 1e-11 * scale
    w = oracle.wavelet(F, sigma, fs, N, wavelet=kind)
    wref = ref / np.sqrt(np.sum(np.abs(ref) ** 2))
    assert np.abs(w - wref).max() <= 1e-11


def test_unresolved_route_is_taken_and_resolved_route_kept():
    """Both sides of the switch: a wavelet half a bin below the first bin
    (replicas cancel to ~1e-11 of their amplitude) and a resolved one agree with the
    Poisson-summed closed form of Eq. 3 (the spectral side, computed here in
    numpy) to 1e-11 of the peak."""
    for F, sigma, fs, N in [(7.8, 7.0, 500.0, 32), (10.0, 7.0, 500.0, 512)]:
        p = oracle.periodised_wavelet(F, sigma, fs, N)
        a = sigma / (2 * PI * F)
        expected = fs * a * np.sqrt(2 * PI) * morlet_closed_form(F, sigma, fs, N)
        P = np.fft.fft(p)
        assert np.abs(P - expected).max() <= 1e-11 * np.abs(expected).max()


@pytest.mark.parametrize("F,sigma,fs,N", [(10.0, 7.0, 500.0, 4096), (3.0, 3.0, 250.0, 2048),
                                          (40.0, 10.0, 1000.0, 4096)])
def test_mne_normalisation_closed_form(F, sigma, fs, N):
    """MNE-python's convention (sum |w|^2 = 2) against the closed-form energy of
    a well-sampled Gaussian-windowed complex sinusoid with the zero-mean term:
    sum_m |psi(m / fs)|^2 = fs * a sqrt(pi) (1 + kappa^2 - 2 kappa exp(-sigma^2 / 4))
    (Riemann sum of the integral; aliasing and truncation are below 1e-12 for
    these cases), so w_mne = p * sqrt(2 / that)."""
    a = sigma / (2 * PI * F)
    kappa = np.exp(-0.5 * sigma**2)
    energy = fs * a * np.sqrt(PI) * (1 + kappa**2 - 2 * kappa * np.exp(-sigma**2 / 4))
    p = oracle.periodised_wavelet(F, sigma, fs, N)
    w = oracle.wavelet(F, sigma, fs, N, normalization="mne")
    assert np.abs(w - p * np.sqrt(2.0 / energy)).max() <= 1e-10 * np.abs(w).max()
    wu = oracle.wavelet(F, sigma, fs, N)
    assert np.abs(w - np.sqrt(2.0) * wu).max() <= 1e-13
    # and the coefficients scale by sqrt(2), power by 2
    x = np.random.default_rng(5).standard_normal((1, 300))
    cu = oracle.cwt(x, N, fs, [F], [sigma])
    cm = oracle.cwt(x, N, fs, [F], [sigma], normalization="mne")
    assert np.abs(cm - np.sqrt(2.0) * cu).max() <= 1e-12 * np.abs(cm).max()
