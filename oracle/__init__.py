"""FP64 CPU oracle for the FFT-based Morlet CWT (arXiv 2506.07793).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this package.  The CUDA library never
calls it and shares no code with it.

The arithmetic lives in plain C (cwt_oracle.c, loaded through ctypes); this
module only marshals numpy arrays and derives power and phase from the complex
coefficients (Section "Precision": real part, imaginary part, phase and power
of the CWT result).  See cwt_oracle.c for the definition being computed:
the cyclic convolution of the zero-padded signal with the N-periodised,
unit-energy Morlet wavelet of Eq. 3, which is what Eq. 2 evaluates.

Parity pins live in tests/test_oracle_pins.py and tests/test_oracle_pins_gmw.py;
every function here is pinned.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_periodised_wavelet.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                  dp, dp]
        lib.oracle_periodised_wavelet.restype = ctypes.c_int
        lib.oracle_wavelet.argtypes = lib.oracle_periodised_wavelet.argtypes
        lib.oracle_wavelet.restype = ctypes.c_int
        lib.oracle_cwt_rows.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, ip, ip, ctypes.c_int, ctypes.c_double, dp, dp,
                                        ctypes.c_int]
        lib.oracle_wavelet_norm.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_double, dp, dp]
        lib.oracle_wavelet_norm.restype = ctypes.c_int
        lib.oracle_cwt_rows.restype = ctypes.c_int
        lib.oracle_gmw_spectrum.argtypes = [ctypes.c_double] * 4
        lib.oracle_gmw_spectrum.restype = ctypes.c_double
        lib.oracle_dft.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_dft.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


WAVELETS = {"morlet": 0, "gabor": 1, "gmw": 2}


def gmw_spectrum(nu, freq, beta, gamma):
    """Eq. 5 with the Heaviside step: the GMW spectrum at nu Hz, peak 2 at freq."""
    return _load().oracle_gmw_spectrum(float(nu), float(freq), float(beta), float(gamma))


def periodised_wavelet(freq, n_cycles, fs, N, wavelet="morlet", gamma=3.0):
    """p[m] = sum_r psi((m + rN)/fs), m in [0, N) -- before normalisation.

    For wavelet="gmw", n_cycles is beta and gamma is Eq. 5's gamma."""
    lib = _load()
    re = np.zeros(N)
    im = np.zeros(N)
    rc = lib.oracle_periodised_wavelet(WAVELETS[wavelet], float(freq), float(n_cycles),
                                       float(gamma), float(fs), int(N), _dp(re), _dp(im))
    if rc != 0:
        raise ValueError("oracle_periodised_wavelet: bad argument")
    return re + 1j * im


NORMS = {"unit": 1.0, "mne": 2.0}


def wavelet(freq, n_cycles, fs, N, wavelet="morlet", gamma=3.0, normalization="unit"):
    """N-periodised sampled wavelet of one scale (complex128) with unit energy,
    or sum |w|^2 = 2 for normalization="mne" (MNE-python's convention)."""
    lib = _load()
    re = np.zeros(N)
    im = np.zeros(N)
    rc = lib.oracle_wavelet_norm(WAVELETS[wavelet], float(freq), float(n_cycles), float(gamma),
                                 float(fs), int(N), NORMS[normalization], _dp(re), _dp(im))
    if rc != 0:
        raise ValueError("oracle_wavelet: bad argument")
    return re + 1j * im


def cwt_rows(x, N, fs, freqs, n_cycles, rows, decimation=1, wavelet="morlet", threads=None,
             gamma=3.0, normalization="unit"):
    """Complex CWT coefficients of the (channel, scale) pairs in `rows`.

    x: [C][n] real signal.  Returns complex128 [len(rows)][ceil(n/d)].
    For wavelet="gmw", n_cycles holds beta per scale and gamma is shared.
    """
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if x.ndim == 1:
        x = x[None, :]
    C, n = x.shape
    freqs = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
    n_cycles = np.ascontiguousarray(np.broadcast_to(np.asarray(n_cycles, dtype=np.float64),
                                                    freqs.shape))
    rows = np.asarray(rows, dtype=np.int64).reshape(-1, 2)
    rc_ = np.ascontiguousarray(rows[:, 0].astype(np.int32))
    rs_ = np.ascontiguousarray(rows[:, 1].astype(np.int32))
    d = int(decimation)
    n_out = (n + d - 1) // d
    out_re = np.zeros((len(rows), n_out))
    out_im = np.zeros((len(rows), n_out))
    if threads is None:
        threads = os.cpu_count() or 1
    rc = lib.oracle_cwt_rows(_dp(x), C, n, int(N), float(fs), _dp(freqs), _dp(n_cycles),
                             len(freqs), WAVELETS[wavelet], float(gamma), d, _ip(rc_), _ip(rs_),
                             len(rows), NORMS[normalization],
                             _dp(out_re), _dp(out_im), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_cwt_rows failed ({rc})")
    return out_re + 1j * out_im


def cwt(x, N, fs, freqs, n_cycles, decimation=1, wavelet="morlet", threads=None, gamma=3.0,
        normalization="unit"):
    """Complex CWT of every row: complex128 [C][S][ceil(n/d)]."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    C = x.shape[0]
    S = len(np.atleast_1d(freqs))
    rows = [(c, s) for c in range(C) for s in range(S)]
    out = cwt_rows(x, N, fs, freqs, n_cycles, rows, decimation, wavelet, threads, gamma,
                   normalization)
    return out.reshape(C, S, -1)


def power(c):
    """|c|^2 (Section "Precision": power of the CWT result)."""
    return c.real * c.real + c.imag * c.imag


def phase(c):
    """atan2(Im c, Re c) in (-pi, pi] (Section "Precision": phase part)."""
    return np.arctan2(c.imag, c.real)


def dft(z, sign=-1):
    """Brute-force O(N^2) DFT (no 1/N), for tiny-input pins only."""
    lib = _load()
    z = np.asarray(z, dtype=np.complex128)
    re = np.ascontiguousarray(z.real)
    im = np.ascontiguousarray(z.imag)
    ore = np.zeros(len(z))
    oim = np.zeros(len(z))
    if lib.oracle_dft(_dp(re), _dp(im), len(z), int(sign), _dp(ore), _dp(oim)) != 0:
        raise ValueError("oracle_dft: bad argument")
    return ore + 1j * oim
