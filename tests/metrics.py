"""Error metrics shared by the parity tests and the benchmark's checks.

Per (channel, scale) row: relative error on power normalised by its maximum,
taken row by row (stricter than a global maximum):
  power:   max_t |P_gpu - P_ref| / max_t P_ref
  complex: max_t |c_gpu - c_ref| / max_t |c_ref|
  phase:   max_t |e^{i phi_gpu} - e^{i phi_ref}| * |c_ref[t]| / max_t |c_ref|
(phase is weighted by magnitude because it is ill-conditioned where |c| -> 0).
"""
import numpy as np

FP32_TOL = 1e-5   # FP32 paths
TC_TOL = 2e-3     # reduced-precision (tensor-core) paths


def row_max(a):
    m = np.max(a, axis=-1)
    return np.where(m > 0, m, 1.0)


def power_err(p_gpu, c_ref):
    p_ref = c_ref.real ** 2 + c_ref.imag ** 2
    return np.max(np.abs(np.asarray(p_gpu, np.float64) - p_ref), axis=-1) / row_max(p_ref)


def complex_err(c_gpu, c_ref):
    return np.max(np.abs(np.asarray(c_gpu, np.complex128) - c_ref), axis=-1) / row_max(np.abs(c_ref))


def phase_err(ph_gpu, c_ref):
    mag = np.abs(c_ref)
    d = np.abs(np.exp(1j * np.asarray(ph_gpu, np.float64)) - np.exp(1j * np.angle(c_ref)))
    return np.max(d * mag, axis=-1) / row_max(mag)
