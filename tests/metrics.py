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


def paper_style_error(test, ref, interior=(0.2, 0.8), threshold_sd=1e-5):
    """Table 1's report: |test - ref| / SD(ref) over the interior of each row.

    The paper compares its coefficients with MNE-python's as the absolute
    difference divided by the standard deviation of the reference, over the
    middle of the recording, and counts points above 1e-5 SD (Section
    "Precision", Table 1).  Returns (max, mean, count above threshold) over
    the interior window [round(0.2 n), round(0.8 n)) for the real and the
    imaginary parts; SD is the population standard deviation of the
    reference's interior.  Pinned by tests/test_metrics.py on a hand-computed
    case.
    """
    n = ref.shape[-1]
    lo, hi = int(round(interior[0] * n)), int(round(interior[1] * n))
    out = {}
    for name, f in (("real", np.real), ("imag", np.imag)):
        r = f(ref)[..., lo:hi]
        t = f(test)[..., lo:hi]
        sd = np.std(r)
        diff = np.abs(t - r) / sd
        out[name] = (float(diff.max()), float(diff.mean()), int((diff > threshold_sd).sum()))
    return out
