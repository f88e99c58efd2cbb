"""The phase output's atan2 (csrc/phase.cuh): octant reduction plus a minimax
polynomial for atan on [0, 1].  Evaluated here in float32 with the constants
read from the header, against numpy's float64 arctan2: the error bound the GPU
kernels rely on (the GPU parity tests then check the kernels' phase against
the oracle)."""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2506_07793_gb300", "csrc", "phase.cuh")


def coefficients():
    text = open(HDR).read()
    body = text[text.index("phase_atan2"):]
    c = [float(v) for v in re.findall(r"(-?\d\.\d+)f", body.split("float t =")[0])]
    return c  # highest degree first, as in the Horner chain


def phase_f32(y, x):
    f = np.float32
    c = [f(v) for v in coefficients()]
    y = np.asarray(y, f)
    x = np.asarray(x, f)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(invalid="ignore", divide="ignore"):
        a = np.where(mx > 0, mn / mx, f(0)).astype(f)
    u = (a * a).astype(f)
    p = np.full_like(u, c[0])
    for ci in c[1:]:
        p = (p * u + ci).astype(f)
    t = (a * p).astype(f)
    t = np.where(ay > ax, f(np.pi / 2) - t, t).astype(f)
    t = np.where(x < 0, f(np.pi) - t, t).astype(f)
    return np.copysign(t, y)


def test_eight_coefficients_parsed():
    assert len(coefficients()) == 8


def test_error_bound_all_octants():
    rng = np.random.default_rng(5)
    ang = rng.uniform(-np.pi, np.pi, 200000)
    r = np.exp(rng.uniform(-30, 30, ang.size))
    y, x = (r * np.sin(ang)).astype(np.float32), (r * np.cos(ang)).astype(np.float32)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    got = phase_f32(y, x).astype(np.float64)
    d = np.abs(np.angle(np.exp(1j * (got - ref))))
    assert d.max() < 5e-7


def test_axes_and_zeros():
    y = np.array([0.0, 1.0, 0.0, -1.0, 0.0, 2.0, -3.0, 5.0, -5.0], np.float32)
    x = np.array([1.0, 0.0, -1.0, 0.0, 0.0, 2.0, -3.0, -5.0, 5.0], np.float32)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    got = phase_f32(y, x).astype(np.float64)
    assert np.abs(got - ref).max() < 5e-7
