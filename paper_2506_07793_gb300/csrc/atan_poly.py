"""Coefficients of the odd polynomial atan(x) ~ x P(x^2) on [0, 1] used by
phase.cuh, by the Remez exchange algorithm (minimax absolute error in x).

    python atan_poly.py [degree_in_u]

prints the coefficients c_0..c_n of P(u) = sum c_i u^i and the maximum
absolute error of x P(x^2) against math.atan, in double and with float32
Horner evaluation.  Not used at build or run time; kept so that the
constants in phase.cuh can be regenerated and checked.
"""
import math
import sys

import numpy as np


def remez(n, iters=40, grid=200001):
    # minimise max_x |atan(x) - x Q(x^2)| over x in [0, 1]
    xs = np.linspace(0.0, 1.0, grid)
    # initial reference: Chebyshev extrema mapped to [0, 1]
    k = np.arange(n + 2)
    ref = 0.5 - 0.5 * np.cos(np.pi * k / (n + 1))
    for _ in range(iters):
        # unknowns c_0..c_n, E:  x_j Q(x_j^2) + (-1)^j E = atan(x_j)
        A = np.zeros((n + 2, n + 2))
        for j, x in enumerate(ref):
            A[j, :n + 1] = x * (x * x) ** np.arange(n + 1)
            A[j, n + 1] = (-1.0) ** j
        b = np.arctan(ref)
        sol = np.linalg.solve(A, b)
        c = sol[:n + 1]
        err = np.arctan(xs) - xs * np.polyval(c[::-1], xs * xs)
        # new reference: the n + 2 alternating extrema of err
        idx = [0]
        for i in range(1, grid - 1):
            if (err[i] - err[i - 1]) * (err[i + 1] - err[i]) <= 0:
                idx.append(i)
        idx.append(grid - 1)
        idx = np.array(sorted(set(idx)))
        # keep alternating signs, largest magnitude per sign run
        pts = []
        for i in idx:
            if pts and np.sign(err[i]) == np.sign(err[pts[-1]]):
                if abs(err[i]) > abs(err[pts[-1]]):
                    pts[-1] = i
            else:
                pts.append(i)
        while len(pts) > n + 2:
            # drop the smaller end
            if abs(err[pts[0]]) < abs(err[pts[-1]]):
                pts.pop(0)
            else:
                pts.pop()
        if len(pts) < n + 2:
            break
        ref = xs[pts]
    return c, np.abs(err).max()


def eval_f32(c, x):
    x = np.float32(x)
    u = x * x
    p = np.float32(c[-1])
    for ci in c[-2::-1]:
        p = np.float32(p * u + np.float32(ci))
    return np.float32(x * p)


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 7
    c, e = remez(n)
    xs = np.linspace(0.0, 1.0, 100001, dtype=np.float32)
    e32 = np.abs(np.array([eval_f32(c, x) for x in xs[::10]], dtype=np.float64)
                 - np.arctan(xs[::10].astype(np.float64))).max()
    for i, ci in enumerate(c):
        print(f"c{i} = {ci:.17g}")
    print(f"max |err| double {e:.3e}, float32 Horner {e32:.3e}")
