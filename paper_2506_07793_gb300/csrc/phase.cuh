// phase.cuh -- the phase output of the CWT (Section "Precision": real part,
// imaginary part, phase and power of the result), atan2(Im c, Re c).
//
// Octant reduction (a standard construction): with a = min(|x|, |y|) /
// max(|x|, |y|) in [0, 1], atan(a) is approximated by a P(a^2), P the
// degree-7 polynomial that minimises the maximum absolute error on [0, 1]
// (Remez exchange; atan_poly.py regenerates the coefficients: 3.7e-8 rad in
// double, 1.3e-7 rad evaluated in FP32).  Then t -> pi/2 - t when |y| > |x|,
// t -> pi - t when x < 0, and the sign of y.  Result in [-pi, pi]; (0, 0)
// gives 0.  A short, branch-free sequence: it matters on workloads that write
// the phase of every coefficient.
#pragma once

namespace cwtk {

__device__ __forceinline__ float phase_atan2(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    const float u = a * a;
    float p = -0.0040545672131782756f;
    p = fmaf(p, u, 0.021862957873980654f);
    p = fmaf(p, u, -0.055912326767600447f);
    p = fmaf(p, u, 0.096421973278836032f);
    p = fmaf(p, u, -0.13908629549907653f);
    p = fmaf(p, u, 0.19946565651286613f);
    p = fmaf(p, u, -0.33329860784331006f);
    p = fmaf(p, u, 0.99999933557833987f);
    float t = a * p;
    if (ay > ax) t = 1.57079632679489661923f - t;
    if (x < 0.f) t = 3.14159265358979323846f - t;
    return copysignf(t, y);
}

}  // namespace cwtk
