// mixed_radix.cuh -- Stockham FFT for 2,3,5,7-smooth lengths N <= 16384 in one
// CTA (longer rows run it per residue class on a cluster, smooth_cluster.cuh).
//
// Section "Fast Fourier transform" of arXiv 2506.07793 pads each signal to the
// smallest length whose prime factors are 2, 3, 5 and 7 (the fftpack radices)
// rather than to a power of two.  This header runs such rows with the same
// structure as the power-of-two kernels of fft_core.cuh:
//
//  * N = R_0 R_1 ... R_{P-1} with every radix a 7-smooth number in [4, 32]
//    (a host-side cost model picks the factorisation and the order).  Pass p
//    (radix R, Ns = R_0 ... R_{p-1}) has N/R butterflies; butterfly b takes
//    the inputs b + r N/R, multiplies input r by w^r, w = exp(+-2 pi i k/(Ns R))
//    with k = b mod Ns, runs an R-point DFT and writes output r to
//    (b - k) R + k + r Ns (self-sorting, natural order after the last pass).
//  * A row has T threads; in pass p thread j runs the butterflies j + g T,
//    g < G_p = ceil(N / (R T)), holding all of its R G_p <= 32 values in
//    registers, so each pass is one read of the row's shared-memory
//    buffer, a barrier, and one write (a single buffer of N + N/16 float2).
//  * Several rows share a CTA when T is small (short signals).
//  * The first pass reads through a caller functor (global memory, fused
//    spectrum product); the last pass leaves the row in natural order in the
//    buffer, and the caller's epilogue streams it out with a rolled,
//    coalesced loop (fused reduction and stores).  When every first-pass
//    butterfly meets at most one nonzero input (a narrow band) its DFT is a
//    twiddle chain.
//  * Composite radices are nested Cooley-Tukey DFTs in registers whose
//    internal twiddles are compile-time constants; prime radices 3, 5, 7 use
//    the symmetric form X[k], X[R-k] = A_k +- B_k.
//  * b mod Ns uses a multiply-high by ceil(2^32 / Ns): for b < 2^14 and
//    Ns <= 2^13 the quotient is exact (division by invariant integers,
//    Granlund and Montgomery 1994).
//  * Pass twiddles w = exp(+-2 pi i k / (Ns R)) are entry k N/(Ns R) of a
//    per-length FP64-generated table of the N-th roots of unity; their powers
//    come from a short multiplication chain.
#pragma once


#include "fft_core.cuh"

namespace cwtk {

constexpr int kMrThreads = 512;   // largest CTA (the register budget of 32 values per thread)
constexpr int kMrPoints = 32;     // complex values per thread per pass
constexpr int kMrMaxPasses = 14;

struct MrPass {
    int R;          // radix
    int G;          // butterflies per thread, <= kMrPoints / R
    int Ns;         // product of the earlier radices
    unsigned mag;   // ceil(2^32 / Ns) (0 when Ns == 1)
    int tws;        // N / (Ns R): twiddle-table stride
};

struct MrSchedule {
    int N;           // row length
    int T;           // threads per row (rows per CTA are chosen per launch)
    int np;          // passes
    int fast;        // index of the inlined radix pair that runs it, or -1 (generic)
    int fixed;       // index of the fixed-length kernel that runs it, or -1
    int fixed_cl;    // as the local row of a cluster: index of its fixed-length kernel, or -1
    unsigned mag0;   // ceil(2^32 / (N / R_0)), for the sparse first pass
    MrPass p[kMrMaxPasses];
};

// ---- compile-time cos / sin (2 pi m / R): Taylor series after reduction to
// |x| <= pi/4 (octant symmetries with exact integer arithmetic) -------------
__host__ __device__ constexpr double ct_sin_red(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int i = 1; i < 14; ++i) {
        term *= -x2 / ((2.0 * i) * (2.0 * i + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos_red(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) {
        term *= -x2 / ((2.0 * i - 1.0) * (2.0 * i));
        sum += term;
    }
    return sum;
}
// cos and sin of phi = (pi/2) rem / R for 0 <= rem < R
__host__ __device__ constexpr double ct_cos_q(int rem, int R) {
    constexpr double kHalfPi = 1.57079632679489661923;
    return 2 * rem <= R ? ct_cos_red(kHalfPi * rem / R) : ct_sin_red(kHalfPi * (R - rem) / R);
}
__host__ __device__ constexpr double ct_sin_q(int rem, int R) {
    constexpr double kHalfPi = 1.57079632679489661923;
    return 2 * rem <= R ? ct_sin_red(kHalfPi * rem / R) : ct_cos_red(kHalfPi * (R - rem) / R);
}
__host__ __device__ constexpr double ct_cos2pi(int m, int R) {
    const int mm = ((m % R) + R) % R;
    const int q = (4 * mm) / R, rem = 4 * mm - q * R;
    const double c = ct_cos_q(rem, R), s = ct_sin_q(rem, R);
    return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
__host__ __device__ constexpr double ct_sin2pi(int m, int R) {
    const int mm = ((m % R) + R) % R;
    const int q = (4 * mm) / R, rem = 4 * mm - q * R;
    const double c = ct_cos_q(rem, R), s = ct_sin_q(rem, R);
    return q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
}

// a * exp(SIGN 2 pi i M / R), M a compile-time constant.
template <int R, int SIGN, int M>
__device__ __forceinline__ float2 rot_c(float2 a) {
    constexpr int m = ((M % R) + R) % R;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == R) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (4 * m == R) {
        return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (4 * m == 3 * R) {
        return SIGN > 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else {
        constexpr float c = (float)ct_cos2pi(m, R);
        constexpr float s = (float)(SIGN > 0 ? ct_sin2pi(m, R) : -ct_sin2pi(m, R));
        return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
    }
}

// Compile-time loop: f(int_c<I>{}) for I < N (int_c<I>::value == I).  The
// sequence types are the header's own, so that it needs no standard library
// header (the plan-time compiler, jit.cu, builds it without one).
template <int I>
struct int_c {
    static constexpr int value = I;
};
template <int... I>
struct int_seq {};
template <int N, int... I>
struct make_int_seq : make_int_seq<N - 1, N - 1, I...> {};
template <int... I>
struct make_int_seq<0, I...> {
    using type = int_seq<I...>;
};
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, int_seq<I...>) {
    (f(int_c<I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, typename make_int_seq<N>::type{});
}

// cos / sin (2 pi m / R) for the odd primes, m = 1..(R-1)/2.
__host__ __device__ constexpr float odd_cos(int R, int m) { return (float)ct_cos2pi(m, R); }
__host__ __device__ constexpr float odd_sin(int R, int m) { return (float)ct_sin2pi(m, R); }

template <int R, int SIGN>
__device__ __forceinline__ void dft_odd(float2 *v) {
    constexpr int H = (R - 1) / 2;
    float2 s[H], d[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        s[r - 1] = cadd(v[r], v[R - r]);
        d[r - 1] = csub(v[r], v[R - r]);
    }
    float2 out[R];
    out[0] = v[0];
#pragma unroll
    for (int r = 0; r < H; ++r) out[0] = cadd(out[0], s[r]);
    static_for<H>([&](auto kc) {
        constexpr int k = decltype(kc)::value + 1;
        float2 a = v[0], b = make_float2(0.f, 0.f);
        static_for<H>([&](auto rc) {
            constexpr int r = decltype(rc)::value + 1;
            constexpr int m = (r * k) % R;              // 1..R-1
            constexpr int mm = m <= H ? m : R - m;      // cos even, sin odd about R/2
            constexpr float c = odd_cos(R, mm);
            constexpr float sn = (m <= H ? 1.f : -1.f) * (SIGN > 0 ? 1.f : -1.f) * odd_sin(R, mm);
            a.x = fmaf(s[r - 1].x, c, a.x);
            a.y = fmaf(s[r - 1].y, c, a.y);
            b.x = fmaf(-d[r - 1].y, sn, b.x);           // i * d * sn
            b.y = fmaf(d[r - 1].x, sn, b.y);
        });
        out[k] = cadd(a, b);
        out[R - k] = csub(a, b);
    });
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = out[i];
}

__host__ __device__ constexpr bool is_pow2c(int r) { return r > 0 && (r & (r - 1)) == 0; }
__host__ __device__ constexpr int low_pow2(int r) { return r & (-r); }
__host__ __device__ constexpr int small_prime(int r) { return r % 3 == 0 ? 3 : r % 5 == 0 ? 5 : 7; }
// First factor of a composite radix: its power-of-two part, else its smallest prime.
__host__ __device__ constexpr int first_factor(int r) { return (r & 1) == 0 ? low_pow2(r) : small_prime(r); }

// X[k] = sum_n v[n] exp(SIGN 2 pi i k n / R), natural order, in registers.
template <int R, int SIGN>
__device__ __forceinline__ void dft_r(float2 *v);

__host__ __device__ constexpr int ct_gcd(int a, int b) { return b == 0 ? a : ct_gcd(b, a % b); }
// x with a x = 1 (mod m), for gcd(a, m) = 1 and m >= 2.
__host__ __device__ constexpr int ct_inv_mod(int a, int m) {
    int x = 1;
    while ((a * x) % m != 1) ++x;
    return x;
}

// R = R1 R2 with gcd(R1, R2) = 1: the prime-factor (Good-Thomas) algorithm,
// no twiddles between the two stages.  Input index n = (R2 n1 + R1 n2) mod R
// and output index k with k = k1 (mod R1), k = k2 (mod R2), i.e.
// k = (k1 R2 u2 + k2 R1 u1) mod R, u2 = R2^-1 mod R1, u1 = R1^-1 mod R2:
//   w_R^(n k) = w_R1^(n1 k1) w_R2^(n2 k2), so
//   X[k] = sum_n2 w_R2^(n2 k2) sum_n1 x[(R2 n1 + R1 n2) mod R] w_R1^(n1 k1).
template <int R, int SIGN, int R1, int R2>
__device__ __forceinline__ void dft_pfa(float2 *v) {
    constexpr int u2 = ct_inv_mod(R2 % R1, R1), u1 = ct_inv_mod(R1 % R2, R2);
    float2 t[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
        float2 a[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[(R2 * n1 + R1 * n2) % R];
        dft_r<R1, SIGN>(a);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) t[n2 * R1 + k1] = a[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 b[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) b[n2] = t[n2 * R1 + k1];
        dft_r<R2, SIGN>(b);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[(k1 * R2 * u2 + k2 * R1 * u1) % R] = b[k2];
    }
}

// R1, R2 sharing a factor (9, 25, 27): Cooley-Tukey, n = R2 n1 + n2, k = k1 + R1 k2:
//   X[k1 + R1 k2] = sum_n2 w_R2^(n2 k2) w_R^(n2 k1) sum_n1 x[R2 n1 + n2] w_R1^(n1 k1)
template <int R, int SIGN, int R1, int R2>
__device__ __forceinline__ void dft_ct(float2 *v) {
    float2 t[R];
    static_for<R2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        float2 a[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[R2 * n1 + n2];
        dft_r<R1, SIGN>(a);
        static_for<R1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            t[n2 * R1 + k1] = rot_c<R, SIGN, n2 * k1>(a[k1]);
        });
    });
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 b[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) b[n2] = t[n2 * R1 + k1];
        dft_r<R2, SIGN>(b);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
    }
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_composite(float2 *v) {
    constexpr int R1 = first_factor(R), R2 = R / R1;
    if constexpr (ct_gcd(R1, R2) == 1)
        dft_pfa<R, SIGN, R1, R2>(v);
    else
        dft_ct<R, SIGN, R1, R2>(v);
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_r(float2 *v) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (is_pow2c(R)) {
        dft<R, SIGN>(v);
    } else if constexpr (R == 3 || R == 5 || R == 7) {
        dft_odd<R, SIGN>(v);
    } else {
        dft_composite<R, SIGN>(v);
    }
}

// v[r] *= w1^r, r = 1..R-1: w1^1..w1^7 by a square-and-multiply chain, higher
// powers as w1^(8h) w1^(r mod 8).
template <int R>
__device__ __forceinline__ void mr_twiddle(float2 *v, float2 w1) {
    if constexpr (is_pow2c(R)) {
        twiddle_chain<R>(v, w1);
    } else {
        constexpr int LO = R < 8 ? R : 8;
        float2 wl[LO];
        wl[0] = make_float2(1.f, 0.f);
        wl[1] = w1;
#pragma unroll
        for (int r = 2; r < LO; ++r) wl[r] = (r & 1) ? cmul(wl[r - 1], w1) : cmul(wl[r >> 1], wl[r >> 1]);
#pragma unroll
        for (int r = 1; r < LO; ++r) v[r] = cmul(v[r], wl[r]);
        if constexpr (R > 8) {
            const float2 w8 = cmul(wl[4], wl[4]);
            float2 wh = w8;
#pragma unroll
            for (int h = 1; 8 * h < R; ++h) {
                v[8 * h] = cmul(v[8 * h], wh);
#pragma unroll
                for (int l = 1; l < 8; ++l)
                    if (8 * h + l < R) v[8 * h + l] = cmul(cmul(v[8 * h + l], wh), wl[l]);
                if (8 * (h + 1) < R) wh = cmul(wh, w8);
            }
        }
    }
}

// ---- passes -----------------------------------------------------------------
// Butterflies per thread and pass: at most 32 values.
template <int R>
__host__ __device__ constexpr int mr_gmax() {
    return kMrPoints / R >= 1 ? kMrPoints / R : 1;
}

// Butterfly b of pass (R, Ns): twiddle its inputs, DFT, and return k = b mod Ns
// and q = b / Ns.
template <int R, int SIGN>
__device__ __forceinline__ void mr_butterfly(float2 *v, const MrPass &ps, const float2 *__restrict__ twN,
                                             int b, int &q, int &k) {
    q = (int)__umulhi((unsigned)b, ps.mag);
    k = b - q * ps.Ns;
    float2 w1 = __ldg(&twN[k * ps.tws]);
    if (SIGN < 0) w1.y = -w1.y;
    mr_twiddle<R>(v, w1);
    dft_r<R, SIGN>(v);
}

// Linear addressing (LIN): the buffer index spad2(i) = i + i/16 is not
// linear in i, but spad2(x + 16 m) = spad2(x) + 17 m, so a run of accesses
// whose stride is a multiple of 16 is one padded base plus constant offsets.
// The fixed-length kernels (every stride a compile-time constant) take that
// form wherever it applies; with runtime strides the extra branches cost more
// than they save, and the runtime-schedule kernels keep the plain form.

// Pass 0 (Ns = 1): inputs from load(k), outputs to the row's buffer.  The
// dense and sparse forms hold no barrier: rows of one CTA (even of one warp)
// may take different forms, and mr_row places the barrier after either.
template <int R, int SIGN, bool LIN = false, typename Load>
__device__ __forceinline__ void mr_first_body(const MrPass &ps, float2 *__restrict__ sm, int N, int T,
                                              int j, bool active, const Load &load) {
    constexpr int GM = mr_gmax<R>();
    const int nb = N / R;
#pragma unroll
    for (int g = 0; g < GM; ++g) {
        const int b = j + g * T;
        if (g < ps.G && active && b < nb) {
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = load(b + r * nb);
            dft_r<R, SIGN>(v);
            if constexpr (LIN && R % 16 == 0) {
                float2 *dst = sm + spad2(b * R);
#pragma unroll
                for (int r = 0; r < R; ++r) *CWT_SMEM(&dst[spad2(r)]) = v[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) *CWT_SMEM(&sm[spad2(b * R + r)]) = v[r];
            }
        }
    }
}

// Pass 0 when each butterfly meets at most one nonzero input:
// first_nz(b, nb, mag0, r, x) gives its position r and value x; the R-point
// DFT is then x exp(SIGN 2 pi i r t / R), t < R.
template <int R, int SIGN, bool LIN = false, typename First>
__device__ __forceinline__ void mr_first_sparse_body(const MrPass &ps, float2 *__restrict__ sm,
                                                     const float2 *__restrict__ twN, int N, int T, int j,
                                                     bool active, unsigned mag0, const First &first_nz) {
    constexpr int GM = mr_gmax<R>();
    const int nb = N / R;
#pragma unroll
    for (int g = 0; g < GM; ++g) {
        const int b = j + g * T;
        if (g < ps.G && active && b < nb) {
            int r = 0;
            float2 x = make_float2(0.f, 0.f);
            const bool nz = first_nz(b, nb, mag0, r, x);
            float2 w = __ldg(&twN[r * nb]);  // exp(+2 pi i r / R)
            if (SIGN < 0) w.y = -w.y;
            if (!nz) x = make_float2(0.f, 0.f);
            float2 v[R];
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = x;
            mr_twiddle<R>(v, w);
            if constexpr (LIN && R % 16 == 0) {
                float2 *dst = sm + spad2(b * R);
#pragma unroll
                for (int t = 0; t < R; ++t) *CWT_SMEM(&dst[spad2(t)]) = v[t];
            } else {
#pragma unroll
                for (int t = 0; t < R; ++t) *CWT_SMEM(&sm[spad2(b * R + t)]) = v[t];
            }
        }
    }
}

// A middle pass: buffer -> registers, barrier, butterflies -> buffer.
template <int R, int SIGN, bool LIN = false>
__device__ __forceinline__ void mr_mid_body(const MrPass &ps, float2 *__restrict__ sm,
                                            const float2 *__restrict__ twN, int N, int T, int j, bool active) {
    constexpr int GM = mr_gmax<R>();
    const int nb = N / R;
    const bool lin_in = LIN && (nb & 15) == 0, lin_out = LIN && (ps.Ns & 15) == 0;
    const int nbp = nb + (nb >> 4), nsp = ps.Ns + (ps.Ns >> 4);
    float2 v[GM][R];
#pragma unroll
    for (int g = 0; g < GM; ++g) {
        const int b = j + g * T;
        if (g < ps.G && active && b < nb) {
            if (lin_in) {
                const float2 *src = sm + spad2(b);
#pragma unroll
                for (int r = 0; r < R; ++r) v[g][r] = *CWT_SMEM(&src[r * nbp]);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[g][r] = *CWT_SMEM(&sm[spad2(b + r * nb)]);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < GM; ++g) {
        const int b = j + g * T;
        if (g < ps.G && active && b < nb) {
            int q, k;
            mr_butterfly<R, SIGN>(v[g], ps, twN, b, q, k);
            const int base = q * ps.Ns * R + k;
            if (lin_out) {
                float2 *dst = sm + spad2(base);
#pragma unroll
                for (int r = 0; r < R; ++r) *CWT_SMEM(&dst[r * nsp]) = v[g][r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) *CWT_SMEM(&sm[spad2(base + r * ps.Ns)]) = v[g][r];
            }
        }
    }
    __syncthreads();
}

// Out-of-line forms of the passes: one register allocation per radix, for
// the generic kernels that dispatch over every radix (one function holding
// all of them inline spills and compiles for minutes).
template <int R, int SIGN, typename Load>
__device__ __noinline__ void mr_first(const MrPass ps, float2 *__restrict__ sm, int N, int T, int j,
                                      bool active, Load load) {
    mr_first_body<R, SIGN>(ps, sm, N, T, j, active, load);
}
template <int R, int SIGN, typename First>
__device__ __noinline__ void mr_first_sparse(const MrPass ps, float2 *__restrict__ sm,
                                             const float2 *__restrict__ twN, int N, int T, int j,
                                             bool active, unsigned mag0, First first_nz) {
    mr_first_sparse_body<R, SIGN>(ps, sm, twN, N, T, j, active, mag0, first_nz);
}
template <int R, int SIGN>
__device__ __noinline__ void mr_mid(const MrPass ps, float2 *__restrict__ sm, const float2 *__restrict__ twN,
                                    int N, int T, int j, bool active) {
    mr_mid_body<R, SIGN>(ps, sm, twN, N, T, j, active);
}

// Threads of a CTA: `rows` rows of T threads; thread (rr, j) works on row
// blockIdx.x * rows + rr.
struct RowSlot {
    int rr, j;
    bool active;
};
__device__ __forceinline__ RowSlot row_slot(const MrSchedule &sch, int rows, int total_rows) {
    RowSlot s;
    s.rr = (int)threadIdx.x / sch.T;
    s.j = (int)threadIdx.x - s.rr * sch.T;
    s.active = s.rr < rows && (int)blockIdx.x * rows + s.rr < total_rows;
    return s;
}

#define CWT_MR_RADICES(X) \
    X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(12) X(14) X(15) X(16) X(18) X(20) X(21) X(24) X(25) X(27) X(28) X(30) X(32)

// The whole row (at least two passes).  `sm` is this row's buffer of
// N + N/16 float2; on return it holds X[t] at spad2(t) (natural order) for
// every active row, after a barrier, for the caller's epilogue.  All threads
// of the CTA call it together.  Each pass of each radix is a separate (not
// inlined) function with its own register allocation, and the last pass is
// an ordinary buffer-to-buffer pass, so a schedule that repeats a radix
// (10000 = 16 x 25 x 25) runs the same code twice; the functors are passed
// by value and must capture by value.
template <int SIGN, typename Load, typename First>
__device__ __forceinline__ void mr_row(const MrSchedule &sch, float2 *__restrict__ sm,
                                       const float2 *__restrict__ twN, int j, bool active,
                                       bool sparse, const Load &load, const First &first_nz) {
    const int N = sch.N, T = sch.T;
    {
        const MrPass ps = sch.p[0];
        if (sparse) {
            switch (ps.R) {
#define CWT_MR_CASE(RR) \
    case RR: mr_first_sparse<RR, SIGN>(ps, sm, twN, N, T, j, active, sch.mag0, first_nz); break;
                CWT_MR_RADICES(CWT_MR_CASE)
#undef CWT_MR_CASE
                default: break;
            }
        } else {
            switch (ps.R) {
#define CWT_MR_CASE(RR) \
    case RR: mr_first<RR, SIGN>(ps, sm, N, T, j, active, load); break;
                CWT_MR_RADICES(CWT_MR_CASE)
#undef CWT_MR_CASE
                default: break;
            }
        }
        __syncthreads();  // pass-0 outputs visible; every thread arrives here
    }
#pragma unroll 1
    for (int p = 1; p < sch.np; ++p) {
        const MrPass ps = sch.p[p];
        switch (ps.R) {
#define CWT_MR_CASE(RR) \
    case RR: mr_mid<RR, SIGN>(ps, sm, twN, N, T, j, active); break;
            CWT_MR_RADICES(CWT_MR_CASE)
#undef CWT_MR_CASE
            default: break;
        }
    }
}

// The row for schedules that use only the radices RA and RB, with every pass
// inlined: no call overhead or register save/restore between passes, and
// two radices are few enough for one register allocation (about 1.35x the
// throughput of the out-of-line form at N = 10000 = 16 x 25 x 25).
template <int SIGN, int RA, int RB, typename Load, typename First>
__device__ __forceinline__ void mr_row_pair(const MrSchedule &sch, float2 *__restrict__ sm,
                                            const float2 *__restrict__ twN, int j, bool active,
                                            bool sparse, const Load &load, const First &first_nz) {
    const int N = sch.N, T = sch.T;
    {
        const MrPass ps = sch.p[0];
        if (sparse) {
            if (ps.R == RA) mr_first_sparse_body<RA, SIGN>(ps, sm, twN, N, T, j, active, sch.mag0, first_nz);
            else mr_first_sparse_body<RB, SIGN>(ps, sm, twN, N, T, j, active, sch.mag0, first_nz);
        } else {
            if (ps.R == RA) mr_first_body<RA, SIGN>(ps, sm, N, T, j, active, load);
            else mr_first_body<RB, SIGN>(ps, sm, N, T, j, active, load);
        }
        __syncthreads();  // pass-0 outputs visible; every thread arrives here
    }
#pragma unroll 1
    for (int p = 1; p < sch.np; ++p) {
        const MrPass ps = sch.p[p];
        if (ps.R == RA) mr_mid_body<RA, SIGN>(ps, sm, twN, N, T, j, active);
        else mr_mid_body<RB, SIGN>(ps, sm, twN, N, T, j, active);
    }
}

// ---- fixed-length rows --------------------------------------------------------
// A row length compiled with its whole schedule as constants: N = R_0 ... R_{P-1}
// (the order the host scheduler picks for N), T threads per row, ROWS rows
// per CTA, and registers for MINB such CTAs per SM.  Every stride, butterfly
// count and magic divisor is then a compile-time constant, and the passes use
// linear addressing where the strides allow it.  The host runs one only when
// the scheduler's MrSchedule for N equals pass() field by field.
__host__ __device__ constexpr unsigned mr_magic(int d) {
    return d <= 1 ? 0u : (unsigned)(((1ull << 32) + (unsigned)d - 1) / (unsigned)d);
}

template <int N_, int T_, int ROWS_, int MINB_, int... Rs>
struct MrFixed {
    static constexpr int N = N_, T = T_, ROWS = ROWS_, MINB = MINB_, NP = (int)sizeof...(Rs);
    static constexpr int THREADS = (ROWS * T + 31) / 32 * 32;  // whole warps
    __host__ __device__ static constexpr int radix(int p) {  // R_p
        int i = 0, r = 0;
        ((r = (i++ == p ? Rs : r)), ...);
        return r;
    }
    __host__ __device__ static constexpr int ns(int p) {
        int v = 1;
        for (int i = 0; i < p; ++i) v *= radix(i);
        return v;
    }
    __host__ __device__ static constexpr MrPass pass(int p) {
        return MrPass{radix(p), (N / radix(p) + T - 1) / T, ns(p), mr_magic(ns(p)), N / (ns(p) * radix(p))};
    }
    static constexpr unsigned mag0 = mr_magic(N / radix(0));
    static_assert(NP >= 2 && NP <= kMrMaxPasses && ns(NP) == N, "N = R_0 ... R_{P-1}");
    static_assert(ROWS >= 1 && THREADS <= kMrThreads, "one CTA holds ROWS rows");
    __host__ __device__ static constexpr bool fits() {
        for (int p = 0; p < NP; ++p)
            if (pass(p).G * radix(p) > kMrPoints && pass(p).G > 1) return false;
        return true;
    }
    static_assert(fits(), "at most 32 values per thread and pass");
};

// The row of a fixed-length schedule FX (all passes inlined).
template <class FX, int SIGN, typename Load, typename First>
__device__ __forceinline__ void mr_row_fixed(float2 *__restrict__ sm, const float2 *__restrict__ twN, int j,
                                             bool active, bool sparse, const Load &load, const First &first_nz) {
    constexpr int R0 = FX::radix(0);
    const MrPass p0 = FX::pass(0);
    if (sparse) mr_first_sparse_body<R0, SIGN, true>(p0, sm, twN, FX::N, FX::T, j, active, FX::mag0, first_nz);
    else mr_first_body<R0, SIGN, true>(p0, sm, FX::N, FX::T, j, active, load);
    __syncthreads();  // pass-0 outputs visible
    static_for<FX::NP - 1>([&](auto P) {
        constexpr int p = decltype(P)::value + 1;
        mr_mid_body<FX::radix(p), SIGN, true>(FX::pass(p), sm, twN, FX::N, FX::T, j, active);
    });
}

}  // namespace cwtk
