// smooth_cluster_device.cuh -- the device side of the smooth-length cluster
// kernels (smooth_cluster.cuh has the decomposition and the launches): the
// row arguments, the local-row functors, the cross-CTA stage and the kernels.
// Its cluster primitives are inline PTX (dsmem.cuh) and it includes no host
// or toolkit header, so that the plan-time compiler (jit.cu) builds these
// kernels for a local length that has none compiled in.
#pragma once

#include "dsmem.cuh"
#include "smooth_device.cuh"

namespace cwtk {

struct ClMrArgs {
    const float2 *spec;  // [C][N]
    const float *bank;   // [S][N]
    const int *band;     // [S][2]
    const float2 *twL;   // exp(2 pi i m / NL), m < NL: the local passes
    const float2 *twN;   // exp(2 pi i m / N), m < N: the cross-CTA stage
    void *out_c, *out_p, *out_ph;
    int S, n_out, sub, f64;
};

namespace cl_mr {

// FX = void: the runtime schedule; else a fixed-length one (MrFixed).
template <class T>
struct is_void {
    static constexpr bool value = false;
};
template <>
struct is_void<void> {
    static constexpr bool value = true;
};

// Functors of the local row, the same types for every cluster size so that
// the out-of-line passes of the runtime schedule are instantiated once.
// Residue class `rank` of `cl`: local point m is global bin k = rank + cl m.
struct BandLoad {  // the band product W_s[k] X_c[k], zero off the band
    const float2 *X;
    const float *W;
    int b0, B, N, rank, cl;
    __device__ __forceinline__ float2 operator()(int m) const {
        const int k = rank + cl * m;
        int dk = k - b0;  // the band is [b0, b0 + B) modulo N
        if (dk < 0) dk += N;
        if (dk < B) {
            const float2 xv = X[k];
            const float w = W[k];
            return make_float2(xv.x * w, xv.y * w);
        }
        return make_float2(0.f, 0.f);
    }
};

// The class's in-band m form one cyclic run [m_first, m_first + Bm) of the
// NL local points; with Bm <= nb = NL / R_0 each first-pass butterfly b
// (inputs b + r nb) meets at most one of them.
struct BandFirst {
    const float2 *X;
    const float *W;
    int m_first, Bm, NL, rank, cl;
    __device__ __forceinline__ bool operator()(int b, int nb, unsigned mag, int &r, float2 &x) const {
        const unsigned d = (unsigned)(b - m_first + NL);  // > 0; NL is a multiple of nb
        const int u = (int)(d - __umulhi(d, mag) * (unsigned)nb);  // (b - m_first) mod nb
        if (u >= Bm) return false;
        int m = m_first + u;
        if (m >= NL) m -= NL;
        r = (int)__umulhi((unsigned)(m - b), mag);  // (m - b) / nb: m = b (mod nb), m >= b
        const int k = rank + cl * m;
        const float2 xv = X[k];
        const float w = W[k];
        x = make_float2(xv.x * w, xv.y * w);
        return true;
    }
};

struct SignalLoad {  // samples rank + cl m of the zero-padded channel
    const float *xf;
    const double *xd;
    int f64, n, rank, cl;
    __device__ __forceinline__ float2 operator()(int m) const {
        const int i = rank + cl * m;
        float v = 0.f;
        if (i < n) v = f64 ? (float)xd[i] : xf[i];
        return make_float2(v, 0.f);
    }
};

struct NoFirst {
    __device__ __forceinline__ bool operator()(int, int, unsigned, int &, float2 &) const { return false; }
};

template <class FX, int SIGN, typename Load, typename First>
__device__ __forceinline__ void local_row(const MrSchedule &sch, float2 *sm, const float2 *twL, int j,
                                          bool sparse, const Load &load, const First &first_nz) {
    if constexpr (is_void<FX>::value)
        mr_row<SIGN>(sch, sm, twL, j, j < sch.T, sparse, load, first_nz);
    else
        mr_row_fixed<FX, SIGN>(sm, twL, j, j < FX::T, sparse, load, first_nz);
}

template <class FX>
__device__ __forceinline__ int local_n(const MrSchedule &sch) {
    if constexpr (is_void<FX>::value) return sch.N;
    else return FX::N;
}

// Threads per CTA the kernel is compiled for.
template <class FX>
constexpr int max_threads() {
    if constexpr (is_void<FX>::value) return kMrThreads;
    else return FX::THREADS;
}

// CTAs per SM the register budget is set for.
template <class FX>
constexpr int min_blocks() {
    if constexpr (is_void<FX>::value) return 1;
    else return FX::MINB;
}

template <class FX>
__device__ __forceinline__ int first_radix(const MrSchedule &sch) {
    if constexpr (is_void<FX>::value) return sch.p[0].R;
    else return FX::radix(0);
}

// The cross-CTA stage of a row whose local results sit in each CTA's `sm` in
// natural order: every t1 of this CTA's range, the CL values A_c[t1], their
// twiddles w_N^(SIGN c t1), a CL-point DFT, and out(t1 + NL t2, X).
template <int CL, int SIGN, typename Out>
__device__ __forceinline__ void cross(const float2 *sm, const float2 *__restrict__ twN, int NL, int rank,
                                      const Out &out) {
    const int t_lo = (int)(((long long)rank * NL) / CL), t_hi = (int)(((long long)(rank + 1) * NL) / CL);
#pragma unroll 1
    for (int t1 = t_lo + (int)threadIdx.x; t1 < t_hi; t1 += (int)blockDim.x) {
        float2 a[CL];
#pragma unroll
        for (int c = 0; c < CL; ++c) a[c] = ld_cluster(CWT_SMEM(&sm[spad2(t1)]), (unsigned)c);
#pragma unroll
        for (int c = 1; c < CL; ++c) {
            float2 w = __ldg(&twN[c * t1]);  // c t1 < CL NL = N
            if (SIGN < 0) w.y = -w.y;
            a[c] = cmul(a[c], w);
        }
        dft_r<CL, SIGN>(a);
#pragma unroll
        for (int t2 = 0; t2 < CL; ++t2) out(t1 + NL * t2, a[t2]);
    }
}

template <int CL, class FX>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(max_threads<FX>(), min_blocks<FX>())
scale_block_kernel(const ClMrArgs a, const MrSchedule sch) {
    extern __shared__ float2 mrsm[];
    float2 *sm = mrsm;
    const int NL = local_n<FX>(sch), N = CL * NL;
    const int rank = (int)cluster_rank();
    const int row = (int)blockIdx.x / CL;
    const int c = row / a.S, s = row - c * a.S;
    const float2 *X = a.spec + (size_t)c * N;
    const float *W = a.bank + (size_t)s * N;
    const int b0 = a.band[2 * s], B = a.band[2 * s + 1];
    int delta = (rank - b0) % CL;  // first in-band bin of the class: b0 + delta
    if (delta < 0) delta += CL;
    const int Bm = delta < B ? (B - delta + CL - 1) / CL : 0;
    const int m_first = (int)(((unsigned)(((b0 + delta) % N) - rank) / (unsigned)CL) % (unsigned)NL);
    const BandLoad load{X, W, b0, B, N, rank, CL};
    const BandFirst first_nz{X, W, m_first, Bm, NL, rank, CL};
    local_row<FX, +1>(sch, sm, a.twL, (int)threadIdx.x, Bm <= NL / first_radix<FX>(sch), load, first_nz);
    cluster_sync();  // every CTA's A_c in natural order
    const size_t obase = (size_t)row * (size_t)a.n_out;
    const int sub = a.sub, n_out = a.n_out;
    auto out = [&](int t, float2 v) {
        int o = t;
        if (sub != 1) {
            if (t % sub) return;
            o = t / sub;
        }
        if (o >= n_out) return;
        if (a.f64) {
            if (a.out_c) ((double2 *)a.out_c)[obase + o] = make_double2(v.x, v.y);
            if (a.out_p) ((double *)a.out_p)[obase + o] = (double)fmaf(v.x, v.x, v.y * v.y);
            if (a.out_ph) mr_phase_d((double *)a.out_ph + obase + o, v);
        } else {
            if (a.out_c) ((float2 *)a.out_c)[obase + o] = v;
            if (a.out_p) ((float *)a.out_p)[obase + o] = fmaf(v.x, v.x, v.y * v.y);
            if (a.out_ph) mr_phase_f((float *)a.out_ph + obase + o, v);
        }
    };
    cross<CL, +1>(sm, a.twN, NL, rank, out);
    cluster_sync();  // no CTA still reads this CTA's buffer
}

template <int CL, class FX>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(max_threads<FX>(), min_blocks<FX>())
forward_kernel(const void *__restrict__ x, int f64, int n, float2 *__restrict__ spec,
               const float2 *__restrict__ twL, const float2 *__restrict__ twN, const MrSchedule sch) {
    extern __shared__ float2 mrsm[];
    float2 *sm = mrsm;
    const int NL = local_n<FX>(sch), N = CL * NL;
    const int rank = (int)cluster_rank();
    const int row = (int)blockIdx.x / CL;
    const SignalLoad load{(const float *)x + (size_t)row * n, (const double *)x + (size_t)row * n, f64, n,
                          rank, CL};
    local_row<FX, -1>(sch, sm, twL, (int)threadIdx.x, false, load, NoFirst{});
    cluster_sync();
    float2 *o = spec + (size_t)row * N;
    cross<CL, -1>(sm, twN, NL, rank, [&](int t, float2 v) { o[t] = v; });
    cluster_sync();
}

}  // namespace cl_mr
}  // namespace cwtk
