// smooth_cluster.cuh -- forward FFT and fused scale block for 2,3,5,7-smooth
// padded lengths above one CTA's 16384 points (the padding policy of Section
// "Fast Fourier transform"), e.g. the 122880 samples of a minute at 2048 Hz,
// which are smooth (2^13 3 5) and need no padding at all.
//
// A row of N = CL NL points (CL = 2 ... 8, NL <= 16384 smooth) runs on a
// thread-block cluster of CL CTAs with the decomposition of fft_cluster.cuh:
// CTA c transforms the residue class k = c + CL m (m < NL) with the
// mixed-radix row of mixed_radix.cuh (the scheduler's schedule for NL), and
// one cross-CTA radix-CL stage over distributed shared memory finishes it:
//     X[t1 + NL t2] = sum_c w_CL^(c t2) w_N^(c t1) A_c[t1],
// CTA c taking t1 in [c NL / CL, (c + 1) NL / CL).  The per-row arithmetic
// (band product, inverse FFT, reduction) is that of smooth_kernel.cuh and
// cluster.cu (Eq. 2).  The local row is the runtime schedule (FX = void,
// smooth_cluster.cu) or a fixed-length one compiled in (smooth_cluster_fixed.cu).
// The same kernels run the smooth lengths of at most 16384 points that no
// one-CTA schedule covers (e.g. 14175 = 3 x 4725, 15625 = 5 x 3125).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "fft_cluster.cuh"
#include "smooth_kernel.cuh"

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

// Cluster sizes (CTAs per row) the kernels are built for; the runtime-
// schedule kernels of the first group are in smooth_cluster.cu, of the
// second in smooth_cluster_wide.cu (two translation units that compile in
// parallel).
#define CWT_CL_SIZES_NARROW(X) X(2) X(3) X(4)
#define CWT_CL_SIZES_WIDE(X) X(5) X(6) X(7) X(8)
#define CWT_CL_SIZES(X) CWT_CL_SIZES_NARROW(X) CWT_CL_SIZES_WIDE(X)

// Local lengths whose schedule is compiled in (index, NL, T, rows = 1, CTAs
// per SM, radices), each in a translation unit of its own
// (smooth_cluster_fixed_<index>.cu): 15360 = 16 x 30 x 32, the local row of
// a minute at 512, 1024 or 2048 Hz (30720, 61440, 122880); 15000 =
// 10 x 10 x 10 x 15 (30000, 60000, 120000: a minute at 500, 1000, 2000 Hz);
// 10000 = 16 x 25 x 25 (20000, 40000, 80000), whose 85 KB CTAs fit two per SM.
#define CWT_CL_MR_FIXED_0(X) X(0, 15360, 512, 1, 1, 16, 30, 32)
#define CWT_CL_MR_FIXED_1(X) X(1, 15000, 512, 1, 1, 10, 10, 10, 15)
#define CWT_CL_MR_FIXED_2(X) X(2, 10000, 512, 1, 2, 16, 25, 25)
#define CWT_CL_MR_FIXED(X) CWT_CL_MR_FIXED_0(X) CWT_CL_MR_FIXED_1(X) CWT_CL_MR_FIXED_2(X)

// Index in CWT_CL_MR_FIXED of the local schedule s, or -1 (smooth_cluster_fixed.cu).
int cl_mr_fixed_index(const MrSchedule &s);
// The fixed-length launches (smooth_cluster_fixed.cu).
cudaError_t cl_mr_fixed_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st);
cudaError_t cl_mr_fixed_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st);
// Entry I of CWT_CL_MR_FIXED on any cluster size (smooth_cluster_fixed_<I>.cu).
template <int I>
cudaError_t cl_fixed_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st);
template <int I>
cudaError_t cl_fixed_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st);
// The runtime-schedule launches for CWT_CL_SIZES_WIDE (smooth_cluster_wide.cu).
cudaError_t cl_mr_wide_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st);
cudaError_t cl_mr_wide_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st);

namespace cl_mr {

namespace cg = cooperative_groups;

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
    if constexpr (std::is_void_v<FX>)
        mr_row<SIGN>(sch, sm, twL, j, j < sch.T, sparse, load, first_nz);
    else
        mr_row_fixed<FX, SIGN>(sm, twL, j, j < FX::T, sparse, load, first_nz);
}

template <class FX>
__device__ __forceinline__ int local_n(const MrSchedule &sch) {
    if constexpr (std::is_void_v<FX>) return sch.N;
    else return FX::N;
}

// CTAs per SM the register budget is set for.
template <class FX>
constexpr int min_blocks() {
    if constexpr (std::is_void_v<FX>) return 1;
    else return FX::MINB;
}

template <class FX>
__device__ __forceinline__ int first_radix(const MrSchedule &sch) {
    if constexpr (std::is_void_v<FX>) return sch.p[0].R;
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
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kMrThreads, min_blocks<FX>())
scale_block_kernel(const ClMrArgs a, const MrSchedule sch) {
    extern __shared__ float2 mrsm[];
    float2 *sm = mrsm;
    const int NL = local_n<FX>(sch), N = CL * NL;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
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
    cl.sync();  // every CTA's A_c in natural order
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
    cl.sync();  // no CTA still reads this CTA's buffer
}

template <int CL, class FX>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kMrThreads, min_blocks<FX>())
forward_kernel(const void *__restrict__ x, int f64, int n, float2 *__restrict__ spec,
               const float2 *__restrict__ twL, const float2 *__restrict__ twN, const MrSchedule sch) {
    extern __shared__ float2 mrsm[];
    float2 *sm = mrsm;
    const int NL = local_n<FX>(sch), N = CL * NL;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int row = (int)blockIdx.x / CL;
    const SignalLoad load{(const float *)x + (size_t)row * n, (const double *)x + (size_t)row * n, f64, n,
                          rank, CL};
    local_row<FX, -1>(sch, sm, twL, (int)threadIdx.x, false, load, NoFirst{});
    cl.sync();
    float2 *o = spec + (size_t)row * N;
    cross<CL, -1>(sm, twN, NL, rank, [&](int t, float2 v) { o[t] = v; });
    cl.sync();
}

template <int CL, class FX>
cudaError_t sb_launch(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    const int smem = (p->sch.N + (p->sch.N >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(scale_block_kernel<CL, FX>, kMrMaxSmem, &done);
    if (e != cudaSuccess) return e;
    const int threads = (p->sch.T + 31) & ~31;
    scale_block_kernel<CL, FX><<<p->C * p->S * CL, threads, smem, st>>>(a, p->sch);
    return cudaGetLastError();
}

template <int CL, class FX>
cudaError_t fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    const int smem = (p->sch.N + (p->sch.N >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(forward_kernel<CL, FX>, kMrMaxSmem, &done);
    if (e != cudaSuccess) return e;
    const int threads = (p->sch.T + 31) & ~31;
    forward_kernel<CL, FX><<<p->C * CL, threads, smem, st>>>(signal, p->io == CWT_DTYPE_F64, p->n, p->spec,
                                                            p->twL, p->twN, p->sch);
    return cudaGetLastError();
}

template <class FX>
cudaError_t sb_any_cl(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st) {
    switch (p->cl) {
#define CWT_CL_CASE(CL) \
    case CL: return sb_launch<CL, FX>(p, a, st);
        CWT_CL_SIZES(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <class FX>
cudaError_t fwd_any_cl(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    switch (p->cl) {
#define CWT_CL_CASE(CL) \
    case CL: return fwd_launch<CL, FX>(p, signal, st);
        CWT_CL_SIZES(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cl_mr

// The definitions of cl_fixed_sb<I> / cl_fixed_fwd<I> for one entry of
// CWT_CL_MR_FIXED (expanded in that entry's translation unit).
#define CWT_CL_FIXED_DEFINE(I, N, T, ROWS, MINB, ...)                                              \
    template <>                                                                                    \
    cudaError_t cl_fixed_sb<I>(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st) {          \
        return cl_mr::sb_any_cl<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(p, a, st);                 \
    }                                                                                              \
    template <>                                                                                    \
    cudaError_t cl_fixed_fwd<I>(const cwt_plan_s *p, const void *signal, cudaStream_t st) {        \
        return cl_mr::fwd_any_cl<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(p, signal, st);           \
    }

}  // namespace cwtk
