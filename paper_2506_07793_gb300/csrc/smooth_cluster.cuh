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

#include <cuda_runtime.h>

#include "smooth_cluster_device.cuh"
#include "smooth_kernel.cuh"

namespace cwtk {


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
// The fixed-length launches (smooth_cluster_fixed.cu); rows as sb_launch's.
cudaError_t cl_mr_fixed_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows = -1);
cudaError_t cl_mr_fixed_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st);
// Entry I of CWT_CL_MR_FIXED on any cluster size (smooth_cluster_fixed_<I>.cu).
template <int I>
cudaError_t cl_fixed_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows);
template <int I>
cudaError_t cl_fixed_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st);
// The cluster scale block compiled at plan creation (p->jit, jit.cu).
cudaError_t jit_cl_sb_launch(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st);
// The runtime-schedule launches for CWT_CL_SIZES_WIDE (smooth_cluster_wide.cu).
cudaError_t cl_mr_wide_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st);
cudaError_t cl_mr_wide_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st);

namespace cl_mr {

// rows < 0: every row of the plan; else the first `rows` (the tuner's timing).
template <int CL, class FX>
cudaError_t sb_launch(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows = -1) {
    static std::atomic<unsigned> done{0};
    const int smem = (p->sch.N + (p->sch.N >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(scale_block_kernel<CL, FX>, kMrMaxSmem, &done);
    if (e != cudaSuccess) return e;
    const int threads = (p->sch.T + 31) & ~31;
    scale_block_kernel<CL, FX><<<(rows < 0 ? p->C * p->S : rows) * CL, threads, smem, st>>>(a, p->sch);
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
cudaError_t sb_any_cl(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows) {
    switch (p->cl) {
#define CWT_CL_CASE(CL) \
    case CL: return sb_launch<CL, FX>(p, a, st, rows);
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
    cudaError_t cl_fixed_sb<I>(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows) { \
        return cl_mr::sb_any_cl<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(p, a, st, rows);           \
    }                                                                                              \
    template <>                                                                                    \
    cudaError_t cl_fixed_fwd<I>(const cwt_plan_s *p, const void *signal, cudaStream_t st) {        \
        return cl_mr::fwd_any_cl<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(p, signal, st);           \
    }

}  // namespace cwtk
