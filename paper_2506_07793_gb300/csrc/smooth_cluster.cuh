// smooth_cluster.cuh -- forward FFT and fused scale block for 2,3,5,7-smooth
// padded lengths above one CTA's 16384 points (the padding policy of Section
// "Fast Fourier transform"), e.g. the 122880 samples of a minute at 2048 Hz,
// which are smooth (2^13 3 5) and need no padding at all.
//
// A row of N = CL NL points (CL = 2 ... 16, NL <= 16384 smooth) runs on a
// thread-block cluster of CL CTAs with the decomposition of fft_cluster.cuh:
// CTA c transforms the residue class k = c + CL m (m < NL) with the
// mixed-radix row of mixed_radix.cuh (the scheduler's schedule for NL), and
// one cross-CTA radix-CL stage over distributed shared memory finishes it:
//     X[t1 + NL t2] = sum_c w_CL^(c t2) w_N^(c t1) A_c[t1],
// CTA c taking t1 in [c NL / CL, (c + 1) NL / CL).  The per-row arithmetic
// (band product, inverse FFT, reduction) is that of smooth_kernel.cuh and
// cluster.cu (Eq. 2).  The local row is the runtime schedule (FX = void,
// smooth_cluster.cu, CL <= 8) or a fixed-length one compiled in
// (smooth_cluster_fixed.cu) or at plan creation (jit.cu); clusters of more
// than 8 CTAs (a non-portable size, opted into per kernel) run only those.
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

// Local lengths whose schedule is compiled in (index, the cluster sizes it is
// built for as a bit mask, NL, T, rows = 1, CTAs per SM, radices), each in a
// translation unit of its own (smooth_cluster_fixed_<index>.cu): 15360 =
// 16 x 30 x 32 (30720, 61440: a minute at 512 or 1024 Hz); 15000 =
// 10 x 10 x 10 x 15 (a minute at 500 Hz); and three local rows whose 85 - 105
// KB CTAs fit two per SM, which the split prefers: 10000 = 16 x 25 x 25
// (20000, 30000, 50000, 100000), 12000 = 16 x 25 x 30 (24000, 60000, 120000)
// and 12288 = 32 x 16 x 24 (a minute at 2048 Hz: 122880 = 10 x 12288), the
// last three also on clusters of 10 CTAs (non-portable cluster size).
#define CWT_CL_PORTABLE 0x1FCu  // cluster sizes 2 ... 8
#define CWT_CL_MR_FIXED_0(X) X(0, CWT_CL_PORTABLE, 15360, 512, 1, 1, 16, 30, 32)
#define CWT_CL_MR_FIXED_1(X) X(1, CWT_CL_PORTABLE, 15000, 512, 1, 1, 10, 10, 10, 15)
#define CWT_CL_MR_FIXED_2(X) X(2, CWT_CL_PORTABLE | (1u << 10), 10000, 416, 1, 2, 16, 25, 25)
#define CWT_CL_MR_FIXED_3(X) X(3, CWT_CL_PORTABLE | (1u << 10), 12000, 512, 1, 2, 16, 25, 30)
#define CWT_CL_MR_FIXED_4(X) X(4, CWT_CL_PORTABLE | (1u << 10), 12288, 512, 1, 2, 32, 16, 24)
#define CWT_CL_MR_FIXED(X) \
    CWT_CL_MR_FIXED_0(X) CWT_CL_MR_FIXED_1(X) CWT_CL_MR_FIXED_2(X) CWT_CL_MR_FIXED_3(X) CWT_CL_MR_FIXED_4(X)

// Largest cluster (CTAs per row): 2 ... 8 is the portable range; 9 ... 16
// run only on kernels compiled in for that size or compiled at plan creation.
constexpr int kMaxClusterCtas = 16;

// Index in CWT_CL_MR_FIXED of the local schedule s built for cluster size
// cl, or -1; the CTAs per SM entry I is built for (smooth_cluster_fixed.cu).
int cl_mr_fixed_index(const MrSchedule &s, int cl);
int cl_mr_fixed_minb(int I);
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

// Clusters above 8 CTAs launch once the kernel allows non-portable sizes.
template <int CL, typename K>
cudaError_t ensure_cluster_attr(K *kernel, std::atomic<unsigned> *done) {
    if constexpr (CL <= 8) {
        return cudaSuccess;
    } else {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 32 && (done->load(std::memory_order_acquire) & (1u << dev))) return cudaSuccess;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess && dev < 32) done->fetch_or(1u << dev, std::memory_order_acq_rel);
        return e;
    }
}

// rows < 0: every row of the plan; else the first `rows` (the tuner's timing).
template <int CL, class FX>
cudaError_t sb_launch(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows = -1) {
    static std::atomic<unsigned> done{0}, done_cl{0};
    const int smem = (p->sch.N + (p->sch.N >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(scale_block_kernel<CL, FX>, kMrMaxSmem, &done);
    if (e == cudaSuccess) e = ensure_cluster_attr<CL>(scale_block_kernel<CL, FX>, &done_cl);
    if (e != cudaSuccess) return e;
    const int threads = (p->sch.T + 31) & ~31;
    scale_block_kernel<CL, FX><<<(rows < 0 ? p->C * p->S : rows) * CL, threads, smem, st>>>(a, p->sch);
    return cudaGetLastError();
}

template <int CL, class FX>
cudaError_t fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    static std::atomic<unsigned> done{0}, done_cl{0};
    const int smem = (p->sch.N + (p->sch.N >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(forward_kernel<CL, FX>, kMrMaxSmem, &done);
    if (e == cudaSuccess) e = ensure_cluster_attr<CL>(forward_kernel<CL, FX>, &done_cl);
    if (e != cudaSuccess) return e;
    const int threads = (p->sch.T + 31) & ~31;
    forward_kernel<CL, FX><<<p->C * CL, threads, smem, st>>>(signal, p->io == CWT_DTYPE_F64, p->n, p->spec,
                                                            p->twL, p->twN, p->sch);
    return cudaGetLastError();
}

// The launch on cluster size p->cl among the sizes of MASK (bit CL), instantiated for those only.
template <class FX, unsigned MASK, int CL = 2>
cudaError_t sb_any_cl(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows) {
    if constexpr (CL > kMaxClusterCtas) {
        return cudaErrorInvalidValue;
    } else {
        if constexpr (((MASK >> CL) & 1u) != 0)
            if (p->cl == CL) return sb_launch<CL, FX>(p, a, st, rows);
        return sb_any_cl<FX, MASK, CL + 1>(p, a, st, rows);
    }
}

template <class FX, unsigned MASK, int CL = 2>
cudaError_t fwd_any_cl(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    if constexpr (CL > kMaxClusterCtas) {
        return cudaErrorInvalidValue;
    } else {
        if constexpr (((MASK >> CL) & 1u) != 0)
            if (p->cl == CL) return fwd_launch<CL, FX>(p, signal, st);
        return fwd_any_cl<FX, MASK, CL + 1>(p, signal, st);
    }
}

}  // namespace cl_mr

// The definitions of cl_fixed_sb<I> / cl_fixed_fwd<I> for one entry of
// CWT_CL_MR_FIXED (expanded in that entry's translation unit).
#define CWT_CL_FIXED_DEFINE(I, MASK, N, T, ROWS, MINB, ...)                                        \
    template <>                                                                                    \
    cudaError_t cl_fixed_sb<I>(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows) { \
        return cl_mr::sb_any_cl<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>, (MASK)>(p, a, st, rows);   \
    }                                                                                              \
    template <>                                                                                    \
    cudaError_t cl_fixed_fwd<I>(const cwt_plan_s *p, const void *signal, cudaStream_t st) {        \
        return cl_mr::fwd_any_cl<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>, (MASK)>(p, signal, st);   \
    }

}  // namespace cwtk
