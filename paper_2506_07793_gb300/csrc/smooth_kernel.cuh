// smooth_kernel.cuh -- the forward FFT and the fused scale-block kernel for 2,3,5,7-smooth
// padded lengths (Section "Fast Fourier transform"; the arithmetic per row is
// that of scale_block.cu, Eq. 2), as a template over the row form: RA = RB = 0
// is the generic row (every radix, passes out of line, smooth.cu); a radix
// pair (RA, RB) is the inlined row for schedules that use only those two
// radices (smooth_fast_*.cu), one translation unit per group of pairs so
// that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "smooth_device.cuh"

namespace cwtk {

constexpr int kMrMaxSmem = (kMaxFft + (kMaxFft >> 4)) * 8;

// Rows per CTA for a launch over total_rows rows (smooth.cu).
int mr_launch_rows(const MrSchedule &sch, int total_rows);

// The runtime-schedule kernel: RA = RB = 0 the generic row, else the inlined
// radix pair.
template <int RA, int RB>
__global__ void __launch_bounds__(kMrThreads, 1)
mr_scale_block_kernel(const MrArgs a, const MrSchedule sch, int rows) {
    const RowSlot rs = row_slot(sch, rows, a.total_rows);
    mr_sb_row<false>(a, sch.N, sch.T, sch.p[0].R, rs, rows,
                     [&](float2 *sm, bool sparse, const auto &load, const auto &first_nz) {
                         if constexpr (RA == 0)
                             mr_row<+1>(sch, sm, a.twN, rs.j, rs.active, sparse, load, first_nz);
                         else
                             mr_row_pair<+1, RA, RB>(sch, sm, a.twN, rs.j, rs.active, sparse, load, first_nz);
                     });
}

template <int RA, int RB>
cudaError_t mr_sb_launch(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    cudaError_t e = ensure_smem_attr(mr_scale_block_kernel<RA, RB>, kMrMaxSmem, &done);
    if (e != cudaSuccess) return e;
    const int rows = mr_launch_rows(p->sch, a.total_rows);
    const int smem = rows * (p->N + (p->N >> 4)) * 8;
    const int threads = (rows * p->sch.T + 31) & ~31;
    mr_scale_block_kernel<RA, RB><<<(a.total_rows + rows - 1) / rows, threads, smem, st>>>(a, p->sch, rows);
    return cudaGetLastError();
}

// Forward FFT of each zero-padded channel (float32 or float64 samples), Eq. 2;
// RA = RB = 0 is the generic row, else the inlined radix pair.
template <int RA, int RB>
__global__ void __launch_bounds__(kMrThreads, 1)
mr_forward_kernel(const void *__restrict__ x, int f64, int n, float2 *__restrict__ spec,
                  const float2 *__restrict__ twN, const MrSchedule sch, int rows, int C) {
    extern __shared__ float2 mrsm[];
    const int N = sch.N;
    const RowSlot rs = row_slot(sch, rows, C);
    const int row = rs.active ? (int)blockIdx.x * rows + rs.rr : 0;
    const int rr = rs.rr < rows ? rs.rr : 0;
    float2 *sm = mrsm + (size_t)rr * (N + (N >> 4));
    const float *xf = (const float *)x + (size_t)row * n;
    const double *xd = (const double *)x + (size_t)row * n;
    float2 *out = spec + (size_t)row * N;
    auto load = [=](int i) -> float2 {
        float v = 0.f;
        if (i < n) v = f64 ? (float)xd[i] : xf[i];
        return make_float2(v, 0.f);
    };
    auto none = [](int, int, unsigned, int &, float2 &) -> bool { return false; };
    if constexpr (RA == 0)
        mr_row<-1>(sch, sm, twN, rs.j, rs.active, false, load, none);
    else
        mr_row_pair<-1, RA, RB>(sch, sm, twN, rs.j, rs.active, false, load, none);
    if (rs.active) {
#pragma unroll 4
        for (int t = rs.j; t < N; t += sch.T) out[t] = *CWT_SMEM(&sm[spad2(t)]);
    }
}

template <int RA, int RB>
cudaError_t mr_fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    cudaError_t e = ensure_smem_attr(mr_forward_kernel<RA, RB>, kMrMaxSmem, &done);
    if (e != cudaSuccess) return e;
    const int rows = mr_launch_rows(p->sch, p->C);
    const int smem = rows * (p->N + (p->N >> 4)) * 8;
    const int threads = (rows * p->sch.T + 31) & ~31;
    mr_forward_kernel<RA, RB><<<(p->C + rows - 1) / rows, threads, smem, st>>>(
        signal, p->io == CWT_DTYPE_F64, p->n, p->spec, p->twN, p->sch, rows, p->C);
    return cudaGetLastError();
}

// Fixed-length kernels (index = MrSchedule::fixed): index, N, T, rows per CTA,
// CTAs per SM for the register budget, the radices in the scheduler's order
// (for most of them the pass order the plan-time tuner measured fastest,
// smooth.cu's kMeasuredOrders).  Whole seconds of EEG at 250 / 500 / 1000 Hz;
// rows and CTAs per SM measured per length, or those the tuner ran with
// (several CTAs per SM hide one row's pass barriers behind the others' work,
// fewer leave more registers per thread).  The kernels of list A are in
// smooth_fixed.cu, of list B in smooth_fixed_b.cu (two translation units that
// compile in parallel).
#define CWT_MR_FIXED_A(X)                     \
    X(0, 10000, 416, 1, 2, 16, 25, 25)        \
    X(1, 8000, 416, 1, 2, 16, 25, 20)         \
    X(2, 5000, 256, 1, 4, 20, 10, 25)         \
    X(3, 4000, 256, 1, 4, 16, 10, 25)         \
    X(4, 2500, 100, 2, 4, 25, 10, 10)         \
    X(5, 2000, 100, 2, 4, 20, 10, 10)         \
    X(6, 1000, 50, 5, 4, 10, 10, 10)          \
    X(7, 500, 25, 10, 3, 20, 25)              \
    X(8, 12000, 512, 1, 2, 16, 25, 30)        \
    X(9, 7500, 384, 1, 2, 25, 10, 30)         \
    X(10, 6000, 256, 1, 4, 24, 10, 25)        \
    X(11, 15000, 512, 1, 1, 10, 10, 10, 15)   \
    X(12, 3000, 125, 2, 4, 24, 5, 25)         \
    X(13, 9000, 384, 1, 2, 24, 15, 25)        \
    X(14, 1500, 50, 4, 4, 10, 10, 15)
#define CWT_MR_FIXED_B(X)                     \
    X(15, 14000, 512, 1, 1, 14, 10, 10, 10)   \
    X(16, 13500, 512, 1, 1, 6, 10, 15, 15)    \
    X(17, 12500, 512, 1, 2, 10, 10, 5, 25)    \
    X(18, 10500, 448, 1, 2, 28, 15, 25)       \
    X(19, 7000, 288, 1, 3, 28, 10, 25)        \
    X(20, 4500, 160, 1, 4, 10, 15, 30)        \
    X(21, 3750, 256, 1, 4, 25, 6, 25)         \
    X(22, 3500, 192, 1, 4, 28, 5, 25)         \
    X(23, 2250, 75, 2, 3, 10, 15, 15)         \
    X(24, 1750, 70, 3, 4, 14, 5, 25)          \
    X(25, 1250, 50, 5, 4, 25, 10, 5)          \
    X(26, 750, 30, 8, 3, 25, 30)
#define CWT_MR_FIXED(X) CWT_MR_FIXED_A(X) CWT_MR_FIXED_B(X)

// Index of the fixed-length kernel whose schedule equals s, or -1.
int mr_fixed_index(const MrSchedule &s);
cudaError_t mr_fixed_sb_launch(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st);
// Entry I of CWT_MR_FIXED: its scale-block and forward launches (defined in
// the translation unit of its list).
template <int I>
cudaError_t mr_fixed_sb(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st);
template <int I>
cudaError_t mr_fixed_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st);
// The forward FFTs of a plan whose schedule is a fixed-length one (same
// schedule, SIGN -1, the forward kernel's epilogue).
cudaError_t mr_fixed_fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st);
// The kernels compiled at plan creation (p->jit, jit.cu).
cudaError_t jit_sb_launch(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st);
cudaError_t jit_fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st);

// The inlined radix pairs (index = MrSchedule::fast), chosen for 2^a 5^b
// lengths (whole seconds of EEG at 250 / 500 / 1000 Hz), each instantiated in
// smooth_fast_*.cu.
#define CWT_MR_FAST_PAIRS(X) \
    X(0, 16, 25) X(1, 20, 25) X(2, 10, 16) X(3, 16, 20) X(4, 8, 25) X(5, 10, 32) X(6, 10, 20) X(7, 10, 25)

#define CWT_MR_DECLARE_PAIR(I, A, B)                                                                  \
    extern template cudaError_t mr_sb_launch<A, B>(const cwt_plan_s *, const MrArgs &, cudaStream_t); \
    extern template cudaError_t mr_fwd_launch<A, B>(const cwt_plan_s *, const void *, cudaStream_t);
CWT_MR_FAST_PAIRS(CWT_MR_DECLARE_PAIR)
#undef CWT_MR_DECLARE_PAIR

}  // namespace cwtk
