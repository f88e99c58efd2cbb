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
#include "mixed_radix.cuh"
#include "phase.cuh"

namespace cwtk {

constexpr int kMrMaxSmem = (kMaxFft + (kMaxFft >> 4)) * 8;

// Rows per CTA for a launch over total_rows rows (smooth.cu).
int mr_launch_rows(const MrSchedule &sch, int total_rows);

struct MrArgs {
    const float2 *spec;
    const float *bank;
    const int *band;
    const float2 *twN;
    void *out_c, *out_p, *out_ph;
    int S, n_out, sub, total_rows, f64;
};

__device__ __noinline__ inline void mr_phase_f(float *dst, float2 v) { *dst = phase_atan2(v.y, v.x); }
__device__ __noinline__ inline void mr_phase_d(double *dst, float2 v) { *dst = (double)phase_atan2(v.y, v.x); }

// Fused spectrum product, inverse FFT and epilogue of one (channel, scale)
// row, shared by the runtime-schedule and fixed-length kernels:
// run_row(sm, sparse, load, first_nz) runs the inverse FFT of the row held
// in `sm`.  LIN: the epilogue steps through the buffer by a constant padded
// stride when T sub is a multiple of 16 (fixed-length kernels).
template <bool LIN, typename RunRow>
__device__ __forceinline__ void mr_sb_row(const MrArgs &a, int N, int T, int R0, const RowSlot &rs, int rows,
                                          const RunRow &run_row) {
    extern __shared__ float2 mrsm[];
    const int row = rs.active ? (int)blockIdx.x * rows + rs.rr : 0;
    const int rr = rs.rr < rows ? rs.rr : 0;
    float2 *sm = mrsm + (size_t)rr * (N + (N >> 4));
    const int c = row / a.S, s = row - c * a.S;
    const float2 *X = a.spec + (size_t)c * N;
    const float *W = a.bank + (size_t)s * N;
    const int b0 = a.band[2 * s], B = a.band[2 * s + 1];
    auto load = [=](int k) -> float2 {
        int dk = k - b0;  // the band is [b0, b0 + B) modulo N
        if (dk < 0) dk += N;
        if (dk < B) {
            const float2 xv = X[k];
            const float w = W[k];
            return make_float2(xv.x * w, xv.y * w);
        }
        return make_float2(0.f, 0.f);
    };
    // Narrow band (B <= N/R_0): butterfly b's inputs b + r nb, r < R_0, meet
    // the band at most once, at e = b0 + u (mod N) with u = (b - b0) mod nb.
    auto first_nz = [=](int b, int nb, unsigned mag, int &r, float2 &x) -> bool {
        const unsigned d = (unsigned)(b - b0 + N);  // > 0; N is a multiple of nb
        const int u = (int)(d - __umulhi(d, mag) * (unsigned)nb);
        if (u >= B) return false;
        int e = b0 + u;
        if (e >= N) e -= N;
        r = (int)__umulhi((unsigned)(e - b), mag);  // (e - b) / nb, exact: e = b (mod nb), e >= b
        const float2 xv = X[e];
        const float w = W[e];
        x = make_float2(xv.x * w, xv.y * w);
        return true;
    };
    run_row(sm, B <= N / R0, load, first_nz);
    if (!rs.active) return;
    // epilogue: crop to t < n, keep t = sub * o, write the requested outputs
    // (consecutive threads take consecutive o: coalesced stores)
    const size_t obase = (size_t)row * (size_t)a.n_out;
    const int sub = a.sub, n_out = a.n_out;
    if (a.f64) {
        double2 *oc = (double2 *)a.out_c + obase;
        double *op = (double *)a.out_p + obase, *oph = (double *)a.out_ph + obase;
#pragma unroll 1
        for (int o = rs.j; o < n_out; o += T) {
            const float2 v = *CWT_SMEM(&sm[spad2(o * sub)]);
            if (a.out_c) oc[o] = make_double2(v.x, v.y);
            if (a.out_p) op[o] = (double)fmaf(v.x, v.x, v.y * v.y);
            if (a.out_ph) mr_phase_d(oph + o, v);
        }
    } else {
        float2 *oc = (float2 *)a.out_c + obase;
        float *op = (float *)a.out_p + obase, *oph = (float *)a.out_ph + obase;
        if (LIN && ((T * sub) & 15) == 0) {
            // spad2(o sub) advances by spad2(T sub) per step
            const float2 *src = sm + spad2(rs.j * sub);
            const int step = spad2(T * sub);
#pragma unroll 2
            for (int o = rs.j; o < n_out; o += T, src += step) {
                const float2 v = *CWT_SMEM(src);
                if (a.out_c) oc[o] = v;
                if (a.out_p) op[o] = fmaf(v.x, v.x, v.y * v.y);
                if (a.out_ph) mr_phase_f(oph + o, v);
            }
        } else {
#pragma unroll 2
            for (int o = rs.j; o < n_out; o += T) {
                const float2 v = *CWT_SMEM(&sm[spad2(o * sub)]);
                if (a.out_c) oc[o] = v;
                if (a.out_p) op[o] = fmaf(v.x, v.x, v.y * v.y);
                if (a.out_ph) mr_phase_f(oph + o, v);
            }
        }
    }
}

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

// The fixed-length kernel: FX::ROWS rows of FX::N points per CTA, FX::T
// threads each, with registers for FX::MINB such CTAs per SM.
template <class FX>
__global__ void __launch_bounds__(FX::THREADS, FX::MINB) mr_fixed_scale_block_kernel(const MrArgs a) {
    RowSlot rs;
    rs.rr = (int)threadIdx.x / FX::T;
    rs.j = (int)threadIdx.x - rs.rr * FX::T;
    rs.active = rs.rr < FX::ROWS && (int)blockIdx.x * FX::ROWS + rs.rr < a.total_rows;
    mr_sb_row<true>(a, FX::N, FX::T, FX::radix(0), rs, FX::ROWS,
                    [&](float2 *sm, bool sparse, const auto &load, const auto &first_nz) {
                        mr_row_fixed<FX, +1>(sm, a.twN, rs.j, rs.active, sparse, load, first_nz);
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
// CTAs per SM for the register budget, the radices in the scheduler's order.
// Whole seconds of EEG at 250 / 500 / 1000 Hz; the CTAs per SM were measured
// per length (several CTAs per SM hide one row's pass barriers behind the
// others' work, fewer leave more registers per thread).  The kernels of list A are in smooth_fixed.cu, of list B in
// smooth_fixed_b.cu (two translation units that compile in parallel).
#define CWT_MR_FIXED_A(X)                     \
    X(0, 10000, 512, 1, 2, 16, 25, 25)        \
    X(1, 8000, 512, 1, 2, 20, 20, 20)         \
    X(2, 5000, 256, 1, 4, 8, 25, 25)          \
    X(3, 4000, 256, 1, 4, 10, 20, 20)         \
    X(4, 2500, 125, 2, 3, 10, 10, 25)         \
    X(5, 2000, 100, 2, 4, 10, 10, 20)         \
    X(6, 1000, 50, 5, 4, 10, 10, 10)          \
    X(7, 500, 25, 10, 3, 20, 25)              \
    X(8, 12000, 512, 1, 2, 16, 25, 30)        \
    X(9, 7500, 384, 1, 2, 12, 25, 25)         \
    X(10, 6000, 256, 1, 4, 10, 24, 25)        \
    X(11, 15000, 512, 1, 1, 10, 10, 10, 15)   \
    X(12, 3000, 100, 2, 3, 10, 10, 30)        \
    X(13, 9000, 384, 1, 2, 10, 30, 30)        \
    X(14, 1500, 50, 4, 4, 10, 10, 15)
#define CWT_MR_FIXED_B(X)                     \
    X(15, 14000, 512, 1, 1, 10, 10, 10, 14)   \
    X(16, 13500, 512, 1, 1, 15, 30, 30)       \
    X(17, 12500, 512, 1, 2, 5, 10, 10, 25)    \
    X(18, 10500, 512, 1, 2, 15, 25, 28)       \
    X(19, 7000, 384, 1, 2, 10, 25, 28)        \
    X(20, 4500, 256, 1, 3, 10, 15, 30)        \
    X(21, 3750, 256, 1, 4, 6, 25, 25)         \
    X(22, 3500, 256, 1, 3, 5, 25, 28)         \
    X(23, 2250, 75, 2, 3, 10, 15, 15)         \
    X(24, 1750, 70, 2, 4, 5, 14, 25)          \
    X(25, 1250, 50, 4, 4, 5, 10, 25)          \
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

// Forward FFT of each zero-padded channel on a fixed-length schedule FX.
template <class FX>
__global__ void __launch_bounds__(FX::THREADS, FX::MINB)
mr_fixed_forward_kernel(const void *__restrict__ x, int f64, int n, float2 *__restrict__ spec,
                        const float2 *__restrict__ twN, int C) {
    extern __shared__ float2 mrsm[];
    constexpr int N = FX::N;
    RowSlot rs;
    rs.rr = (int)threadIdx.x / FX::T;
    rs.j = (int)threadIdx.x - rs.rr * FX::T;
    rs.active = rs.rr < FX::ROWS && (int)blockIdx.x * FX::ROWS + rs.rr < C;
    const int row = rs.active ? (int)blockIdx.x * FX::ROWS + rs.rr : 0;
    const int rr = rs.rr < FX::ROWS ? rs.rr : 0;
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
    mr_row_fixed<FX, -1>(sm, twN, rs.j, rs.active, false, load, none);
    if (rs.active) {
#pragma unroll 4
        for (int t = rs.j; t < N; t += FX::T) out[t] = *CWT_SMEM(&sm[spad2(t)]);
    }
}

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
