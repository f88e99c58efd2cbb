// smooth_device.cuh -- the device side of the fixed-length smooth kernels
// (Section "Fast Fourier transform"; Eq. 2 per row): the row arguments, the
// fused band product / inverse FFT / epilogue of one (channel, scale) row,
// and the fixed-length scale-block and forward kernels.  It includes no host
// or standard-library header, so that the plan-time compiler (jit.cu) can
// build these kernels for a length that has none compiled in; the library's
// own translation units reach it through smooth_kernel.cuh.
#pragma once

#include "mixed_radix.cuh"
#include "phase.cuh"

namespace cwtk {

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
            // four steps in flight; streaming stores (st.global.cs): the outputs are
            // written once and not read again here (0.2199 against 0.2232 ms at N = 10000)
#pragma unroll 4
            for (int o = rs.j; o < n_out; o += T, src += step) {
                const float2 v = *CWT_SMEM(src);
                if (a.out_c) __stcs(oc + o, v);
                if (a.out_p) __stcs(op + o, fmaf(v.x, v.x, v.y * v.y));
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

}  // namespace cwtk
