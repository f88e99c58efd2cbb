// smooth_fwd.cu -- forward FFT of each zero-padded channel for 2,3,5,7-smooth
// padded lengths (Section "Fast Fourier transform"; Eq. 2: one forward FFT per
// channel), on the mixed-radix rows of mixed_radix.cuh.  Kept apart from
// smooth.cu (the scale block and the schedule) so that the two compile in
// parallel.
#include <cuda_runtime.h>

#include "internal.h"
#include "mixed_radix.cuh"

namespace cwtk {

int mr_launch_rows(const MrSchedule &sch, int total_rows);

namespace {


// Forward FFT of each zero-padded channel (float32 or float64 samples).
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
    mr_row<-1>(sch, sm, twN, rs.j, rs.active, false, load, none);
    if (rs.active) {
#pragma unroll 4
        for (int t = rs.j; t < N; t += sch.T) out[t] = sm[spad2(t)];
    }
}

}  // namespace

cudaError_t launch_forward_mr(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    static unsigned done = 0;
    constexpr int kMaxSmem = (kMaxFft + (kMaxFft >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(mr_forward_kernel, kMaxSmem, &done);
    if (e != cudaSuccess) return e;
    const int rows = mr_launch_rows(p->sch, p->C);
    const int smem = rows * (p->N + (p->N >> 4)) * 8;
    const int threads = (rows * p->sch.T + 31) & ~31;
    mr_forward_kernel<<<(p->C + rows - 1) / rows, threads, smem, st>>>(
        signal, p->io == CWT_DTYPE_F64, p->n, p->spec, p->twN, p->sch, rows, p->C);
    return cudaGetLastError();
}

}  // namespace cwtk
