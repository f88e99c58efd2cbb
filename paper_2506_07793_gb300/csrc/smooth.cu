// smooth.cu -- forward FFT and fused scale block for 2,3,5,7-smooth padded
// lengths (the padding policy of Section "Fast Fourier transform" of arXiv
// 2506.07793), one row per CTA (mixed_radix.cuh).  The
// arithmetic per row is that of fft_kernels.cu and scale_block.cu (Eq. 2);
// only the FFT length and its radices differ.
#include <cuda_runtime.h>

#include "internal.h"
#include "mixed_radix.cuh"

namespace cwtk {

namespace {

__global__ void twiddle_n_kernel(float2 *tw, int N) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < N) {
        double s, c;
        sincospi(2.0 * (double)m / (double)N, &s, &c);
        tw[m] = make_float2((float)c, (float)s);
    }
}

template <typename IO, bool PP>
__global__ void __launch_bounds__(PP ? kMrThreadsPP : kMrThreads, 1)
mr_forward_kernel(const IO *__restrict__ x, int n, int N, float2 *__restrict__ spec,
                  const float2 *__restrict__ twN, const MrSchedule sch) {
    extern __shared__ float2 mrsm[];
    const int row = blockIdx.x;
    const IO *xr = x + (size_t)row * n;
    float2 *out = spec + (size_t)row * N;
    auto load = [&](int i) -> float2 { return make_float2(i < n ? (float)xr[i] : 0.f, 0.f); };
    auto store = [&](int t, float2 v) { out[t] = v; };
    mr_row<-1, PP>(mrsm, twN, N, sch, load, store);
}

template <typename IO> struct IO2m;
template <> struct IO2m<float> { using type = float2; };
template <> struct IO2m<double> { using type = double2; };

__device__ __noinline__ void mr_phase_f(float *dst, float2 v) { *dst = atan2f(v.y, v.x); }
__device__ __noinline__ void mr_phase_d(double *dst, float2 v) { *dst = (double)atan2f(v.y, v.x); }
__device__ __forceinline__ void mr_phase(float *dst, float2 v) { mr_phase_f(dst, v); }
__device__ __forceinline__ void mr_phase(double *dst, float2 v) { mr_phase_d(dst, v); }

struct MrArgs {
    const float2 *spec;
    const float *bank;
    const int *band;
    const float2 *twN;
    void *out_c, *out_p, *out_ph;
    int S, N, n_out, sub;
};

template <typename IO, bool PP>
__global__ void __launch_bounds__(PP ? kMrThreadsPP : kMrThreads, 1)
mr_scale_block_kernel(const MrArgs a, const MrSchedule sch) {
    using V2 = typename IO2m<IO>::type;
    extern __shared__ float2 mrsm[];
    const int row = blockIdx.x;
    const int c = row / a.S, s = row - c * a.S;
    const int N = a.N;
    const float2 *X = a.spec + (size_t)c * N;
    const float *W = a.bank + (size_t)s * N;
    const int b0 = a.band[2 * s], B = a.band[2 * s + 1];
    auto load = [&](int k) -> float2 {
        int dk = k - b0;  // band is [b0, b0 + B) modulo N
        if (dk < 0) dk += N;
        if (dk < B) {
            const float2 xv = X[k];
            const float w = W[k];
            return make_float2(xv.x * w, xv.y * w);
        }
        return make_float2(0.f, 0.f);
    };
    const size_t obase = (size_t)row * (size_t)a.n_out;
    V2 *oc = (V2 *)a.out_c;
    IO *op = (IO *)a.out_p;
    IO *oph = (IO *)a.out_ph;
    const int sub = a.sub, n_out = a.n_out;
    auto store = [&](int t, float2 v) {
        int o = t;
        if (sub != 1) {
            if (t % sub) return;
            o = t / sub;
        }
        if (o >= n_out) return;
        if (oc) {
            V2 z;
            z.x = (IO)v.x;
            z.y = (IO)v.y;
            oc[obase + o] = z;
        }
        if (op) op[obase + o] = (IO)fmaf(v.x, v.x, v.y * v.y);
        if (oph) mr_phase(oph + obase + o, v);
    };
    mr_row<+1, PP>(mrsm, a.twN, N, sch, load, store);
}

size_t mr_smem(int N) {
    return sizeof(float2) * (size_t)(N + (N >> 4)) * (N <= kMrPingPongMax ? 2 : 1);
}

template <typename K>
cudaError_t mr_attr(K *kernel, unsigned *done) {
    return ensure_smem_attr(kernel, (int)mr_smem(kMrPingPongMax), done);
}

template <typename IO, bool PP>
cudaError_t mr_forward_t(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    static unsigned done = 0;
    cudaError_t e = mr_attr(mr_forward_kernel<IO, PP>, &done);
    if (e != cudaSuccess) return e;
    mr_forward_kernel<IO, PP><<<p->C, PP ? kMrThreadsPP : kMrThreads, mr_smem(p->N), st>>>(
        (const IO *)signal, p->n, p->N, p->spec, p->twN, p->sch);
    return cudaGetLastError();
}

template <typename IO, bool PP>
cudaError_t mr_sb_t(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st) {
    static unsigned done = 0;
    cudaError_t e = mr_attr(mr_scale_block_kernel<IO, PP>, &done);
    if (e != cudaSuccess) return e;
    mr_scale_block_kernel<IO, PP><<<p->C * p->S, PP ? kMrThreadsPP : kMrThreads, mr_smem(p->N), st>>>(a, p->sch);
    return cudaGetLastError();
}

}  // namespace

bool mr_schedule(int N, MrSchedule *out) {
    int x = N, e2 = 0, e3 = 0, e5 = 0, e7 = 0;
    while (x % 2 == 0) x /= 2, ++e2;
    while (x % 3 == 0) x /= 3, ++e3;
    while (x % 5 == 0) x /= 5, ++e5;
    while (x % 7 == 0) x /= 7, ++e7;
    if (x != 1 || N < kMinFft || N > kMaxFft) return false;
    MrSchedule s{};
    while (e2 >= 4 && s.np < kMrMaxPasses) s.radix[s.np++] = 16, e2 -= 4;
    if (e2 && s.np < kMrMaxPasses) s.radix[s.np++] = 1 << e2;
    for (int i = 0; i < e3 && s.np < kMrMaxPasses; ++i) s.radix[s.np++] = 3;
    for (int i = 0; i < e5 && s.np < kMrMaxPasses; ++i) s.radix[s.np++] = 5;
    for (int i = 0; i < e7 && s.np < kMrMaxPasses; ++i) s.radix[s.np++] = 7;
    // each thread holds at most kMrPoints values: N / R butterflies must fit
    // in (kMrPoints / R) per thread
    for (int p = 0; p < s.np; ++p) {
        const int R = s.radix[p];
        const int per = kMrPoints / R > 0 ? kMrPoints / R : 1;
        if (N / R > per * kMrThreads) return false;
    }
    *out = s;
    return true;
}

cudaError_t make_twiddles_n(int N, float2 *tw, cudaStream_t st) {
    twiddle_n_kernel<<<(N + 255) / 256, 256, 0, st>>>(tw, N);
    return cudaGetLastError();
}

cudaError_t launch_forward_mr(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    const bool pp = p->N <= kMrPingPongMax;
    if (p->io == CWT_DTYPE_F64)
        return pp ? mr_forward_t<double, true>(p, signal, st) : mr_forward_t<double, false>(p, signal, st);
    return pp ? mr_forward_t<float, true>(p, signal, st) : mr_forward_t<float, false>(p, signal, st);
}

cudaError_t launch_scale_block_mr(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                  cudaStream_t st) {
    MrArgs a;
    a.spec = p->spec;
    a.bank = p->bank;
    a.band = p->band;
    a.twN = p->twN;
    a.out_c = out_c;
    a.out_p = out_p;
    a.out_ph = out_ph;
    a.S = p->S;
    a.N = p->N;
    a.n_out = p->n_out;
    a.sub = p->d;
    const bool pp = p->N <= kMrPingPongMax;
    if (p->io == CWT_DTYPE_F64)
        return pp ? mr_sb_t<double, true>(p, a, st) : mr_sb_t<double, false>(p, a, st);
    return pp ? mr_sb_t<float, true>(p, a, st) : mr_sb_t<float, false>(p, a, st);
}

}  // namespace cwtk
