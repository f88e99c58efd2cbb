// fft_kernels.cu -- forward FFT of every channel, and the generic batched FFT.
//
// Eq. 2 of arXiv 2506.07793 needs one forward FFT per channel of the
// zero-padded signal (Section "Fourier transformed formula"); the zero padding
// of Section "Fast Fourier transform" happens in the load (indices >= n read
// as zero), so no padded copy of the signal exists in memory.  The full
// N-point spectrum is kept (the inverse stage reads arbitrary bands, including
// negative frequencies) in the plan's workspace, where it stays L2-resident
// for the scale-block kernel that follows.
#include <cuda_runtime.h>

#include "fft_core.cuh"
#include "internal.h"

namespace cwtk {

namespace {

template <int N, typename IO>
__global__ void __launch_bounds__(RowConfig<N>::THREADS)
forward_kernel(const IO *__restrict__ x, int C, int n, float2 *__restrict__ spec,
               const float2 *__restrict__ tw) {
    using RC = RowConfig<N>;
    extern __shared__ float2 smem2[];
    const int rl = threadIdx.x / RC::T, j = threadIdx.x % RC::T;
    const int row = blockIdx.x * RC::ROWS + rl;
    const bool act = row < C;
    float2 *sm = smem2 + rl * FftShape<N, RC::R>::SMEM_F2;
    const IO *xr = x + (size_t)(act ? row : 0) * (size_t)n;
    float2 *out = spec + (size_t)(act ? row : 0) * (size_t)N;
    auto load = [&](int i) -> float2 {
        return make_float2((act && i < n) ? (float)xr[i] : 0.f, 0.f);
    };
    auto store = [&](int t, float2 v) {
        if (act) out[t] = v;
    };
    fft_row<N, RC::R, -1>(sm, tw, j, load, store);
}

template <int N, int SIGN>
__global__ void __launch_bounds__(RowConfig<N>::THREADS)
fft_kernel(const float2 *in, float2 *out, int batch, const float2 *__restrict__ tw) {
    using RC = RowConfig<N>;
    extern __shared__ float2 smem2[];
    const int rl = threadIdx.x / RC::T, j = threadIdx.x % RC::T;
    const int row = blockIdx.x * RC::ROWS + rl;
    const bool act = row < batch;
    float2 *sm = smem2 + rl * FftShape<N, RC::R>::SMEM_F2;
    const float2 *ir = in + (size_t)(act ? row : 0) * N;
    float2 *orow = out + (size_t)(act ? row : 0) * N;
    auto load = [&](int i) -> float2 { return act ? ir[i] : make_float2(0.f, 0.f); };
    auto store = [&](int t, float2 v) {
        if (act) orow[t] = v;
    };
    fft_row<N, RC::R, SIGN>(sm, tw, j, load, store);
}

template <int N, typename IO>
cudaError_t forward_n(const void *x, int C, int n, float2 *spec, const float2 *tw, cudaStream_t st) {
    using RC = RowConfig<N>;
    static std::atomic<unsigned> attr_done{0};
    cudaError_t e = ensure_smem_attr(forward_kernel<N, IO>, RC::SMEM_BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int grid = (C + RC::ROWS - 1) / RC::ROWS;
    forward_kernel<N, IO><<<grid, RC::THREADS, RC::SMEM_BYTES, st>>>((const IO *)x, C, n, spec, tw);
    return cudaGetLastError();
}

template <int N, int SIGN>
cudaError_t fft_n(const float2 *in, float2 *out, int batch, const float2 *tw, cudaStream_t st) {
    using RC = RowConfig<N>;
    static std::atomic<unsigned> attr_done{0};
    cudaError_t e = ensure_smem_attr(fft_kernel<N, SIGN>, RC::SMEM_BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int grid = (batch + RC::ROWS - 1) / RC::ROWS;
    fft_kernel<N, SIGN><<<grid, RC::THREADS, RC::SMEM_BYTES, st>>>(in, out, batch, tw);
    return cudaGetLastError();
}

template <typename IO>
cudaError_t forward_dispatch(int log2n, const void *x, int C, int n, float2 *spec, const float2 *tw,
                             cudaStream_t st) {
    switch (log2n) {
        case 5: return forward_n<1 << 5, IO>(x, C, n, spec, tw, st);
        case 6: return forward_n<1 << 6, IO>(x, C, n, spec, tw, st);
        case 7: return forward_n<1 << 7, IO>(x, C, n, spec, tw, st);
        case 8: return forward_n<1 << 8, IO>(x, C, n, spec, tw, st);
        case 9: return forward_n<1 << 9, IO>(x, C, n, spec, tw, st);
        case 10: return forward_n<1 << 10, IO>(x, C, n, spec, tw, st);
        case 11: return forward_n<1 << 11, IO>(x, C, n, spec, tw, st);
        case 12: return forward_n<1 << 12, IO>(x, C, n, spec, tw, st);
        case 13: return forward_n<1 << 13, IO>(x, C, n, spec, tw, st);
        case 14: return forward_n<1 << 14, IO>(x, C, n, spec, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int SIGN>
cudaError_t fft_dispatch(int log2n, const float2 *in, float2 *out, int batch, const float2 *tw,
                         cudaStream_t st) {
    switch (log2n) {
        case 5: return fft_n<1 << 5, SIGN>(in, out, batch, tw, st);
        case 6: return fft_n<1 << 6, SIGN>(in, out, batch, tw, st);
        case 7: return fft_n<1 << 7, SIGN>(in, out, batch, tw, st);
        case 8: return fft_n<1 << 8, SIGN>(in, out, batch, tw, st);
        case 9: return fft_n<1 << 9, SIGN>(in, out, batch, tw, st);
        case 10: return fft_n<1 << 10, SIGN>(in, out, batch, tw, st);
        case 11: return fft_n<1 << 11, SIGN>(in, out, batch, tw, st);
        case 12: return fft_n<1 << 12, SIGN>(in, out, batch, tw, st);
        case 13: return fft_n<1 << 13, SIGN>(in, out, batch, tw, st);
        case 14: return fft_n<1 << 14, SIGN>(in, out, batch, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_forward(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    if (p->mr) return launch_forward_mr(p, signal, st);
    const int log2n = ilog2c(p->N);
    if (log2n > kMaxFftLog2) return launch_forward_cluster(p, signal, st);
    if (p->io == CWT_DTYPE_F64)
        return forward_dispatch<double>(log2n, signal, p->C, p->n, p->spec, p->tw, st);
    return forward_dispatch<float>(log2n, signal, p->C, p->n, p->spec, p->tw, st);
}

cudaError_t launch_fft(const float2 *in, float2 *out, int log2n, int batch, int sign,
                       const float2 *tw, cudaStream_t st) {
    if (log2n > kMaxFftLog2) return launch_fft_cluster(in, out, log2n, batch, sign, tw, st);
    if (sign < 0) return fft_dispatch<-1>(log2n, in, out, batch, tw, st);
    return fft_dispatch<+1>(log2n, in, out, batch, tw, st);
}

}  // namespace cwtk
