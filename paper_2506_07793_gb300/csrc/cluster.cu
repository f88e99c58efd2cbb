// cluster.cu -- forward FFT, fused scale block and generic FFT for rows of
// 32768 to 131072 points, each row on a thread-block cluster of 2-8 CTAs (see
// fft_cluster.cuh: per-CTA residue-class FFTs plus one cross-CTA stage).  The
// arithmetic per row is that of fft_kernels.cu and scale_block.cu (Eq. 2:
// forward FFT per channel; band product, inverse FFT and reduction per
// (channel, scale) row).
#include <cuda_runtime.h>

#include "fft_cluster.cuh"
#include "internal.h"
#include "phase.cuh"

namespace cwtk {

namespace {

template <typename IO> struct IO2c;
template <> struct IO2c<float> { using type = float2; };
template <> struct IO2c<double> { using type = double2; };

__device__ __forceinline__ void cl_store_phase_f(float *dst, float2 v) { *dst = phase_atan2(v.y, v.x); }
__device__ __forceinline__ void cl_store_phase_d(double *dst, float2 v) { *dst = (double)phase_atan2(v.y, v.x); }
__device__ __forceinline__ void cl_store_phase(float *dst, float2 v) { cl_store_phase_f(dst, v); }
__device__ __forceinline__ void cl_store_phase(double *dst, float2 v) { cl_store_phase_d(dst, v); }

template <int N, typename IO>
__global__ void __cluster_dims__(N / kClPoints, 1, 1) __launch_bounds__(kClThreads, 1)
cl_forward_kernel(const IO *__restrict__ x, int n, float2 *__restrict__ spec,
                  const float2 *__restrict__ tw) {
    extern __shared__ float2 clsm[];
    constexpr int CL = ClusterShape<N>::CL;
    const int row = blockIdx.x / CL;
    const IO *xr = x + (size_t)row * n;
    float2 *out = spec + (size_t)row * N;
    auto load = [&](int i) -> float2 { return make_float2(i < n ? (float)xr[i] : 0.f, 0.f); };
    auto store = [&](int t, float2 v) { out[t] = v; };
    fft_cluster_row<N, -1>(clsm, tw, load, store);
}

template <int N, int SIGN>
__global__ void __cluster_dims__(N / kClPoints, 1, 1) __launch_bounds__(kClThreads, 1)
cl_fft_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw) {
    extern __shared__ float2 clsm[];
    constexpr int CL = ClusterShape<N>::CL;
    const int row = blockIdx.x / CL;
    const float2 *ir = in + (size_t)row * N;
    float2 *orow = out + (size_t)row * N;
    auto load = [&](int i) -> float2 { return ir[i]; };
    auto store = [&](int t, float2 v) { orow[t] = v; };
    // every input is read before the cluster barrier inside fft_cluster_row,
    // so `out` may alias `in`
    fft_cluster_row<N, SIGN>(clsm, tw, load, store);
}

struct ClArgs {
    const float2 *spec;
    const float *bank;
    const int *band;
    const float2 *tw;
    void *out_c, *out_p, *out_ph;
    int S, n_out, sub;
};

// PLAIN: no decimation (output o = t), so each output needs only the crop
// test; the general form also keeps t = 0 (mod sub).
template <int N, typename IO, bool PLAIN>
__global__ void __cluster_dims__(N / kClPoints, 1, 1) __launch_bounds__(kClThreads, 1)
cl_scale_block_kernel(const ClArgs a) {
    using V2 = typename IO2c<IO>::type;
    extern __shared__ float2 clsm[];
    constexpr int CL = ClusterShape<N>::CL;
    const int row = blockIdx.x / CL;
    const int c = row / a.S, s = row - c * a.S;
    const float2 *X = a.spec + (size_t)c * N;
    const float *W = a.bank + (size_t)s * N;
    const int b0 = a.band[2 * s], B = a.band[2 * s + 1];
    auto load = [&](int k) -> float2 {
        if (((k - b0) & (N - 1)) < B) {
            const float2 x = X[k];
            const float w = W[k];
            return make_float2(x.x * w, x.y * w);
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
        if constexpr (!PLAIN) {
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
        if (oph) cl_store_phase(oph + obase + o, v);
    };
    // Narrow band: this CTA's residue class k = rank + CL m holds Bm
    // consecutive (cyclic) in-band m, starting at m_first; if Bm <= NL/R0 each
    // local pass-0 butterfly {jj + r NL/R0} meets at most one of them.
    constexpr int NL = ClusterShape<N>::NL;
    constexpr int Q = NL / FftShape<NL, kClR>::R0;
    const int rank = (int)cg::this_cluster().block_rank();
    const int delta = (rank - b0) & (CL - 1);
    const int Bm = delta < B ? (B - delta + CL - 1) / CL : 0;
    const int m_first = ((((b0 + delta) & (N - 1)) - rank) / CL) & (NL - 1);
    auto first = [&](int jj, int &r, float2 &x) -> bool {
        const int d0 = (jj - m_first) & (Q - 1);
        if (d0 >= Bm) return false;
        const int m = (m_first + d0) & (NL - 1);
        r = (m - jj) / Q;
        const int k = rank + CL * m;
        const float2 xv = X[k];
        const float w = W[k];
        x = make_float2(xv.x * w, xv.y * w);
        return true;
    };
    fft_cluster_row<N, +1>(clsm, a.tw, load, Bm <= Q, first, store);
}

template <typename K>
cudaError_t cl_attr(K *kernel, int bytes, std::atomic<unsigned> *done) {
    cudaError_t e = ensure_smem_attr(kernel, bytes, done);
    if (e == cudaSuccess) {
        // clusters of 8 are portable; nothing larger is requested
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
    }
    return e;
}

template <int N, typename IO>
cudaError_t cl_forward_n(const void *x, int C, int n, float2 *spec, const float2 *tw, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    cudaError_t e = cl_attr(cl_forward_kernel<N, IO>, ClusterShape<N>::SMEM_BYTES, &done);
    if (e != cudaSuccess) return e;
    cl_forward_kernel<N, IO><<<C * ClusterShape<N>::CL, kClThreads, ClusterShape<N>::SMEM_BYTES, st>>>(
        (const IO *)x, n, spec, tw);
    return cudaGetLastError();
}

template <int N, typename IO, bool PLAIN>
cudaError_t cl_sb_nk(const ClArgs &a, int rows, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    cudaError_t e = cl_attr(cl_scale_block_kernel<N, IO, PLAIN>, ClusterShape<N>::SMEM_BYTES, &done);
    if (e != cudaSuccess) return e;
    cl_scale_block_kernel<N, IO, PLAIN>
        <<<rows * ClusterShape<N>::CL, kClThreads, ClusterShape<N>::SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

template <int N, typename IO>
cudaError_t cl_sb_n(const ClArgs &a, int rows, cudaStream_t st) {
    return a.sub == 1 ? cl_sb_nk<N, IO, true>(a, rows, st) : cl_sb_nk<N, IO, false>(a, rows, st);
}

template <int N, int SIGN>
cudaError_t cl_fft_n(const float2 *in, float2 *out, int batch, const float2 *tw, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    cudaError_t e = cl_attr(cl_fft_kernel<N, SIGN>, ClusterShape<N>::SMEM_BYTES, &done);
    if (e != cudaSuccess) return e;
    cl_fft_kernel<N, SIGN><<<batch * ClusterShape<N>::CL, kClThreads, ClusterShape<N>::SMEM_BYTES, st>>>(
        in, out, tw);
    return cudaGetLastError();
}

template <typename IO>
cudaError_t cl_forward_dispatch(int log2n, const void *x, int C, int n, float2 *spec, const float2 *tw,
                                cudaStream_t st) {
    switch (log2n) {
        case 15: return cl_forward_n<1 << 15, IO>(x, C, n, spec, tw, st);
        case 16: return cl_forward_n<1 << 16, IO>(x, C, n, spec, tw, st);
        case 17: return cl_forward_n<1 << 17, IO>(x, C, n, spec, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename IO>
cudaError_t cl_sb_dispatch(int log2n, const ClArgs &a, int rows, cudaStream_t st) {
    switch (log2n) {
        case 15: return cl_sb_n<1 << 15, IO>(a, rows, st);
        case 16: return cl_sb_n<1 << 16, IO>(a, rows, st);
        case 17: return cl_sb_n<1 << 17, IO>(a, rows, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_forward_cluster(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    const int log2n = ilog2c(p->N);
    if (p->io == CWT_DTYPE_F64)
        return cl_forward_dispatch<double>(log2n, signal, p->C, p->n, p->spec, p->tw, st);
    return cl_forward_dispatch<float>(log2n, signal, p->C, p->n, p->spec, p->tw, st);
}

cudaError_t launch_scale_block_cluster(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                       cudaStream_t st) {
    ClArgs a;
    a.spec = p->spec;
    a.bank = p->bank;
    a.band = p->band;
    a.tw = p->tw;
    a.out_c = out_c;
    a.out_p = out_p;
    a.out_ph = out_ph;
    a.S = p->S;
    a.n_out = p->n_out;
    a.sub = p->d;  // fold is 1 on this path
    const int rows = p->C * p->S;
    const int log2n = ilog2c(p->N);
    if (p->io == CWT_DTYPE_F64) return cl_sb_dispatch<double>(log2n, a, rows, st);
    return cl_sb_dispatch<float>(log2n, a, rows, st);
}

cudaError_t launch_fft_cluster(const float2 *in, float2 *out, int log2n, int batch, int sign,
                               const float2 *tw, cudaStream_t st) {
    switch (log2n * 2 + (sign > 0)) {
        case 30: return cl_fft_n<1 << 15, -1>(in, out, batch, tw, st);
        case 31: return cl_fft_n<1 << 15, +1>(in, out, batch, tw, st);
        case 32: return cl_fft_n<1 << 16, -1>(in, out, batch, tw, st);
        case 33: return cl_fft_n<1 << 16, +1>(in, out, batch, tw, st);
        case 34: return cl_fft_n<1 << 17, -1>(in, out, batch, tw, st);
        case 35: return cl_fft_n<1 << 17, +1>(in, out, batch, tw, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwtk
