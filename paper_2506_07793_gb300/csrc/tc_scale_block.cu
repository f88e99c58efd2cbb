// tc_scale_block.cu -- the fused scale block with its inverse FFT's radix
// stages on the tensor cores (FP16 or BF16 operands, hi/lo compensation, FP32
// accumulation; see fft_tc.cuh), for rows of N = 16384 ... 131072 points.
//
// Per (channel, scale) row the arithmetic is that of cluster.cu (Eq. 2:
// band product, inverse FFT, reduction to complex / power / phase): the row
// runs on a cluster of CL = N / 16384 CTAs, CTA c transforms the residue
// class k = c + CL m of the banded spectrum (16384 points, fft_tc.cuh) and one
// cross-CTA radix-CL stage over distributed shared memory finishes the row
// (fft_cluster.cuh's decomposition).  N = 16384 runs on single CTAs.
//
// Range (FP16): the row's spectrum Y = X W is scaled by 2^e with
// e = 15 - ceil(log2 U), U = 2 max_k max(|Re X_k|, |Im X_k|) sum_k |W_k| >= sum_k |Y_k|,
// which bounds every intermediate of the FFT by 2^15 (< 65504); outputs are
// unscaled exactly (complex by 2^-e, power by 2^-2e; the phase is unchanged).
// The per-channel maxima come from tc_chmax_kernel after the forward FFT and
// the per-scale sums from tc_wl1_kernel at plan creation.  BF16 has FP32's
// exponent range; it takes the same exact scaling.
#include <cuda_runtime.h>

#include "fft_cluster.cuh"
#include "fft_tc.cuh"
#include "internal.h"
#include "phase.cuh"

namespace cwtk {

namespace {

template <typename IO> struct TcIO2;
template <> struct TcIO2<float> { using type = float2; };
template <> struct TcIO2<double> { using type = double2; };

struct TcArgs {
    const float2 *spec;   // [C][N] forward spectra
    const float *bank;    // [S][N] W_s / N
    const int *band;      // [S][2]
    const float *chmax;   // [C] max_k max(|Re X|, |Im X|)
    const float *wl1;     // [S] sum_k |W_s[k]| over the band
    const float2 *tw;
    void *out_c, *out_p, *out_ph;
    int S, n_out, sub;
};

// Exact power-of-two scale of one row (see the file comment).
__device__ __forceinline__ int tc_row_exponent(float chmax, float wl1) {
    const float U = 2.f * chmax * wl1;
    if (!(U > 0.f) || !(U < 3.0e38f)) return 0;
    int ex = 0;
    frexpf(U, &ex);  // U < 2^ex
    return max(-120, min(120, 15 - ex));
}

template <int CL, class T, typename IO>
__device__ __forceinline__ void tc_row(const TcArgs &a, float2 *sm, int row, int rank) {
    using V2 = typename TcIO2<IO>::type;
    constexpr int N = CL * kTcNL;
    const int c = row / a.S, s = row - c * a.S;
    const float2 *X = a.spec + (size_t)c * N;
    const float *W = a.bank + (size_t)s * N;
    const int b0 = a.band[2 * s], B = a.band[2 * s + 1];
    const int ex = tc_row_exponent(a.chmax[c], a.wl1[s]);
    const float sc = ldexpf(1.f, ex), inv = ldexpf(1.f, -ex), inv2 = inv * inv;
    // residue class `rank`: local point m is global bin rank + CL m
    auto load = [&](int m) -> float2 {
        const int k = rank + CL * m;
        if (((k - b0) & (N - 1)) < B) {
            const float2 x = X[k];
            const float w = W[k] * sc;
            return make_float2(x.x * w, x.y * w);
        }
        return make_float2(0.f, 0.f);
    };
    // Narrow band: the class holds Bm consecutive (cyclic) in-band m from
    // m_first; with Bm <= 4096 every radix-4 butterfly {j + 4096 r} of pass 0
    // meets at most one of them.
    constexpr int Q = kTcNL / 4;
    const int delta = (rank - b0) & (CL - 1);
    const int Bm = delta < B ? (B - delta + CL - 1) / CL : 0;
    const int m_first = ((((b0 + delta) & (N - 1)) - rank) / CL) & (kTcNL - 1);
    // Branch-free: a butterfly with no in-band input reads bin `rank` (in
    // bounds, the same address for every such lane) and returns x = 0.
    auto first = [&](int j, int &r, float2 &x) {
        const int d0 = (j - m_first) & (Q - 1);
        const bool in = d0 < Bm;
        const int m = (m_first + d0) & (kTcNL - 1);
        r = (m - j) >> 12;  // m = j + r Q when in band (Q = 4096)
        const int k = CWT_IDX(in ? rank + CL * m : rank, N);
        const float2 xv = X[k];
        const float w = in ? W[k] * sc : 0.f;
        x = make_float2(xv.x * w, xv.y * w);
    };
    float2 *tab = sm + kTcNL;
    tc_fill_twiddles<+1>(tab, a.tw);
    __syncthreads();
    tc_fft16384<T, +1>(sm, tab, Bm <= Q, load, first);

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
            z.x = (IO)(v.x * inv);
            z.y = (IO)(v.y * inv);
            oc[obase + o] = z;
        }
        if (op) op[obase + o] = (IO)(fmaf(v.x, v.x, v.y * v.y) * inv2);
        if (oph) {
            const float ph = phase_atan2(v.y, v.x);
            oph[obase + o] = (IO)ph;
        }
    };
    // cross-CTA radix-CL stage: X[t1 + NL t2] = sum_c w_CL^(c t2) w_N^(c t1) A_c[t1]
    if constexpr (CL > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
#pragma unroll 1
        for (int q = 0; q < kTcNL / CL / kTcThreads; ++q) {
            const int t1 = rank * (kTcNL / CL) + q * kTcThreads + (int)threadIdx.x;
            float2 v[CL];
#pragma unroll
            for (int cc = 0; cc < CL; ++cc) v[cc] = ld_cluster(CWT_SMEM(&sm[tc_pad(t1)]), (unsigned)cc);
#pragma unroll
            for (int cc = 1; cc < CL; ++cc) v[cc] = cmul(v[cc], __ldg(&a.tw[(cc * t1) * (kTwN / N)]));
            dft<CL, +1>(v);
            if (sub == 1) {  // no decimation: output o = t, one crop test per output
#pragma unroll
                for (int t2 = 0; t2 < CL; ++t2) {
                    const int o = t1 + kTcNL * t2;
                    if (o < n_out) {
                        if (op) op[obase + o] = (IO)(fmaf(v[t2].x, v[t2].x, v[t2].y * v[t2].y) * inv2);
                        if (oph) oph[obase + o] = (IO)phase_atan2(v[t2].y, v[t2].x);
                        if (oc) {
                            V2 z;
                            z.x = (IO)(v[t2].x * inv);
                            z.y = (IO)(v[t2].y * inv);
                            oc[obase + o] = z;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int t2 = 0; t2 < CL; ++t2) store(t1 + kTcNL * t2, v[t2]);
            }
        }
        cl.sync();  // no CTA still reads this CTA's buffer
    } else {
#pragma unroll 4
        for (int q = 0; q < kTcNL / kTcThreads; ++q) {
            const int t1 = q * kTcThreads + (int)threadIdx.x;
            store(t1, *CWT_SMEM(&sm[tc_pad(t1)]));
        }
    }
}

template <int CL, class T, typename IO>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kTcThreads, 1)
tc_scale_block_cluster_kernel(const TcArgs a) {
    extern __shared__ float2 tcsm[];
    const int rank = (int)cg::this_cluster().block_rank();
    tc_row<CL, T, IO>(a, tcsm, blockIdx.x / CL, rank);
}

template <class T, typename IO>
__global__ void __launch_bounds__(kTcThreads, 1) tc_scale_block_kernel(const TcArgs a) {
    extern __shared__ float2 tcsm[];
    tc_row<1, T, IO>(a, tcsm, blockIdx.x, 0);
}

constexpr int kTcSmemBytes = (kTcNL + kTcTabF2) * (int)sizeof(float2);  // the row + twiddles, 147.3 KB

// chmax[c] = max_k max(|Re X_c[k]|, |Im X_c[k]|): one CTA per channel.
__global__ void __launch_bounds__(512) tc_chmax_kernel(const float2 *__restrict__ spec, int N,
                                                        float *__restrict__ chmax) {
    __shared__ float red[512];
    const float2 *X = spec + (size_t)blockIdx.x * N;
    float m = 0.f;
    for (int k = threadIdx.x; k < N; k += 512) {
        const float2 v = X[k];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 256; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) chmax[blockIdx.x] = red[0];
}

// wl1[s] = sum over the band of |W_s[k]| (fixed-order tree): one CTA per scale.
__global__ void __launch_bounds__(256) tc_wl1_kernel(const float *__restrict__ bank,
                                                     const int *__restrict__ band, int N,
                                                     float *__restrict__ wl1) {
    __shared__ float red[256];
    const int s = blockIdx.x;
    const int b0 = band[2 * s], B = band[2 * s + 1];
    const float *W = bank + (size_t)s * N;
    float acc = 0.f;
    for (int j = threadIdx.x; j < B; j += 256) acc += fabsf(W[(b0 + j) & (N - 1)]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    // rounding of the sum is covered: the bound keeps a factor 2 of headroom
    if (threadIdx.x == 0) wl1[s] = red[0];
}

template <int CL, class T, typename IO>
cudaError_t tc_launch_n(const TcArgs &a, int rows, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    if constexpr (CL > 1) {
        auto *k = tc_scale_block_cluster_kernel<CL, T, IO>;
        cudaError_t e = ensure_smem_attr(k, kTcSmemBytes, &done);
        if (e != cudaSuccess) return e;
        k<<<rows * CL, kTcThreads, kTcSmemBytes, st>>>(a);
    } else {
        auto *k = tc_scale_block_kernel<T, IO>;
        cudaError_t e = ensure_smem_attr(k, kTcSmemBytes, &done);
        if (e != cudaSuccess) return e;
        k<<<rows, kTcThreads, kTcSmemBytes, st>>>(a);
    }
    return cudaGetLastError();
}

template <class T, typename IO>
cudaError_t tc_dispatch(int log2n, const TcArgs &a, int rows, cudaStream_t st) {
    switch (log2n) {
        case 14: return tc_launch_n<1, T, IO>(a, rows, st);
        case 15: return tc_launch_n<2, T, IO>(a, rows, st);
        case 16: return tc_launch_n<4, T, IO>(a, rows, st);
        case 17: return tc_launch_n<8, T, IO>(a, rows, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_tc_row_bounds(const cwt_plan_s *p, cudaStream_t st) {
    tc_chmax_kernel<<<p->C, 512, 0, st>>>(p->spec, p->N, p->tc_chmax);
    return cudaGetLastError();
}

cudaError_t launch_tc_wl1(const cwt_plan_s *p, cudaStream_t st) {
    tc_wl1_kernel<<<p->S, 256, 0, st>>>(p->bank, p->band, p->N, p->tc_wl1);
    return cudaGetLastError();
}

cudaError_t launch_scale_block_tc(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                  cudaStream_t st) {
    TcArgs a;
    a.spec = p->spec;
    a.bank = p->bank;
    a.band = p->band;
    a.chmax = p->tc_chmax;
    a.wl1 = p->tc_wl1;
    a.tw = p->tw;
    a.out_c = out_c;
    a.out_p = out_p;
    a.out_ph = out_ph;
    a.S = p->S;
    a.n_out = p->n_out;
    a.sub = p->d;  // no spectral fold on this path
    const int rows = p->C * p->S;
    const int log2n = ilog2c(p->N);
    const bool bf = p->precision == CWT_PREC_TC_BF16;
    if (p->io == CWT_DTYPE_F64)
        return bf ? tc_dispatch<TcBF16, double>(log2n, a, rows, st)
                  : tc_dispatch<TcF16, double>(log2n, a, rows, st);
    return bf ? tc_dispatch<TcBF16, float>(log2n, a, rows, st)
              : tc_dispatch<TcF16, float>(log2n, a, rows, st);
}

}  // namespace cwtk
