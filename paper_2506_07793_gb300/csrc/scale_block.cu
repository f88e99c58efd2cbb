// scale_block.cu -- the fused hot kernel: spectrum product, inverse FFT and
// reduction of one (channel, scale) row per thread group, on chip.
//
// Eq. 2 of arXiv 2506.07793: c_s = F^-1( F(x) * Psi_s ), one inverse FFT per
// (channel, scale) row; Section "Precision" reduces the coefficients to real /
// imaginary parts, power and phase.  Per row the kernel
//   1. reads the forward spectrum X[c][k] and the wavelet bank W_s[k] only for
//      bins inside the scale's band (the rest of W_s is below 1e-10 of its
//      peak) and forms Y[k] = X[k] W_s[k] in registers (W_s carries the 1/N);
//   2. when the decimation d has a power-of-two factor f, folds the spectrum,
//          Y'[j] = sum_q Y[j + q N/f],   j < N/f,
//      so that an N/f-point inverse FFT yields exactly every f-th sample;
//   3. runs the inverse Stockham FFT (registers + shared memory);
//   4. crops to t < n, keeps t = 0 mod d, and writes only the requested
//      outputs (complex, |c|^2, atan2) with coalesced stores.
// Nothing but the outputs is written to global memory.
#include <cuda_runtime.h>

#include "fft_core.cuh"
#include "internal.h"
#include "phase.cuh"

namespace cwtk {

namespace {

struct SBArgs {
    const float2 *spec;  // [C][N]
    const float *bank;   // [S][N]
    const int *band;     // [S][2]
    const float2 *tw;
    void *out_c, *out_p, *out_ph;
    int C, S, N, n_out, fold, sub, rows;
};

template <typename IO> struct IO2;
template <> struct IO2<float> { using type = float2; };
template <> struct IO2<double> { using type = double2; };

// Keeping the phase out of line keeps the unrolled epilogue small.
template <typename IO>
__device__ __noinline__ void store_phase(IO *dst, float2 v) {
    *dst = (IO)phase_atan2(v.y, v.x);
}

template <int M, typename IO>
__global__ void __launch_bounds__(RowConfig<M>::THREADS)
scale_block_kernel(const SBArgs a) {
    using RC = RowConfig<M>;
    using V2 = typename IO2<IO>::type;
    extern __shared__ float2 smem2[];
    const int rl = threadIdx.x / RC::T, j = threadIdx.x % RC::T;
    const int row = blockIdx.x * RC::ROWS + rl;
    const bool act = row < a.rows;
    const int c = act ? row / a.S : 0;
    const int s = act ? row - c * a.S : 0;
    float2 *sm = smem2 + rl * FftShape<M, RC::R>::SMEM_F2;

    const float2 *X = a.spec + (size_t)c * (size_t)a.N;
    const float *W = a.bank + (size_t)s * (size_t)a.N;
    const int b0 = a.band[2 * s], B = act ? a.band[2 * s + 1] : 0;
    const int nmask = a.N - 1;
    const int fold = a.fold;

    // Folded input j = sum over in-band k = j (mod M).  When the band is no
    // wider than M (always for fold 1), at most one k qualifies:
    // k = b0 + ((j - b0) mod M).
    const bool narrow = B <= M;
    auto load = [&](int jj) -> float2 {
        float2 acc = make_float2(0.f, 0.f);
        if (fold == 1) {  // k = jj: addresses stay base + constant offsets
            if (((jj - b0) & nmask) < B) {
                const float2 x = X[jj];
                const float w = W[jj];
                acc = make_float2(x.x * w, x.y * w);
            }
            return acc;
        }
        if (narrow) {
            const int delta = (jj - b0) & (M - 1);
            if (delta < B) {
                const int k = (b0 + delta) & nmask;
                const float2 x = X[k];
                const float w = W[k];
                acc = make_float2(x.x * w, x.y * w);
            }
            return acc;
        }
        for (int q = 0; q < fold; ++q) {
            const int k = jj + q * M;
            if (((k - b0) & nmask) < B) {
                const float2 x = X[k];
                const float w = W[k];
                acc.x = fmaf(x.x, w, acc.x);
                acc.y = fmaf(x.y, w, acc.y);
            }
        }
        return acc;
    };

    const size_t obase = (size_t)row * (size_t)a.n_out;
    V2 *oc = (V2 *)a.out_c;
    IO *op = (IO *)a.out_p;
    IO *oph = (IO *)a.out_ph;
    const int sub = a.sub, n_out = a.n_out;
    auto store = [&](int t, float2 v) {
        if (!act) return;
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
        if (oph) store_phase(oph + obase + o, v);
    };
    // Narrow band (B <= M/R0): each pass-0 butterfly {jj + r M/R0} meets at
    // most one in-band bin, k = b0 + ((jj - b0) mod M/R0); its position r
    // follows from k's folded index k mod M = jj + r M/R0.
    constexpr int Q = M / FftShape<M, RC::R>::R0;
    float2 v[RC::R];
    if (B <= Q) {
        auto first = [&](int jj, int &r, float2 &x) -> bool {
            const int d0 = (jj - b0) & (Q - 1);
            if (d0 >= B) return false;
            const int k = (b0 + d0) & nmask;
            r = ((k & (M - 1)) - jj) / Q;
            const float2 xv = X[k];
            const float w = W[k];
            x = make_float2(xv.x * w, xv.y * w);
            return true;
        };
        fft_pass0_sparse<M, RC::R, +1>(v, j, a.tw, first);
    } else {
        fft_pass0_dense<M, RC::R, +1>(v, j, load);
    }
    fft_finish<M, RC::R, +1>(v, sm, a.tw, j, store);
}

template <int M, typename IO>
cudaError_t sb_n(const SBArgs &a, cudaStream_t st) {
    using RC = RowConfig<M>;
    static std::atomic<unsigned> attr_done{0};
    cudaError_t e = ensure_smem_attr(scale_block_kernel<M, IO>, RC::SMEM_BYTES, &attr_done);
    if (e != cudaSuccess) return e;
    const int grid = (a.rows + RC::ROWS - 1) / RC::ROWS;
    scale_block_kernel<M, IO><<<grid, RC::THREADS, RC::SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

template <typename IO>
cudaError_t sb_dispatch(int log2m, const SBArgs &a, cudaStream_t st) {
    switch (log2m) {
        case 5: return sb_n<1 << 5, IO>(a, st);
        case 6: return sb_n<1 << 6, IO>(a, st);
        case 7: return sb_n<1 << 7, IO>(a, st);
        case 8: return sb_n<1 << 8, IO>(a, st);
        case 9: return sb_n<1 << 9, IO>(a, st);
        case 10: return sb_n<1 << 10, IO>(a, st);
        case 11: return sb_n<1 << 11, IO>(a, st);
        case 12: return sb_n<1 << 12, IO>(a, st);
        case 13: return sb_n<1 << 13, IO>(a, st);
        case 14: return sb_n<1 << 14, IO>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_scale_block(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                               cudaStream_t st) {
    if (p->mr) return launch_scale_block_mr(p, out_c, out_p, out_ph, st);
    if (p->M > kMaxFft) return launch_scale_block_cluster(p, out_c, out_p, out_ph, st);
    SBArgs a;
    a.spec = p->spec;
    a.bank = p->bank;
    a.band = p->band;
    a.tw = p->tw;
    a.out_c = out_c;
    a.out_p = out_p;
    a.out_ph = out_ph;
    a.C = p->C;
    a.S = p->S;
    a.N = p->N;
    a.n_out = p->n_out;
    a.fold = p->fold;
    a.sub = p->sub;
    a.rows = p->C * p->S;
    const int log2m = ilog2c(p->M);
    if (p->io == CWT_DTYPE_F64) return sb_dispatch<double>(log2m, a, st);
    return sb_dispatch<float>(log2m, a, st);
}

}  // namespace cwtk
