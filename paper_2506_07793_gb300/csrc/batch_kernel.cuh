// batch_kernel.cuh -- shared declarations of the persistent batch kernel
// (see batch.cu for the design).  The kernel itself is instantiated in
// batch_k16.cu and batch_k32.cu (16 or 32 points per thread in the inverse
// FFTs), one instantiation per translation unit so that they compile in
// parallel; batch.cu reaches them through batch_kernel_ptr().
#pragma once

#include <cuda_runtime.h>

#include "fft_core.cuh"
#include "internal.h"
#include "phase.cuh"

namespace cwtk {

constexpr int kBThreads = 256;
constexpr int kTile = 8192;                    // points per item (G channels x N_e)
constexpr int kTileP = kTile + (kTile >> 4);   // the tile, padded: spectra / forward staging
constexpr int kMaxBatchLog2 = 13;              // N_e <= kTile

struct BatchItem {
    long long in_off;   // element offset of channel c0 of the epoch in the packed input
    long long out_off;  // element offset of row (c0, scale 0) in each packed output
    int n;              // epoch length
    int log2n;          // log2 N_e
    int G;              // channels in this item
    int pad;
};

struct BatchArgs {
    const float *in;
    float2 *oc;
    float *op;
    float *oph;
    const BatchItem *items;
    int n_items;
    int *counter;
    const float *bank[kMaxBatchLog2 + 1];  // per log2 N: [S][N]
    const int *band[kMaxBatchLog2 + 1];    // per log2 N: [S][2]
    const float2 *tw;
    int S, d;
};

// Shared memory: the item's tile (kTileP float2: the forward FFTs' padded
// staging, then the G unpadded spectra in place) + staging for the inverse
// rows, kBThreads * RI points (every thread holds RI points of some row in
// flight), padded 17/16.  With RI = 16 that is 104 KB, two CTAs per SM.
template <int RI>
constexpr int batch_smem() { return (kTileP + (kBThreads * RI) * 17 / 16) * 8; }

// Inverse length of a row of N_e = N points at decimation d: N / f, f the
// largest power of two dividing d with N / f >= kMinFft (the spectral fold).
__host__ __device__ inline int batch_inverse_length(int N, int d) {
    int fold = 1;
    while ((d % (2 * fold)) == 0 && N / (2 * fold) >= kMinFft) fold *= 2;
    return N / fold;
}

// The kernel for RI = 16 or 32 (defined in batch_k16.cu / batch_k32.cu).
const void *batch_kernel_ptr(int ri);

#ifdef CWT_BATCH_KERNELS
namespace {

__device__ __noinline__ void batch_store_phase(float *dst, float2 v) { *dst = phase_atan2(v.y, v.x); }

// The G forward FFTs of an item: channel g stages its passes in the padded
// slice spec + g (N + N/16) of the tile; the last pass keeps its outputs in
// registers, and after a barrier they overwrite the tile as the unpadded
// spectra spec + g N.  R = kTile / kBThreads, so G N / R = kBThreads threads
// for every N.
template <int N>
__device__ __noinline__ void batch_forward(const BatchArgs &a, const BatchItem &it, float2 *spec) {
    constexpr int R = kTile / kBThreads;
    constexpr int Tf = N / R;
    static_assert(R <= N, "one pass at least");
    // fields are read once into registers: a and it live in local memory here
    // (this function is not inlined) and stores through generic pointers
    // would otherwise force their reloads
    const float2 *const tw = a.tw;
    const int G = it.G, n = it.n;
    const int g = threadIdx.x / Tf, j = threadIdx.x % Tf;
    const bool act = g < G;
    const float *x = a.in + it.in_off + (long long)(act ? g : 0) * n;
    float2 *st = spec + g * FftShape<N, R>::SMEM_F2;
    float2 *sp = spec + g * N;
    auto load = [&](int i) -> float2 { return make_float2((act && i < n) ? x[i] : 0.f, 0.f); };
    auto store = [&](int t, float2 v) { *CWT_SMEM(&sp[t]) = v; };  // NP = 1: no staging to overwrite
    float2 v[R];
    fft_pass0_dense<N, R, -1>(v, j, load);
    fft_finish<N, R, -1, decltype(store), true>(v, st, tw, j, store);
    if constexpr (FftShape<N, R>::NP > 1) {
        __syncthreads();  // every staging read is done before the spectra overwrite it
#pragma unroll
        for (int r = 0; r < R; ++r) *CWT_SMEM(&sp[j + r * (N / R)]) = v[r];
    }
}

// Rows of M points, RI points per thread: P = kBThreads / (M / RI) rows in
// flight fill the inverse staging (kBThreads * RI points) exactly, which needs
// M <= kBThreads * RI; the host takes RI = 16 only for batches whose every
// inverse length satisfies it.
template <int M, int RI>
__device__ __noinline__ void batch_inverse(const BatchArgs &a, const BatchItem &it,
                                              const float2 *spec, float2 *stage, int N, int fold) {
    static_assert(M <= kBThreads * RI, "rows in flight fit the inverse staging");
    constexpr int R = M < RI ? M : RI;
    constexpr int Ti = M / R;
    constexpr int P = kBThreads / Ti;  // rows in flight
    // fields are read once into registers (see batch_forward)
    const int S = a.S, d = a.d;
    float2 *const oc = a.oc;
    float *const op = a.op;
    float *const oph = a.oph;
    const float2 *const tw = a.tw;
    const long long out_off = it.out_off;
    const int rows = it.G * S;
    const float *bank = a.bank[it.log2n];
    const int *band = a.band[it.log2n];
    const int nmask = N - 1;
    const int sub = d / fold;
    const int n_out = (it.n + d - 1) / d;
    const int rl = threadIdx.x / Ti, j = threadIdx.x % Ti;
    float2 *st = stage + rl * FftShape<M, R>::SMEM_F2;
#pragma unroll 1
    for (int r0 = 0; r0 < rows; r0 += P) {
        const int row = r0 + rl;
        const bool act = row < rows;
        const int g = act ? row / S : 0;
        const int s = act ? row - g * S : 0;
        const float2 *sp = spec + g * N;
        const float *W = bank + (size_t)s * N;
        const int b0 = band[2 * s], B = act ? band[2 * s + 1] : 0;
        // Folded input j = sum over in-band k = j (mod M).  When the band is no
        // wider than M, at most one k qualifies: k = b0 + ((j - b0) mod M).
        const bool narrow = B <= M;
        auto load = [&](int jj) -> float2 {
            float2 acc = make_float2(0.f, 0.f);
            if (narrow) {
                const int delta = (jj - b0) & (M - 1);
                if (delta < B) {
                    const int k = (b0 + delta) & nmask;
                    const float2 xv = *CWT_SMEM(&sp[k]);
                    const float w = __ldg(&W[k]);
                    acc = make_float2(xv.x * w, xv.y * w);
                }
                return acc;
            }
            for (int q = 0; q < fold; ++q) {
                const int k = jj + q * M;
                if (((k - b0) & nmask) < B) {
                    const float2 xv = *CWT_SMEM(&sp[k]);
                    const float w = __ldg(&W[k]);
                    acc.x = fmaf(xv.x, w, acc.x);
                    acc.y = fmaf(xv.y, w, acc.y);
                }
            }
            return acc;
        };
        const long long obase = out_off + (long long)row * n_out;
        auto store = [&](int t, float2 v) {
            if (!act) return;
            int o = t;
            if (sub != 1) {
                if (t % sub) return;
                o = t / sub;
            }
            if (o >= n_out) return;
            if (oc) oc[obase + o] = v;
            if (op) op[obase + o] = fmaf(v.x, v.x, v.y * v.y);
            if (oph) batch_store_phase(oph + obase + o, v);
        };
        fft_row<M, R, +1>(st, tw, j, load, store);
    }
}

template <int RI>
__device__ __forceinline__ void batch_inverse_dispatch(const BatchArgs &a, const BatchItem &it,
                                                       const float2 *spec, float2 *stage) {
    const int N = 1 << it.log2n;
    const int M = batch_inverse_length(N, a.d);
    const int fold = N / M;
    switch (ilog2c(M)) {
#define CWT_BI_CASE(L)                                                                         \
    case L:                                                                                    \
        if constexpr ((1 << L) <= kBThreads * RI) batch_inverse<1 << L, RI>(a, it, spec, stage, N, fold); \
        break;
        CWT_BI_CASE(5) CWT_BI_CASE(6) CWT_BI_CASE(7) CWT_BI_CASE(8) CWT_BI_CASE(9)
        CWT_BI_CASE(10) CWT_BI_CASE(11) CWT_BI_CASE(12) CWT_BI_CASE(13)
#undef CWT_BI_CASE
        default: break;
    }
}

template <int RI>
__global__ void __launch_bounds__(kBThreads, 2) batch_kernel(const BatchArgs a) {
    extern __shared__ float2 bsm[];
    float2 *spec = bsm;
    float2 *stage = bsm + kTileP;
    __shared__ int s_item;
#pragma unroll 1
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) break;
        const BatchItem it = a.items[item];
        switch (it.log2n) {
            case 5: batch_forward<1 << 5>(a, it, spec); break;
            case 6: batch_forward<1 << 6>(a, it, spec); break;
            case 7: batch_forward<1 << 7>(a, it, spec); break;
            case 8: batch_forward<1 << 8>(a, it, spec); break;
            case 9: batch_forward<1 << 9>(a, it, spec); break;
            case 10: batch_forward<1 << 10>(a, it, spec); break;
            case 11: batch_forward<1 << 11>(a, it, spec); break;
            case 12: batch_forward<1 << 12>(a, it, spec); break;
            case 13: batch_forward<1 << 13>(a, it, spec); break;
            default: break;
        }
        __syncthreads();  // spectra complete before any row reads them
        batch_inverse_dispatch<RI>(a, it, spec, stage);
        __syncthreads();  // s_item and the spectra are free again
    }
}

}  // namespace
#endif  // CWT_BATCH_KERNELS

}  // namespace cwtk
