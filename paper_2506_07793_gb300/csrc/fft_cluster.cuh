// fft_cluster.cuh -- FFT of one long row on a thread-block cluster.
//
// Rows longer than one CTA's shared memory (N = CL * 16384, CL = 2, 4, 8;
// e.g. the 131072-point padding of a 60 s recording at 2048 Hz, Section "Fast
// Fourier transform") run on a cluster of CL CTAs of 512 threads.  With
// k = c + CL * m (residue class c) and t = t1 + NL * t2 (NL = N / CL):
//     X[t1 + NL t2] = sum_c w_CL^(c t2) * [ w_N^(c t1) * A_c[t1] ],
//     A_c[t1]       = sum_m x[c + CL m] w_NL^(m t1),
// (w_M = exp(SIGN 2 pi i / M)).  So
//  1. CTA c runs the fast one-CTA 16384-point FFT of its residue class
//     (fft_core.cuh) and keeps A_c in its own shared memory;
//  2. after one cluster barrier, CTA c takes t1 in [c NL/CL, (c+1) NL/CL):
//     each thread reads A_0..A_{CL-1}[t1] from the CTAs' shared memory
//     (ld.shared::cluster), twiddles, runs a CL-point DFT and emits the CL
//     outputs t1 + NL t2 -- consecutive threads write consecutive t1, so the
//     epilogue's global stores are coalesced.
// One bulk exchange per row; every other access stays in the CTA.
#pragma once

#include <cooperative_groups.h>

#include "dsmem.cuh"
#include "fft_core.cuh"

namespace cwtk {

namespace cg = cooperative_groups;

constexpr int kClThreads = 512;
constexpr int kClR = 32;
constexpr int kClPoints = kClThreads * kClR;  // 16384 points per CTA

template <int N>
struct ClusterShape {
    static constexpr int CL = N / kClPoints;
    static constexpr int NL = kClPoints;
    static constexpr int SMEM_F2 = FftShape<NL, kClR>::SMEM_F2;
    static constexpr int SMEM_BYTES = SMEM_F2 * 8;
    static_assert(CL >= 2 && CL <= 8 && CL * kClPoints == N, "N = 2, 4 or 8 x 16384");
};

// Whole-row FFT on the cluster: `load(k)` gives x[k] (k in [0, N)); `store(t,
// X[t])` receives outputs t = t1 + NL t2 for this CTA's t1 range.  When
// `sparse` is true, `first(jj, r, x)` serves the local pass 0 instead (see
// fft_pass0_sparse; jj and r index this CTA's residue class m = jj + r NL/R0).
// All threads of all CTAs of the cluster call it together.
template <int N, int SIGN, typename Load, typename First, typename Store>
__device__ __forceinline__ void fft_cluster_row(float2 *__restrict__ sm, const float2 *__restrict__ tw,
                                                Load &load, bool sparse, First &first, Store &store) {
    using C = ClusterShape<N>;
    constexpr int CL = C::CL, NL = C::NL, TL = kClThreads;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x;
    // 1. local FFT of the residue class `rank`
    auto lload = [&](int m) -> float2 { return load(rank + CL * m); };
    auto nostore = [&](int, float2) {};
    float2 v[kClR];
    if (sparse)
        fft_pass0_sparse<NL, kClR, SIGN>(v, tid, tw, first);
    else
        fft_pass0_dense<NL, kClR, SIGN>(v, tid, lload);
    fft_finish<NL, kClR, SIGN, decltype(nostore), true>(v, sm, tw, tid, nostore);
    __syncthreads();  // every thread has read its last-pass inputs
#pragma unroll
    for (int r = 0; r < kClR; ++r) *CWT_SMEM(&sm[spad2(tid + r * TL)]) = v[r];  // A_rank[t1], natural order
    cl.sync();
    // 2. cross-CTA radix-CL stage over this CTA's t1 range
#pragma unroll 1
    for (int q = 0; q < NL / CL / TL; ++q) {
        const int t1 = rank * (NL / CL) + q * TL + tid;
        float2 a[CL];
#pragma unroll
        for (int c = 0; c < CL; ++c) a[c] = ld_cluster(CWT_SMEM(&sm[spad2(t1)]), (unsigned)c);
#pragma unroll
        for (int c = 1; c < CL; ++c) {
            float2 w = __ldg(&tw[(c * t1) * (kTwN / N)]);  // c * t1 < N
            if (SIGN < 0) w.y = -w.y;
            a[c] = cmul(a[c], w);
        }
        dft<CL, SIGN>(a);
#pragma unroll
        for (int t2 = 0; t2 < CL; ++t2) store(t1 + NL * t2, a[t2]);
    }
    cl.sync();  // no CTA still reads this CTA's buffer
}

// Dense-input convenience form.
template <int N, int SIGN, typename Load, typename Store>
__device__ __forceinline__ void fft_cluster_row(float2 *__restrict__ sm, const float2 *__restrict__ tw,
                                                Load &load, Store &store) {
    auto none = [](int, int &, float2 &) -> bool { return false; };
    fft_cluster_row<N, SIGN>(sm, tw, load, false, none, store);
}

}  // namespace cwtk
