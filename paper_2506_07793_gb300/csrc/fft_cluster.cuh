// fft_cluster.cuh -- Stockham FFT of one long row across a thread-block
// cluster, exchanging through distributed shared memory.
//
// Rows longer than one CTA's shared memory (N = CL * 16384, CL = 2, 4, 8;
// e.g. the 131072-point padding of a 60 s recording at 2048 Hz, Section "Fast
// Fourier transform") run on a cluster of CL CTAs of 512 threads, 32 points per
// thread.  The cluster thread index is J = tid * CL + rank and CTA `rank` owns
// the elements idx = rank (mod CL) at slot idx / CL.  With this interleaving
//  * every pass reads only its own CTA's shared memory (J + r*T = J mod CL);
//  * a pass with Ns >= CL also writes only locally; only pass 0 and passes
//    with Ns < CL write into other CTAs (st through the cluster window);
//  * the last pass writes its outputs to the CTA that owns the contiguous
//    range t / (N / CL), so the epilogue's global stores are coalesced.
// Cluster barriers order the remote writes; local passes use __syncthreads.
#pragma once

#include <cooperative_groups.h>

#include "fft_core.cuh"

namespace cwtk {

namespace cg = cooperative_groups;

constexpr int kClThreads = 512;
constexpr int kClR = 32;
constexpr int kClPoints = kClThreads * kClR;  // 16384 points per CTA

template <int N>
struct ClusterShape {
    static constexpr int CL = N / kClPoints;
    static constexpr int LCL = ilog2c(CL);
    static constexpr int NL = N / CL;  // elements per CTA
    static constexpr int SMEM_F2 = NL + (NL >> 4);
    static constexpr int SMEM_BYTES = SMEM_F2 * 8;
    static_assert(CL >= 2 && CL <= 8 && CL * kClPoints == N, "N = 2, 4 or 8 x 16384");
};

// Passes 0-store .. last of a cluster row; v holds this thread's pass-0
// outputs (from fft_pass0_dense / fft_pass0_sparse with j = J).  `store(t, X[t])`
// is called for the CTA's contiguous output range t in [rank*NL, (rank+1)*NL).
template <int N, int SIGN, typename Store>
__device__ __forceinline__ void fft_cluster_finish(float2 (&v)[kClR], float2 *__restrict__ sm,
                                                   const float2 *__restrict__ tw, Store &store) {
    using S = FftShape<N, kClR>;
    using C = ClusterShape<N>;
    constexpr int R = kClR, T = S::T, R0 = S::R0, G0 = S::G0, TL = kClThreads;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x;
    const int J = tid * C::CL + rank;
    // pass-0 outputs to their owners (every CTA must be done with its buffer)
    cl.sync();
#pragma unroll
    for (int g = 0; g < G0; ++g)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
            const int idx = (J + g * T) * R0 + r;
            float2 *dst = cl.map_shared_rank(sm, idx & (C::CL - 1));
            dst[spad2(idx >> C::LCL)] = v[g * R0 + r];
        }
    cl.sync();
    int Ns = R0;
#pragma unroll 1
    for (int p = 1; p < S::NP; ++p) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sm[spad2(tid + r * TL)];
        const int k = J & (Ns - 1);
        float2 w1 = __ldg(&tw[k * (kTwN / (Ns * R))]);
        if (SIGN < 0) w1.y = -w1.y;
        twiddle_chain<R>(v, w1);
        dft<R, SIGN>(v);
        if (p == S::NP - 1) {
            cl.sync();  // every CTA has read its inputs
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int t = J + r * Ns;
                float2 *dst = cl.map_shared_rank(sm, t / C::NL);
                dst[spad2(t & (C::NL - 1))] = v[r];
            }
            cl.sync();
#pragma unroll 1
            for (int m = 0; m < R; ++m) {
                const int slot = tid + m * TL;
                store(rank * C::NL + slot, sm[spad2(slot)]);
            }
        } else if (Ns >= C::CL) {  // all writes stay in this CTA
            __syncthreads();
            const int base = (J - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[spad2((base + r * Ns) >> C::LCL)] = v[r];
            __syncthreads();
        } else {
            cl.sync();
            const int base = (J - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int idx = base + r * Ns;
                float2 *dst = cl.map_shared_rank(sm, idx & (C::CL - 1));
                dst[spad2(idx >> C::LCL)] = v[r];
            }
            cl.sync();
        }
        Ns *= R;
    }
}

}  // namespace cwtk
