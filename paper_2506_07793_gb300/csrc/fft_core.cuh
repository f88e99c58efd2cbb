// fft_core.cuh -- Stockham FFT building blocks for sm_103a.
//
// The CWT of arXiv 2506.07793 evaluates the cyclic convolution with one
// forward FFT per channel and one inverse FFT per (channel, scale) (Section
// "Fourier transformed formula", Eq. 2); the paper leans on Cooley-Tukey
// factorisations (Section "Fast Fourier transform").  This header holds the
// radix-R Stockham passes used by every kernel of the library:
//
//  * A row of length N is handled by T = N / R threads; each thread keeps R
//    complex values in registers.
//  * Pass p (radix Rp, Ns = product of the earlier radices): thread j owns
//    butterflies jj = j + g*T.  It multiplies input r by w^r with
//    w = exp(+-2 pi i (jj mod Ns) / (Ns Rp)), runs an Rp-point DFT in
//    registers and writes output r to position
//    (jj - jj mod Ns) * Rp + (jj mod Ns) + r * Ns.  This is the self-sorting
//    (Stockham) decimation-in-time order: the last pass writes natural order.
//  * Between passes the row is exchanged through shared memory as float2 with
//    one pad slot per 16 (bank-conflict-free for the strides used here).
//  * Only pass 0 may have a smaller radix; passes 1.. run one rolled loop body
//    so the kernel's code stays small enough for the instruction cache.
//  * The first pass reads its inputs through a caller functor (global memory,
//    fused pre-processing) and the last pass hands each output to a caller
//    functor (fused epilogue), so neither end touches shared memory.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "check.cuh"

namespace cwtk {

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// Twiddle table: tw[m] = exp(+2 pi i m / kTwN), m < kTwN, generated in FP64 and
// rounded to FP32 (one table per device, shared by every plan).
constexpr int kTwLog2 = 17;
constexpr int kTwN = 1 << kTwLog2;

// cos(2 pi j / 32), j = 0..8 (first quadrant), as exact-to-float literals.
__host__ __device__ constexpr float cos_q32(int j) {
    return j == 0 ? 1.0f
         : j == 1 ? 0.980785280403230449126f
         : j == 2 ? 0.923879532511286756128f
         : j == 3 ? 0.831469612302545237079f
         : j == 4 ? 0.707106781186547524401f
         : j == 5 ? 0.555570233019602224743f
         : j == 6 ? 0.382683432365089771728f
         : j == 7 ? 0.195090322016128267848f
                  : 0.0f;
}
// cos(2 pi m / 32) and sin(2 pi m / 32) for any integer m.
__host__ __device__ constexpr float cos32(int m) {
    return ((m & 31) >> 3) == 0 ? cos_q32(m & 7)
         : ((m & 31) >> 3) == 1 ? -cos_q32(8 - (m & 7))
         : ((m & 31) >> 3) == 2 ? -cos_q32(m & 7)
                                : cos_q32(8 - (m & 7));
}
__host__ __device__ constexpr float sin32(int m) { return cos32(m + 24); }

// Complex add / subtract as one packed FP32x2 instruction (add/sub.rn.f32x2,
// sm_100 and later): the same round-to-nearest result per component as two
// scalar adds, in half the issue slots.  (A packed multiply-add form of cmul
// measured slower: the operand shuffles cost more than they save.)
__device__ __forceinline__ unsigned long long f2pack(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a)), "l"(f2pack(b)));
    return f2unpack(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a)), "l"(f2pack(b)));
    return f2unpack(d);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// a * exp(SIGN * 2 pi i * m / 32) with m known at compile time after unrolling;
// the trivial roots reduce to swaps and negations, the eighth roots to one
// multiply per component.
template <int SIGN>
__device__ __forceinline__ float2 rot32(float2 a, int m) {
    m &= 31;
    if (m == 0) return a;
    if (m == 16) return make_float2(-a.x, -a.y);
    if (m == 8) return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    if (m == 24) return SIGN > 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    const float c = cos32(m), s = SIGN > 0 ? sin32(m) : -sin32(m);
    if ((m & 7) == 4) {  // |c| = |s| = sqrt(2)/2: signs fold away at compile time
        const float h = 0.707106781186547524401f;
        const float sc = c > 0.f ? 1.f : -1.f, ss = s > 0.f ? 1.f : -1.f;
        return make_float2(h * (sc * a.x - ss * a.y), h * (ss * a.x + sc * a.y));
    }
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// In-register DFT of R = 2..32 points, natural order in and out:
// X[k] = sum_m v[m] exp(SIGN 2 pi i k m / R).  Radix-2 decimation in frequency
// with compile-time twiddles, then a compile-time bit-reversal (register
// renaming only).
template <int R, int SIGN>
__device__ __forceinline__ void dft(float2 *v) {
    static_assert(R >= 1 && R <= 32 && (R & (R - 1)) == 0, "radix must be a power of two <= 32");
    constexpr int L2 = ilog2c(R);
#pragma unroll
    for (int stage = 0; stage < L2; ++stage) {
        const int half = R >> (stage + 1);
#pragma unroll
        for (int base = 0; base < R; base += 2 * half) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const float2 a = v[base + k], b = v[base + k + half];
                v[base + k] = cadd(a, b);
                v[base + k + half] = rot32<SIGN>(csub(a, b), k * (32 / (2 * half)));
            }
        }
    }
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[bitrev(i, L2)];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
}

// v[r] *= w^r for r = 1..Rp-1.  The low powers w^1..w^7 come from a
// square-and-multiply chain; higher powers are w^(8h) * w^(r mod 8), so each
// factor is at most ~6 roundings from exact and only ~10 twiddles are live.
template <int Rp>
__device__ __forceinline__ void twiddle_chain(float2 *v, float2 w1) {
    constexpr int LO = Rp < 8 ? Rp : 8;
    float2 wl[LO];
    wl[0] = make_float2(1.f, 0.f);
    if (LO > 1) wl[1] = w1;
#pragma unroll
    for (int r = 2; r < LO; ++r) wl[r] = (r & 1) ? cmul(wl[r - 1], w1) : cmul(wl[r >> 1], wl[r >> 1]);
#pragma unroll
    for (int r = 1; r < LO; ++r) v[r] = cmul(v[r], wl[r]);
    if constexpr (Rp > 8) {
        const float2 w8 = cmul(wl[4], wl[4]);
        float2 wh = w8;
#pragma unroll
        for (int h = 1; h < Rp / 8; ++h) {
            v[8 * h] = cmul(v[8 * h], wh);
#pragma unroll
            for (int r = 1; r < 8; ++r) v[8 * h + r] = cmul(cmul(v[8 * h + r], wh), wl[r]);
            if (h + 1 < Rp / 8) wh = cmul(wh, w8);
        }
    }
}

// Pass schedule for a row of N = 2^L points with R = 2^r points per thread.
// The leftover factor comes FIRST: pass 0 has radix 2^(L mod r) (or R), each
// thread running G0 = R / radix0 butterflies of it; every later pass has radix
// R, so passes 1.. share one rolled loop body (small code footprint).
template <int N, int R>
struct FftShape {
    static constexpr int T = N / R;  // threads per row
    static constexpr int L2N = ilog2c(N);
    static constexpr int L2R = ilog2c(R);
    static constexpr int REM = L2N % L2R;
    static constexpr int R0 = REM ? (1 << REM) : R;  // radix of pass 0
    static constexpr int G0 = R / R0;                 // pass-0 butterflies per thread
    static constexpr int NP = 1 + (L2N - ilog2c(R0)) / L2R;  // total passes
    static constexpr int SMEM_F2 = N + (N >> 4);      // padded float2 slots
    static_assert((1 << L2N) == N && (1 << L2R) == R && R <= N, "power-of-two sizes only");
};

// float2 shared-memory slot of element i: one pad slot every 16, so that
// half-warps touching power-of-two strides up to 16 land on distinct banks.
__device__ __forceinline__ int spad2(int i) { return i + (i >> 4); }

// Whole-row FFT, X[t] = sum_k x[k] exp(SIGN 2 pi i k t / N), natural order in
// and out, split in two so that callers can choose how pass 0 is computed:
//   fft_pass0_dense / fft_pass0_sparse  fill the thread's R registers with the
//                                       pass-0 butterfly outputs;
//   fft_finish                          stores them, runs passes 1.. and hands
//                                       every output to `store(t, X[t])`.
// `sm` is this row's padded float2 staging buffer (FftShape::SMEM_F2 slots).
// All threads of the CTA call them together (they contain __syncthreads).

// Pass 0 (radix R0, Ns = 1, no twiddles), inputs from `load(k)`, k in [0, N).
template <int N, int R, int SIGN, typename Load>
__device__ __forceinline__ void fft_pass0_dense(float2 (&v)[R], int j, Load &load) {
    using S = FftShape<N, R>;
    constexpr int T = S::T, R0 = S::R0, G0 = S::G0;
#pragma unroll
    for (int g = 0; g < G0; ++g)
#pragma unroll
        for (int r = 0; r < R0; ++r) v[g * R0 + r] = load(j + g * T + r * (N / R0));
#pragma unroll
    for (int g = 0; g < G0; ++g) dft<R0, SIGN>(&v[g * R0]);
}

// Pass 0 when each butterfly's inputs {jj + r N/R0 : r < R0} hold at most one
// nonzero value: `first(jj, r, x)` returns true with its position r and value
// x (false: all zero).  The R0-point DFT of x at position r is
// x * exp(SIGN 2 pi i r m / R0), m < R0 -- a twiddle chain, not a full DFT.
template <int N, int R, int SIGN, typename First>
__device__ __forceinline__ void fft_pass0_sparse(float2 (&v)[R], int j, const float2 *__restrict__ tw,
                                                 First &first) {
    using S = FftShape<N, R>;
    constexpr int T = S::T, R0 = S::R0, G0 = S::G0;
#pragma unroll
    for (int g = 0; g < G0; ++g) {
        int r = 0;
        float2 x = make_float2(0.f, 0.f);
        const bool nz = first(j + g * T, r, x);
        float2 w = __ldg(&tw[(r & (R0 - 1)) * (kTwN / R0)]);
        if (SIGN < 0) w.y = -w.y;
        if (!nz) x = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < R0; ++m) v[g * R0 + m] = x;
        twiddle_chain<R0>(&v[g * R0], w);
    }
}

// With KEEP = true the last pass leaves its outputs in v (output r of thread
// j is X[j + r * N / R]) instead of calling `store`.
template <int N, int R, int SIGN, typename Store, bool KEEP = false>
__device__ __forceinline__ void fft_finish(float2 (&v)[R], float2 *__restrict__ sm,
                                           const float2 *__restrict__ tw, int j, Store &store) {
    using S = FftShape<N, R>;
    constexpr int T = S::T, R0 = S::R0, G0 = S::G0;
    if constexpr (S::NP == 1) {
#pragma unroll
        for (int g = 0; g < G0; ++g)
#pragma unroll
            for (int r = 0; r < R0; ++r) store(j + g * T + r, v[g * R0 + r]);
        return;
    } else {
        __syncthreads();  // the buffer may still be read by a previous row
#pragma unroll
        for (int g = 0; g < G0; ++g)
#pragma unroll
            for (int r = 0; r < R0; ++r) *CWT_SMEM(&sm[spad2((j + g * T) * R0 + r)]) = v[g * R0 + r];
    }
    // ---- passes 1..NP-1: radix R, Ns = R0 * R^(p-1).  (Per-element padded
    // indices measured faster on GB300 than base-plus-stride addressing.)
    int Ns = R0;
#pragma unroll 1
    for (int p = 1; p < S::NP; ++p) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = *CWT_SMEM(&sm[spad2(j + r * T)]);
        const int k = j & (Ns - 1);
        float2 w1 = __ldg(&tw[k * (kTwN / (Ns * R))]);
        if (SIGN < 0) w1.y = -w1.y;
        twiddle_chain<R>(v, w1);
        dft<R, SIGN>(v);
        if (p == S::NP - 1) {
            if constexpr (!KEEP) {
#pragma unroll
                for (int r = 0; r < R; ++r) store(j + r * Ns, v[r]);
            }
        } else {
            __syncthreads();
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) *CWT_SMEM(&sm[spad2(base + r * Ns)]) = v[r];
        }
        Ns *= R;
    }
}

template <int N, int R, int SIGN, typename Load, typename Store>
__device__ __forceinline__ void fft_row(float2 *__restrict__ sm, const float2 *__restrict__ tw,
                                        int j, Load &load, Store &store) {
    float2 v[R];
    fft_pass0_dense<N, R, SIGN>(v, j, load);
    fft_finish<N, R, SIGN>(v, sm, tw, j, store);
}

// Points per thread: a build-time tuning knob (the largest length and the
// rest), measured on GB300; see RowConfig.
#ifndef CWT_RADIX_16384
#define CWT_RADIX_16384 32
#endif
#ifndef CWT_RADIX_DEFAULT
#define CWT_RADIX_DEFAULT 16
#endif

// Launch shape for a row kernel of size N: R points per thread, several rows
// per CTA for short rows so that a CTA has at least 256 threads.
template <int N, int RR = (N >= 16384 ? CWT_RADIX_16384 : (N >= CWT_RADIX_DEFAULT ? CWT_RADIX_DEFAULT : N))>
struct RowConfig {
    static constexpr int R = RR;
    static constexpr int T = N / R;
    static constexpr int ROWS = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = T * ROWS;
    static constexpr int SMEM_BYTES = ROWS * FftShape<N, R>::SMEM_F2 * 8;
};

}  // namespace cwtk
