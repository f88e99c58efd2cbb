// fft_tc.cuh -- radix-16 DFT passes of a 16384-point row on the tensor cores.
//
// The inverse FFT of each (channel, scale) row (Eq. 2, Section "Fourier
// transformed formula"; its Cooley-Tukey factorisation, Section "Fast Fourier
// transform") is run as pass 0 of radix 4 in FP32 followed by three radix-16
// Stockham passes whose 16-point DFTs are small dense matrix products:
//
//     y = F16 x,   F16[q][m] = exp(SIGN 2 pi i q m / 16),
//
// one column x per butterfly, eight butterflies per mma.sync.m16n8k16.  The
// complex product is written in real arithmetic: the column holds
// (Re x_m, Im x_m) interleaved (K = 32 reals, two k-tiles), the rows hold
// Re y_q for q = 0..15 then Im y_q (M = 32 reals, two m-tiles), and the real
// 32 x 32 matrix has the blocks [[c, -s], [s, c]] of F16's entries
// c + i s.  Operands are FP16 or BF16 with FP32 accumulation.  Each operand
// is split as v = hi + lo (hi = v rounded to 16 bits, lo = the remainder
// rounded to 16 bits) and the product is taken as
//     A_hi B_lo + A_lo B_hi + A_hi B_hi,
// dropping only A_lo B_lo: the compensated product keeps about twice the
// 16-bit significand (2^-22 relative for FP16, 2^-16 for BF16) instead of
// one rounding of 2^-11 / 2^-8 per pass.
//
// Fragment layouts are those of mma.sync.m16n8k16 (PTX ISA, "Matrix
// Fragments for mma.m16n8k16"): lane = 4 g + t holds A rows g and g+8 at
// columns 2t, 2t+1, 2t+8, 2t+9; B rows 2t, 2t+1, 2t+8, 2t+9 of column g;
// and D rows g, g+8 at columns 2t, 2t+1.  So in a pass lane (g, t) feeds
// points m = t, t+4, t+8, t+12 of butterfly g and receives outputs q = g and
// q = g+8 of butterflies 2t and 2t+1.
//
// FP16 has a 5-bit exponent: the caller scales each row by an exact power
// of two chosen so that the row's L1 norm stays below 2^15 (every Stockham
// intermediate is a sum of inputs times unit-modulus twiddles, hence bounded
// by that norm) and unscales the outputs.
//
// Schedule of the 16384-point row (radix 4 x 16 x 16 x 16, Stockham):
//   pass A  pass 0 (radix 4, FP32) computed on the fly from the banded
//           spectrum for each input of the first radix-16 pass (Ns = 4),
//           whose outputs go straight to shared memory;
//   pass B  radix 16, Ns = 64.  The butterflies jj = k (mod 64) read and
//           write exactly the positions = k (mod 64), so a warp that takes
//           whole residue classes k (two MMAs of 8 butterflies each) only
//           has to wait for its own lanes (__syncwarp) between reading and
//           writing;
//   pass C  radix 16, Ns = 1024: butterfly jj reads and writes the positions
//           jj + 1024 m, so the butterflies k + 64 q (q < 16) of pass C touch
//           exactly the class k of pass B: the warp that owns class k runs
//           its pass C right after its pass B, with __syncwarp only (no
//           barrier of the whole CTA between the two passes).
// So no pass holds more than two MMAs' outputs in registers and the row
// stays in place in one 128 KB buffer.
//
// Shared-memory layout (tc_pad): element i of the row sits at i with its
// bits 0-3 XORed by a GF(2)-linear function of bits 6, 7, 8, 10, 11 and 12.
// It is chosen so that every access of the passes (lanes at strides 64 and
// 1024, 128 and 1024, and the Ns = 4 output pattern) and the natural-order
// reads that follow touch 16 distinct 8-byte bank pairs per half-warp: no
// bank conflicts.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "check.cuh"
#include "fft_core.cuh"

namespace cwtk {

constexpr int kTcNL = 16384;      // points per CTA row
constexpr int kTcThreads = 512;   // 16 warps
constexpr int kTcNB = kTcNL / 16; // butterflies per radix-16 pass

// XOR terms of tc_pad: bits 6, 7, 8 of the index -> masks 1, 2, 1 and bits
// 10, 11, 12 -> masks 5, 8, 4, each group as a table of eight nibbles.
__device__ __forceinline__ int tc_lut_lo(int b) { return (int)((0x23013210u >> (b * 4)) & 15u); }
__device__ __forceinline__ int tc_lut(int b) { return (int)((0x9C14D850u >> (b * 4)) & 15u); }

__device__ __forceinline__ int tc_pad(int i) { return i ^ tc_lut_lo((i >> 6) & 7) ^ tc_lut((i >> 10) & 7); }

// The two 16-bit operand types of mma.sync kind f16 (A and B of one MMA
// always share the type).
struct TcF16 {
    static __device__ __forceinline__ uint32_t pack(float a, float b) {  // a -> low half
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t r) {
        return __half22float2(*reinterpret_cast<const __half2 *>(&r));
    }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

struct TcBF16 {
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t r) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r));
    }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

// v = hi + lo, each a pair of 16-bit values (x in the low half).
template <class T>
__device__ __forceinline__ void tc_split(float2 v, uint32_t &hi, uint32_t &lo) {
    hi = T::pack(v.x, v.y);
    const float2 h = T::unpack(hi);
    lo = T::pack(v.x - h.x, v.y - h.y);
}

// This lane's A fragments of the real 32 x 32 form of F16, split hi/lo:
// a[mt][kt][r] for m-tile mt (0: Re y rows, 1: Im y rows), k-tile kt.
// root16[e] = exp(SIGN 2 pi i e / 16), e < 16 (entries 8e of the twiddle
// table tc_fill_twiddles builds).
template <class T>
__device__ __forceinline__ void tc_dft16_afrag(uint32_t (&ahi)[2][2][4], uint32_t (&alo)[2][2][4],
                                               int lane, const float2 *__restrict__ root16, int stride) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int q = g + 8 * (r & 1);
            const int m = 8 * kt + t + 4 * (r >> 1);
            const float2 w = *CWT_SMEM(&root16[((q * m) & 15) * stride]);  // F16[q][m] = c + i s
            // m-tile 0 (Re y_q): (c, -s) on (Re x_m, Im x_m); m-tile 1 (Im y_q): (s, c)
            tc_split<T>(make_float2(w.x, -w.y), ahi[0][kt][r], alo[0][kt][r]);
            tc_split<T>(make_float2(w.y, w.x), ahi[1][kt][r], alo[1][kt][r]);
        }
}

// The 16-point DFTs of eight butterflies (the MMA's columns) on the tensor
// cores: bh/bl are this lane's B fragments (points t, t+4, t+8, t+12 of
// butterfly g, twiddled and split), acc receives outputs g and g+8 of
// butterflies 2t and 2t+1 (acc[0][*] real parts, acc[1][*] imaginary parts;
// index r: 0/1 output g of butterfly 2t/2t+1, 2/3 output g+8).  The small
// products (A_hi B_lo, A_lo B_hi) and A_hi B_hi run as two independent
// accumulation chains per m-tile, summed at the end.
template <class T>
__device__ __forceinline__ void tc_dft16_mma(float (&acc)[2][4], const uint32_t (&ahi)[2][2][4],
                                             const uint32_t (&alo)[2][2][4], const uint32_t (&bh)[4],
                                             const uint32_t (&bl)[4]) {
    __syncwarp();  // the operands may come from divergent paths; mma.sync needs the whole warp
    float lo[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[mt][r] = lo[mt][r] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            T::mma(lo[mt], ahi[mt][kt], bl[2 * kt], bl[2 * kt + 1]);
            T::mma(acc[mt], ahi[mt][kt], bh[2 * kt], bh[2 * kt + 1]);
            T::mma(lo[mt], alo[mt][kt], bh[2 * kt], bh[2 * kt + 1]);
        }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[mt][r] += lo[mt][r];
}

// x * exp(2 pi i n / 4) for any integer n, without branches (the radix-4
// roots are +-1 and +-i).
__device__ __forceinline__ float2 rot4(float2 x, int n) {
    const float2 y = (n & 1) ? make_float2(-x.y, x.x) : x;
    return (n & 2) ? make_float2(-y.x, -y.y) : y;
}

// Twiddles of the three passes in shared memory, after the row (float2),
// laid out so that a warp's reads hit distinct bank pairs or one address:
//   [0, 80)       pass A: exp(SIGN 2 pi i k m / 64),     entry 20 k + m (k < 4)
//   [80, 1104)    pass B: exp(SIGN 2 pi i k m / 1024),   entry 16 k + m (k < 64)
//   [1104, 2128)  pass C: exp(SIGN 2 pi i k m / 16384),  entry 16 k + m (k < 64)
//   [2128, 2448)  pass C: exp(SIGN 2 pi i a m / 256),    entry 20 a + m (a < 16)
//   [2448, 2464)  exp(SIGN 2 pi i e / 16), the DFT matrix's entries
// Pass C's butterfly jj = k + 64 a (k < 64, a < 16) needs exp(SIGN 2 pi i jj m /
// 16384), the product of its two tables' entries.  All come from the
// FP64-generated FP32 table tw of the 2^17-th roots of unity.
constexpr int kTcTabA = 0, kTcTabB = 80, kTcTabC1 = 1104, kTcTabC2 = 2128, kTcTabR = 2448,
              kTcTabF2 = 2464;

template <int SIGN>
__device__ __forceinline__ void tc_fill_twiddles(float2 *__restrict__ tab, const float2 *__restrict__ tw) {
    for (int i = threadIdx.x; i < kTcTabF2; i += kTcThreads) {
        int x;  // exponent in units of 2 pi / 2^17
        if (i < kTcTabB) x = (((i / 20) * (i % 20)) & 63) * (kTwN / 64);
        else if (i < kTcTabC1) x = ((((i - kTcTabB) >> 4) * ((i - kTcTabB) & 15)) & 1023) * (kTwN / 1024);
        else if (i < kTcTabC2) x = (((i - kTcTabC1) >> 4) * ((i - kTcTabC1) & 15)) * (kTwN / kTcNL);
        else if (i < kTcTabR) x = ((((i - kTcTabC2) / 20) * ((i - kTcTabC2) % 20)) & 255) * (kTwN / 256);
        else x = (i - kTcTabR) * (kTwN / 16);
        float2 w = __ldg(&tw[x]);
        if (SIGN < 0) w.y = -w.y;
        *CWT_SMEM(&tab[i]) = w;
    }
}

// The whole 16384-point FFT of the CTA's row (all 512 threads call it):
// X[t] = sum_m x[m] exp(SIGN 2 pi i m t / 16384).  Pass 0 (radix 4) reads its
// inputs through the caller: dense, load(m) for any m < 16384; sparse (every
// radix-4 butterfly {j + 4096 r} holds at most one nonzero input),
// first(j, r, x) gives butterfly j's nonzero input x and its position r, or
// x = 0 when it has none.  `tab` holds the twiddle tables (tc_fill_twiddles, before the
// call, with a barrier).  On return sm holds X[t] at tc_pad(t), natural order.
// The shared-memory indices of passes B and C are tc_pad's, with the XOR
// terms that stay fixed for a lane (bits 6-7 and 10-12 of each access
// pattern) computed once.
template <class T, int SIGN, typename Load, typename First>
__device__ __forceinline__ void tc_fft16384(float2 *__restrict__ sm, const float2 *__restrict__ tab,
                                            bool sparse, Load &load, First &first) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t ahi[2][2][4], alo[2][2][4];
    tc_dft16_afrag<T>(ahi, alo, lane, tab + kTcTabR, 1);
    constexpr int Q0 = kTcNL / 4;
    const int sgn = SIGN > 0 ? 1 : -1;

    // ---- pass A: pass 0 on the fly + radix 16 with Ns = 4 ----
    // input point m of butterfly jj is pass-0 output p = jj + 1024 m, i.e.
    // output p & 3 of radix-4 butterfly p >> 2
    auto pass0_out = [&](int p) -> float2 {
        const int j = p >> 2, m0 = p & 3;
        if (sparse) {  // first() sets x = 0 when the butterfly has no nonzero input
            int r = 0;
            float2 x;
            first(j, r, x);
            return rot4(x, sgn * r * m0);
        }
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 4; ++r) s = cadd(s, rot4(load(j + Q0 * r), sgn * r * m0));
        return s;
    };
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        const int jj0 = (warp + 16 * i) * 8;
        const int jj = jj0 + g, k = jj & 3;
        uint32_t bh[4], bl[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int m = t + 4 * h;
            tc_split<T>(cmul(pass0_out(jj + kTcNB * m), *CWT_SMEM(&tab[kTcTabA + 20 * k + m])), bh[h], bl[h]);
        }
        float acc[2][4];
        tc_dft16_mma<T>(acc, ahi, alo, bh, bl);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int jn = jj0 + 2 * t + e, kn = jn & 3;
            const int base = (jn - kn) * 16 + kn;
            *CWT_SMEM(&sm[tc_pad(base + 4 * g)]) = make_float2(acc[0][e], acc[1][e]);
            *CWT_SMEM(&sm[tc_pad(base + 4 * (g + 8))]) = make_float2(acc[0][2 + e], acc[1][2 + e]);
        }
    }
    __syncthreads();

    // ---- passes B (radix 16, Ns = 64) and C (radix 16, Ns = 1024) ----
    // Warp w owns the residue classes k = 4w .. 4w+3 (mod 64) of both.
    //   pass B: butterflies k + 64 (8 rho + n), loads k + 64 (8 rho + g) + 1024 m
    //           (bits 6-8 = g, 10-12 = m & 7), stores 1024 (8 rho + 2t + e) + k + 64 q
    //           (bits 6-8 = g, 10-12 = 2t + e);
    //   pass C: butterflies k + 64 (8 rho + n), the same loads, stores
    //           k + 64 (8 rho + 2t + e) + 1024 q (bits 6-8 = 2t + e, 10-12 = g).
    {
        int xl[4], xsb[2], xsc[2];
#pragma unroll
        for (int h = 0; h < 4; ++h) xl[h] = tc_lut_lo(g) ^ tc_lut((t + 4 * h) & 7);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            xsb[e] = tc_lut_lo(g) ^ tc_lut(2 * t + e);
            xsc[e] = tc_lut_lo(2 * t + e) ^ tc_lut(g);
        }
#pragma unroll 1
        for (int kk = 0; kk < 4; ++kk) {
            const int k = 4 * warp + kk;
            float acc[2][2][4];
            // pass B
#pragma unroll
            for (int rho = 0; rho < 2; ++rho) {
                const int jj = k + 64 * (8 * rho + g);
                uint32_t bh[4], bl[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int m = t + 4 * h;
                    tc_split<T>(cmul(*CWT_SMEM(&sm[(jj + kTcNB * m) ^ xl[h]]), *CWT_SMEM(&tab[kTcTabB + 16 * k + m])), bh[h], bl[h]);
                }
                tc_dft16_mma<T>(acc[rho], ahi, alo, bh, bl);
            }
            __syncwarp();  // the class's 32 inputs are read before any of its outputs lands
#pragma unroll
            for (int rho = 0; rho < 2; ++rho)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int base = 1024 * (8 * rho + 2 * t + e) + k;
                    *CWT_SMEM(&sm[(base + 64 * g) ^ xsb[e]]) = make_float2(acc[rho][0][e], acc[rho][1][e]);
                    *CWT_SMEM(&sm[(base + 64 * (g + 8)) ^ xsb[e]]) = make_float2(acc[rho][0][2 + e], acc[rho][1][2 + e]);
                }
            __syncwarp();  // pass B's outputs of the class are visible to the warp
            // pass C: twiddle exp(SIGN 2 pi i jj m / 16384), jj = k + 64 a, from the
            // tables of exp(SIGN 2 pi i k m / 16384) and exp(SIGN 2 pi i a m / 256)
#pragma unroll
            for (int rho = 0; rho < 2; ++rho) {
                const int a = 8 * rho + g, jj = k + 64 * a;
                uint32_t bh[4], bl[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int m = t + 4 * h;
                    const float2 w = cmul(*CWT_SMEM(&tab[kTcTabC1 + 16 * k + m]),
                                          *CWT_SMEM(&tab[kTcTabC2 + 20 * a + m]));
                    tc_split<T>(cmul(*CWT_SMEM(&sm[(jj + kTcNB * m) ^ xl[h]]), w), bh[h], bl[h]);
                }
                tc_dft16_mma<T>(acc[rho], ahi, alo, bh, bl);
            }
            __syncwarp();
#pragma unroll
            for (int rho = 0; rho < 2; ++rho)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int base = k + 64 * (8 * rho + 2 * t + e);
                    *CWT_SMEM(&sm[(base + 1024 * g) ^ xsc[e]]) = make_float2(acc[rho][0][e], acc[rho][1][e]);
                    *CWT_SMEM(&sm[(base + 1024 * (g + 8)) ^ xsc[e]]) = make_float2(acc[rho][0][2 + e], acc[rho][1][2 + e]);
                }
        }
    }
    __syncthreads();
}

}  // namespace cwtk
