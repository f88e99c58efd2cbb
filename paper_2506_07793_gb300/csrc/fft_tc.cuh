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
//   pass C  radix 16, Ns = 1024: each butterfly reads and writes the same 16
//           positions, so again one __syncwarp per 8 butterflies.
// So no pass holds more than two MMAs' outputs in registers and the row
// stays in place in one 128 KB buffer.
//
// Shared-memory layout (tc_pad): element i of the row sits at i with its
// bits 0-3 XORed by a GF(2)-linear function of bits 6, 7, 10, 11 and 12.  It is
// chosen so that every access of the three passes (lanes at strides 1 and
// 1024, 2 and 1024, 64 and 1024, and the Ns = 4 output pattern) and the
// natural-order reads that follow touch 16 distinct 8-byte bank pairs per
// half-warp: no bank conflicts.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace cwtk {

constexpr int kTcNL = 16384;      // points per CTA row
constexpr int kTcThreads = 512;   // 16 warps
constexpr int kTcNB = kTcNL / 16; // butterflies per radix-16 pass

__device__ __forceinline__ int tc_pad(int i) {
    // bits 10, 11, 12 -> XOR masks 5, 8, 4 (a nibble table); bits 6, 7 -> 1, 2
    const int hi = (int)((0x9C14D850u >> (((i >> 10) & 7) * 4)) & 15u);
    return i ^ ((i >> 6) & 3) ^ hi;
}

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
template <class T, int SIGN>
__device__ __forceinline__ void tc_dft16_afrag(uint32_t (&ahi)[2][2][4], uint32_t (&alo)[2][2][4],
                                               int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int kt = 0; kt < 2; ++kt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int q = g + 8 * (r & 1);
                const int m = 8 * kt + t + 4 * (r >> 1);
                const int e = (q * m) & 15;          // F16[q][m] = exp(SIGN 2 pi i e / 16)
                const float c = cos32(2 * e);
                const float s = SIGN > 0 ? sin32(2 * e) : -sin32(2 * e);
                const float a0 = mt == 0 ? c : s;    // coefficient of Re x_m
                const float a1 = mt == 0 ? -s : c;   // coefficient of Im x_m
                tc_split<T>(make_float2(a0, a1), ahi[mt][kt][r], alo[mt][kt][r]);
            }
}

// The 16-point DFTs of eight butterflies (the MMA's columns) on the tensor
// cores: bh/bl are this lane's B fragments (points t, t+4, t+8, t+12 of
// butterfly g, twiddled and split), acc receives outputs g and g+8 of
// butterflies 2t and 2t+1 (acc[0][*] real parts, acc[1][*] imaginary parts;
// index r: 0/1 output g of butterfly 2t/2t+1, 2/3 output g+8).
template <class T>
__device__ __forceinline__ void tc_dft16_mma(float (&acc)[2][4], const uint32_t (&ahi)[2][2][4],
                                             const uint32_t (&alo)[2][2][4], const uint32_t (&bh)[4],
                                             const uint32_t (&bl)[4]) {
    __syncwarp();  // the operands may come from divergent paths; mma.sync needs the whole warp
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[mt][r] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            // small terms first, the hi x hi product last
            T::mma(acc[mt], ahi[mt][kt], bl[2 * kt], bl[2 * kt + 1]);
            T::mma(acc[mt], alo[mt][kt], bh[2 * kt], bh[2 * kt + 1]);
            T::mma(acc[mt], ahi[mt][kt], bh[2 * kt], bh[2 * kt + 1]);
        }
    }
}

// Loads of one butterfly column: point m = t + 4h of butterfly jj (k = jj mod
// Ns) is val(m) times w^m, w = exp(SIGN 2 pi i k / (16 Ns)), split hi/lo.
template <class T, int SIGN, typename Val>
__device__ __forceinline__ void tc_column(const float2 *__restrict__ tw, int Ns, int k, int t,
                                          uint32_t (&bh)[4], uint32_t (&bl)[4], Val &val) {
    const int tws = kTwN / (16 * Ns);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int m = t + 4 * h;
        float2 w = __ldg(&tw[(k * m) * tws]);  // k m < 16 Ns: inside the table
        if (SIGN < 0) w.y = -w.y;
        tc_split<T>(cmul(val(m), w), bh[h], bl[h]);
    }
}

// Stores of a pass's outputs: output q of butterfly jj (k = jj mod Ns) goes
// to (jj - k) 16 + k + q Ns; this lane holds q = g, g+8 of columns 2t, 2t+1,
// whose butterflies are jj_of(2t), jj_of(2t+1).
template <typename JJ>
__device__ __forceinline__ void tc_store(float2 *__restrict__ sm, int Ns, int g, int t,
                                         const float (&acc)[2][4], JJ &jj_of) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int jj = jj_of(2 * t + e);
        const int k = jj & (Ns - 1);
        const int base = (jj - k) * 16 + k;
        sm[tc_pad(base + g * Ns)] = make_float2(acc[0][e], acc[1][e]);
        sm[tc_pad(base + (g + 8) * Ns)] = make_float2(acc[0][2 + e], acc[1][2 + e]);
    }
}

// x * exp(SIGN 2 pi i n / 4): the radix-4 roots are +-1 and +-i.
template <int SIGN>
__device__ __forceinline__ float2 rot4(float2 x, int n) {
    n = (SIGN > 0 ? n : -n) & 3;
    if (n == 0) return x;
    if (n == 1) return make_float2(-x.y, x.x);
    if (n == 2) return make_float2(-x.x, -x.y);
    return make_float2(x.y, -x.x);
}

// The whole 16384-point FFT of the CTA's row (all 512 threads call it):
// X[t] = sum_m x[m] exp(SIGN 2 pi i m t / 16384).  Pass 0 (radix 4) reads its
// inputs through the caller: dense, load(m) for any m < 16384; sparse (every
// radix-4 butterfly {j + 4096 r} holds at most one nonzero input),
// first(j, r, x) returns whether butterfly j has one, with its position r and
// value x.  On return sm holds X[t] at tc_pad(t), natural order.
template <class T, int SIGN, typename Load, typename First>
__device__ __forceinline__ void tc_fft16384(float2 *__restrict__ sm, const float2 *__restrict__ tw,
                                            bool sparse, Load &load, First &first) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t ahi[2][2][4], alo[2][2][4];
    tc_dft16_afrag<T, SIGN>(ahi, alo, lane);
    constexpr int Q0 = kTcNL / 4;

    // ---- pass A: pass 0 on the fly + radix 16 with Ns = 4 ----
    // input point m of butterfly jj is pass-0 output p = jj + 1024 m, i.e.
    // output p & 3 of radix-4 butterfly p >> 2
    auto pass0_out = [&](int p) -> float2 {
        const int j = p >> 2, m0 = p & 3;
        if (sparse) {
            int r = 0;
            float2 x;
            if (!first(j, r, x)) return make_float2(0.f, 0.f);
            return rot4<SIGN>(x, r * m0);
        }
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 4; ++r) s = cadd(s, rot4<SIGN>(load(j + Q0 * r), r * m0));
        return s;
    };
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        const int jj0 = (warp + 16 * i) * 8;
        const int jj = jj0 + g;
        auto val = [&](int m) -> float2 { return pass0_out(jj + kTcNB * m); };
        uint32_t bh[4], bl[4];
        tc_column<T, SIGN>(tw, 4, jj & 3, t, bh, bl, val);
        float acc[2][4];
        tc_dft16_mma<T>(acc, ahi, alo, bh, bl);
        auto jj_of = [&](int n) { return jj0 + n; };
        tc_store(sm, 4, g, t, acc, jj_of);
    }
    __syncthreads();

    // ---- pass B: radix 16, Ns = 64; warp w owns residue classes 4w .. 4w+3 ----
#pragma unroll 1
    for (int kk = 0; kk < 4; ++kk) {
        const int k = 4 * warp + kk;
        float acc[2][2][4];
#pragma unroll
        for (int rho = 0; rho < 2; ++rho) {
            const int jj = k + 64 * (8 * rho + g);
            auto val = [&](int m) -> float2 { return sm[tc_pad(jj + kTcNB * m)]; };
            uint32_t bh[4], bl[4];
            tc_column<T, SIGN>(tw, 64, k, t, bh, bl, val);
            tc_dft16_mma<T>(acc[rho], ahi, alo, bh, bl);
        }
        __syncwarp();  // the class's 32 inputs are read before any of its outputs lands
#pragma unroll
        for (int rho = 0; rho < 2; ++rho) {
            auto jj_of = [&](int n) { return k + 64 * (8 * rho + n); };
            tc_store(sm, 64, g, t, acc[rho], jj_of);
        }
    }
    __syncthreads();

    // ---- pass C: radix 16, Ns = 1024; in place per butterfly ----
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        const int jj0 = (warp + 16 * i) * 8;
        const int jj = jj0 + g;
        auto val = [&](int m) -> float2 { return sm[tc_pad(jj + kTcNB * m)]; };
        uint32_t bh[4], bl[4];
        tc_column<T, SIGN>(tw, 1024, jj, t, bh, bl, val);
        float acc[2][4];
        tc_dft16_mma<T>(acc, ahi, alo, bh, bl);
        __syncwarp();  // the eight butterflies' inputs are read before their outputs land
        auto jj_of = [&](int n) { return jj0 + n; };
        tc_store(sm, 1024, g, t, acc, jj_of);
        __syncwarp();
    }
    __syncthreads();
}

}  // namespace cwtk
