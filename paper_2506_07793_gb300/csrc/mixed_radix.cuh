// mixed_radix.cuh -- Stockham FFT for 2,3,5,7-smooth lengths N <= 16384.
//
// Section "Fast Fourier transform" of arXiv 2506.07793 pads each signal to the
// smallest length whose prime factors are 2, 3, 5 and 7 (the fftpack radices)
// rather than to a power of two.  This header runs such a row on one CTA of
// 1024 threads:
//  * N = 16^q * 2^e * 3^b * 5^c * 7^d is split into a runtime pass schedule of
//    radices {16, 8, 4, 2, 3, 5, 7} (the power-of-two part first);
//  * pass p (radix R, Ns = product of the earlier radices) has N/R butterflies;
//    thread tid owns butterflies b = tid + i * 1024 and writes its outputs at
//    (b - k) R + k + r Ns, k = b mod Ns.  Up to N = 13312 two padded shared
//    buffers alternate (ping-pong) and a thread keeps one butterfly in
//    registers at a time; above that one buffer is used and each thread holds
//    all of a pass's inputs (at most 16 complex values) before writing;
//  * twiddles exp(+-2 pi i r k / (Ns R)) come from a per-length FP64-generated
//    table of the N-th roots of unity (index r k N / (Ns R));
//  * odd radices use the symmetric form X[k], X[R-k] = A_k +- B_k with
//    A_k = x0 + sum_r (x_r + x_{R-r}) cos(2 pi r k / R) and
//    B_k = SIGN i sum_r (x_r - x_{R-r}) sin(2 pi r k / R).
#pragma once

#include "fft_core.cuh"

namespace cwtk {

constexpr int kMrThreads = 1024;   // single-buffer mode
constexpr int kMrThreadsPP = 512;  // ping-pong mode (one butterfly live per thread)
constexpr int kMrPoints = 16;      // complex values per thread per pass (single-buffer mode)
constexpr int kMrMaxPasses = 16;

struct MrSchedule {
    int np;
    int radix[kMrMaxPasses];
};

// cos / sin (2 pi m / R) for the odd radices, m = 1..(R-1)/2 (mathematical constants).
__host__ __device__ constexpr float odd_cos(int R, int m) {
    return R == 3 ? -0.5f
         : R == 5 ? (m == 1 ? 0.309016994374947424102f : -0.809016994374947424102f)
         : (m == 1 ? 0.623489801858733530525f : m == 2 ? -0.222520933956314404289f
                                                          : -0.900968867902419126236f);
}
__host__ __device__ constexpr float odd_sin(int R, int m) {
    return R == 3 ? 0.866025403784438646764f
         : R == 5 ? (m == 1 ? 0.951056516295153572116f : 0.587785252292473129169f)
         : (m == 1 ? 0.781831482468029808708f : m == 2 ? 0.974927912181823607018f
                                                          : 0.433883739117558120475f);
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_odd(float2 *v) {
    constexpr int H = (R - 1) / 2;
    float2 s[H], d[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        s[r - 1] = cadd(v[r], v[R - r]);
        d[r - 1] = csub(v[r], v[R - r]);
    }
    float2 out[R];
    out[0] = v[0];
#pragma unroll
    for (int r = 0; r < H; ++r) out[0] = cadd(out[0], s[r]);
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float2 a = v[0], b = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const int m = (r * k) % R;                    // 1..R-1
            const int mm = m <= H ? m : R - m;            // cos is even, sin odd about R/2
            const float c = odd_cos(R, mm);
            const float sn = (m <= H ? 1.f : -1.f) * (SIGN > 0 ? 1.f : -1.f) * odd_sin(R, mm);
            a.x = fmaf(s[r - 1].x, c, a.x);
            a.y = fmaf(s[r - 1].y, c, a.y);
            b.x = fmaf(-d[r - 1].y, sn, b.x);             // i * d * sn
            b.y = fmaf(d[r - 1].x, sn, b.y);
        }
        out[k] = cadd(a, b);
        out[R - k] = csub(a, b);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = out[i];
}

template <int R, int SIGN>
__device__ __forceinline__ void dft_any(float2 *v) {
    if constexpr ((R & (R - 1)) == 0)
        dft<R, SIGN>(v);
    else
        dft_odd<R, SIGN>(v);
}

// v[r] *= w^r, r = 1..R-1 (power-of-two R: square-and-multiply chain).
template <int R>
__device__ __forceinline__ void mr_twiddle(float2 *v, float2 w1) {
    if constexpr ((R & (R - 1)) == 0) {
        twiddle_chain<R>(v, w1);
    } else {
        float2 w = w1;  // R <= 7: at most 5 successive products
#pragma unroll
        for (int r = 1; r < R; ++r) {
            v[r] = cmul(v[r], w);
            if (r + 1 < R) w = cmul(w, w1);
        }
    }
}

// One pass of radix R.  `first`: inputs come from load(k) instead of the
// buffer; `last`: outputs go to store(t, X[t]) instead of the buffer.
template <int R, int SIGN, typename Load, typename Store>
__device__ __forceinline__ void mr_pass(float2 *__restrict__ sm, const float2 *__restrict__ twN,
                                        int N, int Ns, bool first, bool last, Load &load,
                                        Store &store) {
    constexpr int MB = kMrPoints / R > 0 ? kMrPoints / R : 1;
    const int nb = N / R;
    const int tid = threadIdx.x;
    float2 v[MB][R];
#pragma unroll
    for (int i = 0; i < MB; ++i) {
        const int b = tid + i * kMrThreads;
        if (b < nb) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[i][r] = first ? load(b + r * nb) : sm[spad2(b + r * nb)];
        }
    }
    __syncthreads();  // every input of this pass is in registers
#pragma unroll
    for (int i = 0; i < MB; ++i) {
        const int b = tid + i * kMrThreads;
        if (b < nb) {
            const int k = b % Ns;
            if (Ns > 1) {
                float2 w1 = __ldg(&twN[k * (N / (Ns * R))]);
                if (SIGN < 0) w1.y = -w1.y;
                mr_twiddle<R>(v[i], w1);
            }
            dft_any<R, SIGN>(v[i]);
            if (last) {
#pragma unroll
                for (int r = 0; r < R; ++r) store(k + r * Ns, v[i][r]);
            } else {
                const int base = (b - k) * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) sm[spad2(base + r * Ns)] = v[i][r];
            }
        }
    }
    __syncthreads();  // outputs visible to the next pass
}

// Ping-pong form of a pass: inputs from `src` (or `load`), outputs to `dst`
// (or `store`); each thread handles its butterflies one at a time, so only R
// values are live.  Needs two buffers (N <= kMrPingPongMax).
template <int R, int SIGN, typename Load, typename Store>
__device__ __forceinline__ void mr_pass_pp(const float2 *__restrict__ src, float2 *__restrict__ dst,
                                           const float2 *__restrict__ twN, int N, int Ns, bool first,
                                           bool last, Load &load, Store &store) {
    const int nb = N / R;
#pragma unroll 1
    for (int b = threadIdx.x; b < nb; b += kMrThreadsPP) {
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = first ? load(b + r * nb) : src[spad2(b + r * nb)];
        const int k = b % Ns;
        if (Ns > 1) {
            float2 w1 = __ldg(&twN[k * (N / (Ns * R))]);
            if (SIGN < 0) w1.y = -w1.y;
            mr_twiddle<R>(v, w1);
        }
        dft_any<R, SIGN>(v);
        if (last) {
#pragma unroll
            for (int r = 0; r < R; ++r) store(k + r * Ns, v[r]);
        } else {
            const int base = (b - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[spad2(base + r * Ns)] = v[r];
        }
    }
    __syncthreads();
}

// Largest N whose two padded buffers fit one CTA's shared memory.
constexpr int kMrPingPongMax = 13312;

// The whole row: passes from the schedule, first reading `load`, last writing
// `store`.  One row per CTA of kMrThreadsPP (PP) or kMrThreads threads.  PP: `sm` holds two
// buffers of spad2(N) slots each (N <= kMrPingPongMax); otherwise one buffer
// and each pass keeps all of a thread's inputs in registers.
template <int SIGN, bool PP, typename Load, typename Store>
__device__ __forceinline__ void mr_row(float2 *__restrict__ sm, const float2 *__restrict__ twN, int N,
                                       const MrSchedule &sch, Load &load, Store &store) {
    int Ns = 1;
    float2 *src = sm, *dst = sm + (N + (N >> 4));
#pragma unroll 1
    for (int p = 0; p < sch.np; ++p) {
        const bool first = p == 0, last = p == sch.np - 1;
        if constexpr (PP) {
            switch (sch.radix[p]) {
                case 16: mr_pass_pp<16, SIGN>(src, dst, twN, N, Ns, first, last, load, store); break;
                case 8: mr_pass_pp<8, SIGN>(src, dst, twN, N, Ns, first, last, load, store); break;
                case 4: mr_pass_pp<4, SIGN>(src, dst, twN, N, Ns, first, last, load, store); break;
                case 2: mr_pass_pp<2, SIGN>(src, dst, twN, N, Ns, first, last, load, store); break;
                case 3: mr_pass_pp<3, SIGN>(src, dst, twN, N, Ns, first, last, load, store); break;
                case 5: mr_pass_pp<5, SIGN>(src, dst, twN, N, Ns, first, last, load, store); break;
                case 7: mr_pass_pp<7, SIGN>(src, dst, twN, N, Ns, first, last, load, store); break;
                default: break;
            }
            float2 *t = src;
            src = dst;
            dst = t;
        } else {
            switch (sch.radix[p]) {
                case 16: mr_pass<16, SIGN>(sm, twN, N, Ns, first, last, load, store); break;
                case 8: mr_pass<8, SIGN>(sm, twN, N, Ns, first, last, load, store); break;
                case 4: mr_pass<4, SIGN>(sm, twN, N, Ns, first, last, load, store); break;
                case 2: mr_pass<2, SIGN>(sm, twN, N, Ns, first, last, load, store); break;
                case 3: mr_pass<3, SIGN>(sm, twN, N, Ns, first, last, load, store); break;
                case 5: mr_pass<5, SIGN>(sm, twN, N, Ns, first, last, load, store); break;
                case 7: mr_pass<7, SIGN>(sm, twN, N, Ns, first, last, load, store); break;
                default: break;
            }
        }
        Ns *= sch.radix[p];
    }
}

}  // namespace cwtk
