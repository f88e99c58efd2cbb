// smooth.cu -- fused scale block for 2,3,5,7-smooth padded
// lengths (the padding policy of Section "Fast Fourier transform" of arXiv
// 2506.07793), on the mixed-radix rows of mixed_radix.cuh.  The arithmetic
// per row is that of fft_kernels.cu and scale_block.cu (Eq. 2); only the FFT
// length and its radices differ.  The host side picks each length's radix
// schedule with a cost model.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "phase.cuh"
#include "mixed_radix.cuh"

namespace cwtk {

namespace {

__global__ void twiddle_n_kernel(float2 *tw, int N) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < N) {
        double s, c;
        sincospi(2.0 * (double)m / (double)N, &s, &c);
        tw[m] = make_float2((float)c, (float)s);
    }
}

__device__ __noinline__ void mr_phase_f(float *dst, float2 v) { *dst = phase_atan2(v.y, v.x); }
__device__ __noinline__ void mr_phase_d(double *dst, float2 v) { *dst = (double)phase_atan2(v.y, v.x); }


struct MrArgs {
    const float2 *spec;
    const float *bank;
    const int *band;
    const float2 *twN;
    void *out_c, *out_p, *out_ph;
    int S, n_out, sub, total_rows, f64;
};

// Fused spectrum product, inverse FFT and epilogue per (channel, scale) row.
__global__ void __launch_bounds__(kMrThreads, 1)
mr_scale_block_kernel(const MrArgs a, const MrSchedule sch, int rows) {
    extern __shared__ float2 mrsm[];
    const int N = sch.N;
    const RowSlot rs = row_slot(sch, rows, a.total_rows);
    const int row = rs.active ? (int)blockIdx.x * rows + rs.rr : 0;
    const int rr = rs.rr < rows ? rs.rr : 0;
    float2 *sm = mrsm + (size_t)rr * (N + (N >> 4));
    const int c = row / a.S, s = row - c * a.S;
    const float2 *X = a.spec + (size_t)c * N;
    const float *W = a.bank + (size_t)s * N;
    const int b0 = a.band[2 * s], B = a.band[2 * s + 1];
    auto load = [=](int k) -> float2 {
        int dk = k - b0;  // the band is [b0, b0 + B) modulo N
        if (dk < 0) dk += N;
        if (dk < B) {
            const float2 xv = X[k];
            const float w = W[k];
            return make_float2(xv.x * w, xv.y * w);
        }
        return make_float2(0.f, 0.f);
    };
    // Narrow band (B <= N/R_0): butterfly b's inputs b + r nb, r < R_0, meet
    // the band at most once, at e = b0 + u (mod N) with u = (b - b0) mod nb.
    auto first_nz = [=](int b, int nb, unsigned mag, int &r, float2 &x) -> bool {
        const unsigned d = (unsigned)(b - b0 + N);  // > 0; N is a multiple of nb
        const int u = (int)(d - __umulhi(d, mag) * (unsigned)nb);
        if (u >= B) return false;
        int e = b0 + u;
        if (e >= N) e -= N;
        r = (int)__umulhi((unsigned)(e - b), mag);  // (e - b) / nb, exact: e = b (mod nb), e >= b
        const float2 xv = X[e];
        const float w = W[e];
        x = make_float2(xv.x * w, xv.y * w);
        return true;
    };
    const bool sparse = B <= N / sch.p[0].R;
    mr_row<+1>(sch, sm, a.twN, rs.j, rs.active, sparse, load, first_nz);
    if (!rs.active) return;
    // epilogue: crop to t < n, keep t = sub * o, write the requested outputs
    // (consecutive threads take consecutive o: coalesced stores)
    const size_t obase = (size_t)row * (size_t)a.n_out;
    const int sub = a.sub, n_out = a.n_out;
    if (a.f64) {
        double2 *oc = (double2 *)a.out_c + obase;
        double *op = (double *)a.out_p + obase, *oph = (double *)a.out_ph + obase;
#pragma unroll 1
        for (int o = rs.j; o < n_out; o += sch.T) {
            const float2 v = sm[spad2(o * sub)];
            if (a.out_c) oc[o] = make_double2(v.x, v.y);
            if (a.out_p) op[o] = (double)fmaf(v.x, v.x, v.y * v.y);
            if (a.out_ph) mr_phase_d(oph + o, v);
        }
    } else {
        float2 *oc = (float2 *)a.out_c + obase;
        float *op = (float *)a.out_p + obase, *oph = (float *)a.out_ph + obase;
#pragma unroll 2
        for (int o = rs.j; o < n_out; o += sch.T) {
            const float2 v = sm[spad2(o * sub)];
            if (a.out_c) oc[o] = v;
            if (a.out_p) op[o] = fmaf(v.x, v.x, v.y * v.y);
            if (a.out_ph) mr_phase_f(oph + o, v);
        }
    }
}

// ---- host: schedule ------------------------------------------------------

constexpr int kRadixSet[] = {4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 30, 32};

// Relative cost of one radix-R DFT (FP32 operations): radix-2 stages for
// powers of two, the symmetric form for 3, 5, 7, and for composite radices
// their nested factors plus the internal twiddle products.
double dft_cost(int R) {
    switch (R) {
        case 1: return 0.0;
        case 2: return 4.0;
        case 3: return 12.0;
        case 4: return 16.0;
        case 5: return 34.0;
        case 7: return 66.0;
        case 8: return 52.0;
        case 16: return 144.0;
        case 32: return 376.0;
        default: break;
    }
    const int R1 = first_factor(R), R2 = R / R1;
    return R2 * dft_cost(R1) + R1 * dft_cost(R2) + 6.0 * (R1 - 1) * (R2 - 1);
}
// One butterfly of a pass: the DFT, R - 1 twiddle products, staging R values
// in and out, and a fixed cost (twiddle-chain setup, index arithmetic,
// predication).  The fixed cost and the radix-32 weight were fitted to
// measured kernel times of 35 schedules at N = 100 ... 10000 (64 channels,
// 61 or 100 scales on GB300): with them the model picks the fastest measured
// schedule or one within 10% of it.
double butterfly_cost(int R) {
    return dft_cost(R) * (R == 32 ? 2.0 : 1.0) + 6.0 * (R - 1) + 8.0 * R + 120.0;
}
constexpr double kPassOverhead = 24.0;  // per thread and pass: barriers, call

void enumerate(int rem, int min_r, std::vector<int> &cur, std::vector<std::vector<int>> &out) {
    if (rem == 1) {
        out.push_back(cur);
        return;
    }
    if ((int)cur.size() >= kMrMaxPasses) return;
    for (int R : kRadixSet) {
        if (R < min_r || rem % R) continue;
        cur.push_back(R);
        enumerate(rem / R, R, cur, out);
        cur.pop_back();
    }
}

unsigned magic_of(int d) { return d <= 1 ? 0u : (unsigned)(((1ull << 32) + (unsigned)d - 1) / (unsigned)d); }

int g_sm_count[64] = {};

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!g_sm_count[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        g_sm_count[dev] = v;
    }
    return g_sm_count[dev];
}

constexpr int kMrRowSmemCap = 96 * 1024;          // several rows per CTA: at most this much
constexpr int kMrMaxSmem = (kMaxFft + (kMaxFft >> 4)) * 8;

// Rows per CTA for a launch over total_rows rows: up to 256 threads per CTA
// for short rows, but at least two CTAs per SM when there are enough rows.
int launch_rows(const MrSchedule &sch, int total_rows) {
    int rows = std::max(1, std::min(256, kMrThreads) / sch.T);
    const int want = (total_rows + 2 * sm_count() - 1) / (2 * sm_count());
    rows = std::max(1, std::min(rows, want));
    const int per_row = (sch.N + (sch.N >> 4)) * 8;
    while (rows > 1 && rows * per_row > kMrRowSmemCap) --rows;
    return rows;
}

int round_up32(int x) { return (x + 31) & ~31; }

cudaError_t mr_sb_launch(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st) {
    static unsigned done = 0;
    cudaError_t e = ensure_smem_attr(mr_scale_block_kernel, kMrMaxSmem, &done);
    if (e != cudaSuccess) return e;
    const int rows = launch_rows(p->sch, a.total_rows);
    const int smem = rows * (p->N + (p->N >> 4)) * 8;
    mr_scale_block_kernel<<<(a.total_rows + rows - 1) / rows, round_up32(rows * p->sch.T), smem, st>>>(
        a, p->sch, rows);
    return cudaGetLastError();
}

}  // namespace

int mr_launch_rows(const MrSchedule &sch, int total_rows) { return launch_rows(sch, total_rows); }

bool mr_schedule(int N, MrSchedule *out) {
    if (N < kMinFft || N > kMaxFft) return false;
    int x = N;
    for (int f : {2, 3, 5, 7})
        while (x % f == 0) x /= f;
    if (x != 1) return false;
    std::vector<std::vector<int>> cands;
    std::vector<int> cur;
    enumerate(N, 2, cur, cands);
    double best = 0.0;
    int best_i = -1, best_T = 0;
    for (int i = 0; i < (int)cands.size(); ++i) {
        const std::vector<int> &rs = cands[i];
        int Tmin = 1;
        for (int R : rs) {
            const int gm = std::max(1, kMrPoints / R);  // mr_gmax
            Tmin = std::max(Tmin, (N / R + gm - 1) / gm);
        }
        for (int T = Tmin; T <= kMrThreads; ++T) {
            double c = kPassOverhead * (double)rs.size();
            for (int R : rs) c += (double)((N / R + T - 1) / T) * butterfly_cost(R);
            c *= T;
            if (best_i < 0 || c < best * (1.0 - 1e-9) ||
                (c <= best * (1.0 + 1e-9) && rs.size() < cands[best_i].size())) {
                best = c;
                best_i = i;
                best_T = T;
            }
        }
    }
    if (best_i < 0) return false;
    MrSchedule s{};
    s.N = N;
    s.T = best_T;
    s.np = (int)cands[best_i].size();
    int Ns = 1;
    for (int q = 0; q < s.np; ++q) {
        const int R = cands[best_i][q];
        s.p[q].R = R;
        s.p[q].G = (N / R + best_T - 1) / best_T;
        s.p[q].Ns = Ns;
        s.p[q].mag = magic_of(Ns);
        s.p[q].tws = N / (Ns * R);
        Ns *= R;
    }
    s.mag0 = magic_of(N / s.p[0].R);
    *out = s;
    return true;
}

cudaError_t make_twiddles_n(int N, float2 *tw, cudaStream_t st) {
    twiddle_n_kernel<<<(N + 255) / 256, 256, 0, st>>>(tw, N);
    return cudaGetLastError();
}

cudaError_t launch_scale_block_mr(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                  cudaStream_t st) {
    MrArgs a;
    a.spec = p->spec;
    a.bank = p->bank;
    a.band = p->band;
    a.twN = p->twN;
    a.out_c = out_c;
    a.out_p = out_p;
    a.out_ph = out_ph;
    a.S = p->S;
    a.n_out = p->n_out;
    a.sub = p->d;
    a.total_rows = p->C * p->S;
    a.f64 = p->io == CWT_DTYPE_F64;
    return mr_sb_launch(p, a, st);
}

}  // namespace cwtk
