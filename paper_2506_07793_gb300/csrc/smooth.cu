// smooth.cu -- fused scale block for 2,3,5,7-smooth padded
// lengths (the padding policy of Section "Fast Fourier transform" of arXiv
// 2506.07793), on the mixed-radix rows of mixed_radix.cuh.  The arithmetic
// per row is that of fft_kernels.cu and scale_block.cu (Eq. 2); only the FFT
// length and its radices differ.  The host side picks each length's radix
// schedule with a cost model.
#include <cuda_runtime.h>

#include <algorithm>
#include <iterator>
#include <vector>

#include "smooth_kernel.cuh"

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

void enumerate(int rem, int min_r, std::vector<int> &cur, std::vector<std::vector<int>> &out,
               const std::vector<int> &allowed) {
    if (rem == 1) {
        out.push_back(cur);
        return;
    }
    if ((int)cur.size() >= kMrMaxPasses) return;
    for (int R : allowed) {
        if (R < min_r || rem % R) continue;
        cur.push_back(R);
        enumerate(rem / R, R, cur, out, allowed);
        cur.pop_back();
    }
}

std::atomic<int> g_sm_count[64] = {};

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = g_sm_count[dev].load(std::memory_order_relaxed);
    if (!v) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        g_sm_count[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

constexpr int kMrRowSmemCap = 96 * 1024;          // several rows per CTA: at most this much

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



}  // namespace

int mr_launch_rows(const MrSchedule &sch, int total_rows) { return launch_rows(sch, total_rows); }

namespace {

// Cheapest schedule of N over the given radices (cost model above), or
// cost < 0 when none fits 32 values per thread and 512 threads per row.
struct Plan1 {
    double cost = -1.0;
    std::vector<int> radices;
    int T = 0;
};

Plan1 search(int N, const std::vector<int> &allowed) {
    std::vector<std::vector<int>> cands;
    std::vector<int> cur;
    enumerate(N, 2, cur, cands, allowed);
    Plan1 best;
    for (const std::vector<int> &rs : cands) {
        int Tmin = 1;
        for (int R : rs) {
            const int gm = std::max(1, kMrPoints / R);  // mr_gmax
            Tmin = std::max(Tmin, (N / R + gm - 1) / gm);
        }
        for (int T = Tmin; T <= kMrThreads; ++T) {
            double c = kPassOverhead * (double)rs.size();
            for (int R : rs) c += (double)((N / R + T - 1) / T) * butterfly_cost(R);
            c *= T;
            if (best.cost < 0 || c < best.cost * (1.0 - 1e-9) ||
                (c <= best.cost * (1.0 + 1e-9) && rs.size() < best.radices.size())) {
                best.cost = c;
                best.radices = rs;
                best.T = T;
            }
        }
    }
    return best;
}

// An inlined radix pair is taken when its best schedule costs at most this
// much more than the best over all radices (the model counts operations; the
// inlined rows run about 1.35x more of them per second).
constexpr double kFastPairGain = 1.3;

}  // namespace

namespace {

// The schedule of N with passes `radices` (in order) and T threads per row.
MrSchedule build_schedule(int N, const std::vector<int> &radices, int T, int fast) {
    MrSchedule s{};
    s.N = N;
    s.T = T;
    s.fast = fast;
    s.np = (int)radices.size();
    int Ns = 1;
    for (int q = 0; q < s.np; ++q) {
        const int R = radices[q];
        s.p[q].R = R;
        s.p[q].G = (N / R + T - 1) / T;
        s.p[q].Ns = Ns;
        s.p[q].mag = mr_magic(Ns);
        s.p[q].tws = N / (Ns * R);
        Ns *= R;
    }
    s.mag0 = mr_magic(N / s.p[0].R);
    s.fixed = -1;
    s.fixed_cl = -1;
    return s;
}

// Whole warps of 128 for rows of more than 128 threads (see mr_schedule).
int round_threads(int T) { return T > 128 ? std::min(kMrThreads, (T + 127) / 128 * 128) : T; }

}  // namespace

int mr_schedule_candidates(int N, MrSchedule *out, int max_out) {
    MrSchedule first;
    if (max_out < 1 || !mr_schedule(N, &first)) return 0;
    out[0] = first;
    out[0].fast = -1;
    int n = 1;
    // the same passes on fewer or more threads: the least whole-warp count that
    // fits, one warp more, and the count rounded up to 128 (10000 = 16 x 25 x 25
    // ran 8% faster on 416 threads than on 512)
    {
        std::vector<int> rs;
        for (int q = 0; q < first.np; ++q) rs.push_back(first.p[q].R);
        int Tmin = 1;
        for (int R : rs) {
            const int gm = std::max(1, kMrPoints / R);
            Tmin = std::max(Tmin, (N / R + gm - 1) / gm);
        }
        const int w = (Tmin + 31) / 32 * 32;
        int added = 0;
        for (int T : {w, w + 32, round_threads(Tmin)}) {
            if (T == first.T || T > kMrThreads || T < 128 || added == 2 || n >= max_out) continue;
            bool dup = false;
            for (int i = 0; i < n; ++i) dup = dup || out[i].T == T;
            if (dup) continue;
            out[n++] = build_schedule(N, rs, T, -1);
            ++added;
        }
    }
    // the cheapest radix multisets under the cost model, each in its distinct pass orders
    std::vector<std::vector<int>> sets;
    std::vector<int> cur;
    const std::vector<int> all(std::begin(kRadixSet), std::end(kRadixSet));
    enumerate(N, 2, cur, sets, all);
    std::vector<std::pair<double, std::vector<int>>> ranked;
    for (const std::vector<int> &rs : sets) {
        int Tmin = 1;
        for (int R : rs) {
            const int gm = std::max(1, kMrPoints / R);
            Tmin = std::max(Tmin, (N / R + gm - 1) / gm);
        }
        if (Tmin > kMrThreads) continue;
        double best = -1.0;
        for (int T = Tmin; T <= kMrThreads; ++T) {
            double c = kPassOverhead * (double)rs.size();
            for (int R : rs) c += (double)((N / R + T - 1) / T) * butterfly_cost(R);
            c *= T;
            if (best < 0 || c < best) best = c;
        }
        ranked.push_back({best, rs});
    }
    std::sort(ranked.begin(), ranked.end(),
              [](const std::pair<double, std::vector<int>> &a, const std::pair<double, std::vector<int>> &b) {
                  return a.first < b.first;
              });
    for (size_t m = 0; m < ranked.size() && m < 2 && n < max_out; ++m) {
        std::vector<int> order = ranked[m].second;
        std::sort(order.begin(), order.end());
        do {
            int Tmin = 1;
            for (int R : order) {
                const int gm = std::max(1, kMrPoints / R);
                Tmin = std::max(Tmin, (N / R + gm - 1) / gm);
            }
            const MrSchedule c = build_schedule(N, order, round_threads(Tmin), -1);
            bool seen = false;
            for (int i = 0; i < n && !seen; ++i) {
                seen = out[i].np == c.np && out[i].T == c.T;
                for (int q = 0; seen && q < c.np; ++q) seen = out[i].p[q].R == c.p[q].R;
            }
            if (!seen) out[n++] = c;
        } while (n < max_out && std::next_permutation(order.begin(), order.end()));
    }
    return n;
}

// Pass orders measured on GB300 for whole-second lengths with compiled-in
// kernels: the plan-time tuner (cwt_options.specialize = 2) on 64 channels x
// 100 scales found them 3-39% faster than the cost model's order (which
// ranks radix sets, not orders), and the fixed-length kernels are compiled
// for them (CWT_MR_FIXED); 12288 is the cluster local row of CWT_CL_MR_FIXED,
// timed on 32 channels of the 128-scale, 122880-point rows of a minute at
// 2048 Hz.  T is the least thread count that fits.
struct MeasuredOrder {
    int N;
    int radices[4];
    int T;  // threads per row; 0: the least that fits, rounded up to 128
};
constexpr MeasuredOrder kMeasuredOrders[] = {
    {5000, {20, 10, 25}},       {4000, {16, 10, 25}},      {2500, {25, 10, 10}},     {2000, {20, 10, 10}},
    {7500, {25, 10, 30}},       {6000, {24, 10, 25}},      {3000, {24, 5, 25}},      {9000, {24, 15, 25}},
    {14000, {14, 10, 10, 10}},  {13500, {6, 10, 15, 15}},  {12500, {10, 10, 5, 25}}, {3750, {25, 6, 25}},
    {1750, {14, 5, 25}},        {1250, {25, 10, 5}},
    {12288, {32, 16, 24}},  // 122880 = 10 x 12288: 3.90 against 4.04 ms (16, 24, 32)
    // Thread counts below the 128-rounded one: fewer threads idle in the passes with the fewest
    // butterflies, and more registers a thread.  Tuner timings per launch (64 channels x 100
    // scales) against the same passes on the rounded count: 10000 on 416 threads 0.0840 against
    // 0.0901 ms (0.236 against 0.256 ms per step), 10500 on 448 0.0997 against 0.1061, 8000 on
    // 416 0.0795 against 0.0813, 7000 on 288 0.0902 against 0.0941, 4500 on 160 0.0900 against
    // 0.0964, 3500 on 192 0.0853 against 0.0883.
    {10000, {16, 25, 25}, 416}, {10500, {28, 15, 25}, 448}, {8000, {16, 25, 20}, 416},
    {7000, {28, 10, 25}, 288},  {4500, {10, 15, 30}, 160},  {3500, {28, 5, 25}, 192},
};

bool mr_schedule(int N, MrSchedule *out) {
    if (N < kMinFft || N > kMaxFft) return false;
    int x = N;
    for (int f : {2, 3, 5, 7})
        while (x % f == 0) x /= f;
    if (x != 1) return false;
    for (const MeasuredOrder &m : kMeasuredOrders) {
        if (m.N != N) continue;
        std::vector<int> rs;
        for (int R : m.radices)
            if (R) rs.push_back(R);
        int Tmin = 1;
        for (int R : rs) {
            const int gm = std::max(1, kMrPoints / R);
            Tmin = std::max(Tmin, (N / R + gm - 1) / gm);
        }
        MrSchedule s = build_schedule(N, rs, m.T ? m.T : round_threads(Tmin), -1);
        s.fixed = mr_fixed_index(s);
        *out = s;
        return true;
    }
    const std::vector<int> all(std::begin(kRadixSet), std::end(kRadixSet));
    Plan1 best = search(N, all);
    if (best.cost < 0) return false;
    int fast = -1;
    Plan1 fbest;
#define CWT_MR_TRY(I, A, B)                                                               \
    {                                                                                     \
        Plan1 f = search(N, {A, B});                                                      \
        if (f.cost >= 0 && f.cost <= kFastPairGain * best.cost && (fast < 0 || f.cost < fbest.cost)) { \
            fast = I;                                                                     \
            fbest = f;                                                                    \
        }                                                                                 \
    }
    CWT_MR_FAST_PAIRS(CWT_MR_TRY)
#undef CWT_MR_TRY
    if (fast >= 0) best = fbest;
    // A row of more than 128 threads has a CTA to itself; whole warps of 128
    // run it faster than the cost model's tightest T (measured on GB300:
    // N = 10000 at T = 400 -> 512, 354 -> 342 us; N = 5000 at 209 -> 256,
    // 111 -> 106 us).  A larger T never raises a pass's butterflies per thread.
    if (best.T > 128) best.T = std::min(kMrThreads, (best.T + 127) / 128 * 128);
    MrSchedule s = build_schedule(N, best.radices, best.T, fast);
    s.fixed = mr_fixed_index(s);
    *out = s;
    return true;
}

cudaError_t make_twiddles_n(int N, float2 *tw, cudaStream_t st) {
    twiddle_n_kernel<<<(N + 255) / 256, 256, 0, st>>>(tw, N);
    return cudaGetLastError();
}

cudaError_t launch_scale_block_mr(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                  cudaStream_t st) {
    if (p->cl > 1) return launch_scale_block_mr_cluster(p, out_c, out_p, out_ph, st);
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
    if (p->jit) return jit_sb_launch(p, a, st);
    if (p->sch.fixed >= 0) return mr_fixed_sb_launch(p, a, st);
    switch (p->sch.fast) {
#define CWT_MR_CASE(I, A, B) \
    case I: return mr_sb_launch<A, B>(p, a, st);
        CWT_MR_FAST_PAIRS(CWT_MR_CASE)
#undef CWT_MR_CASE
        default: return mr_sb_launch<0, 0>(p, a, st);
    }
}

}  // namespace cwtk
