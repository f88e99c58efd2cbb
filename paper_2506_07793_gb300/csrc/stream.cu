// stream.cu -- streaming overlap-save CWT for live multichannel EEG.
//
// The paper's goal is real-time EEG analysis (Abstract; Discussion: 64
// channels processed several times per second on a laptop GPU and on a
// single-board computer).  This server keeps many live streams on one GPU:
//
//  * Stream s has C_s channels at fs_s Hz, hop H_s = ceil(fs_s * hop_seconds)
//    samples and window W (= the FFT length N).  Its device ring holds the
//    last W + kMaxPending * H_s samples of every channel; samples before the
//    first push are zero.
//  * Hop h (h = 1, 2, ...) ends at sample e_h = h * H_s and is ready once e_h
//    samples have been pushed.  Its result is the cyclic CWT (Eq. 2, N = W) of
//    the window x[e_h - W, e_h), kept at window positions
//    [W - D - H, W - D) with D = floor((W - H) / 2): the H outputs centred in
//    the window, i.e. absolute times [e_h - D - H, e_h - D).
//  * cwt_server_step gathers every ready hop of every open stream into one
//    launch (continuous batching): streams that joined since the last step
//    are simply in the next batch, and closed streams leave it.  Two batches
//    may be in flight; results are copied to each stream's pinned host queue
//    and a host callback stamps the completion time, so latency is measured
//    from the moment a hop became ready to the moment its power is in host
//    memory.
//  * Admission: a stream is refused (CWT_EBUSY) when no slot is free or its
//    device memory (ring + its share of the batch buffers) would exceed the
//    server's budget.  The batch buffers of both in-flight slots are grown at
//    admission to the bound of every open stream (kMaxPending hops each), so
//    cwt_server_step never allocates.
//  * Pushes copy into the rings on a copy stream of their own; each batch
//    waits for an event recorded there, so a push never queues behind a batch
//    in flight.  A push cannot overwrite ring samples that a batch in flight
//    still reads: with at most kMaxPending hops pending, the oldest window in
//    flight starts after the last sample the push overwrites.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "fft_core.cuh"
#include "internal.h"

namespace cwtk {
namespace {

constexpr int kSW = 2048;          // window = FFT length
constexpr int kSThreads = 512;
constexpr int kSR = 16;
constexpr int kMaxPending = 8;     // hops a stream may have waiting for a step
constexpr int kSlots = 2;          // batches in flight

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct StreamItem {
    const float *ring;  // channel row of the stream's ring
    float *out;         // [S][H] block of this (hop, channel)
    const float *bank;  // [S][W]
    const int *band;    // [S][2]
    long long start;    // absolute index of the window's first sample (may be < 0)
    int cap;            // ring length per channel
    int H, D;
};

// One (hop, channel) per CTA: forward FFT of the window into shared memory,
// then every scale's band product + inverse FFT, keeping the H centred outputs.
__global__ void __launch_bounds__(kSThreads) stream_kernel(const StreamItem *__restrict__ items,
                                                           const float2 *__restrict__ tw, int S) {
    constexpr int T = kSW / kSR;  // 128 threads per row
    constexpr int P = kSThreads / T;
    __shared__ float2 spec[kSW];
    extern __shared__ float2 ssm[];
    const StreamItem it = items[blockIdx.x];
    const int rl = threadIdx.x / T, j = threadIdx.x % T;
    float2 *st = ssm + rl * FftShape<kSW, kSR>::SMEM_F2;
    // forward: only row-slot 0 holds data; the other slots transform zeros
    {
        const bool act = rl == 0;
        auto load = [&](int i) -> float2 {
            const long long a = it.start + i;
            float v = 0.f;
            if (act && a >= 0) v = it.ring[a % it.cap];
            return make_float2(v, 0.f);
        };
        auto store = [&](int t, float2 v) {
            if (act) spec[CWT_IDX(t, kSW)] = v;
        };
        fft_row<kSW, kSR, -1>(st, tw, j, load, store);
    }
    __syncthreads();
    const int lo = kSW - it.D - it.H;  // first kept window position
#pragma unroll 1
    for (int s0 = 0; s0 < S; s0 += P) {
        const int s = s0 + rl;
        const bool act = s < S;
        const float *W = it.bank + (size_t)(act ? s : 0) * kSW;
        const int b0 = it.band[2 * (act ? s : 0)], B = act ? it.band[2 * s + 1] : 0;
        auto load = [&](int k) -> float2 {
            if (((k - b0) & (kSW - 1)) < B) {
                const float2 x = spec[CWT_IDX(k, kSW)];
                const float w = __ldg(&W[k]);
                return make_float2(x.x * w, x.y * w);
            }
            return make_float2(0.f, 0.f);
        };
        float *o = it.out + (size_t)(act ? s : 0) * it.H;
        auto store = [&](int t, float2 v) {
            const int q = t - lo;
            if (act && q >= 0 && q < it.H) o[q] = fmaf(v.x, v.x, v.y * v.y);
        };
        fft_row<kSW, kSR, +1>(st, tw, j, load, store);
    }
}

constexpr int kStreamSmem = (kSThreads / (kSW / kSR)) * FftShape<kSW, kSR>::SMEM_F2 * 8;

struct Hop {
    long long e;         // window end (absolute samples)
    double t_ready;      // wall time the hop became ready
    double t_done = -1;  // wall time its output reached host memory
    int slot_out = -1;   // index in the stream's host queue
};

struct Stream {
    int id = -1;
    int C = 0, H = 0, D = 0, cap = 0;
    double fs = 0;
    int bank = -1;
    float *d_ring = nullptr;
    long long pushed = 0;
    long long next_e = 0;  // end of the next hop to become ready
    std::deque<Hop> waiting;     // ready, not yet launched
    std::deque<Hop> inflight;    // launched, not yet complete
    std::deque<Hop> done;        // complete, not yet pulled
    float *h_queue = nullptr;    // pinned [kMaxPending * 2][C][S][H]
    int queue_slots = 0;
    std::vector<int> free_slots;
    size_t dev_bytes = 0;
    bool open = false;
    bool reserved = false;  // slot taken by an open in progress
};

struct Bank {
    double fs;
    float *bank = nullptr;
    int *band = nullptr;
};

struct Slot {
    StreamItem *d_items = nullptr, *h_items = nullptr;
    size_t items_cap = 0;
    float *d_out = nullptr;
    size_t out_cap = 0;  // floats
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<std::pair<int, long long>> hops;  // (stream id, e) carried by this batch
};

}  // namespace
}  // namespace cwtk

struct cwt_server_s {
    int device = 0;
    std::vector<double> freqs, cycles;
    int S = 0, wavelet = 0;
    cwt_server_options opt{};
    std::vector<cwtk::Stream> streams;  // index = stream id
    std::vector<cwtk::Bank> banks;
    cwtk::Slot slots[cwtk::kSlots];
    int next_slot = 0;
    size_t dev_bytes = 0;
    std::mutex mu;  // guards hop completion (host callback) vs. host calls
    std::vector<double> latencies;
    long long admitted = 0, refused = 0, hops_done = 0, launches = 0;
    long long coeffs_done = 0;
    double first_ready = -1, last_done = -1;
    const float2 *tw = nullptr;
    cudaStream_t st = nullptr;   // the server's own CUDA stream (batches)
    cudaStream_t cst = nullptr;  // pushes into the rings
    cudaEvent_t pushed = nullptr;  // recorded on cst before each batch
    size_t bound_items = 0, bound_out = 0;  // batch-buffer bound of the open streams
    std::string last_error;
};

namespace cwtk {
namespace {

struct DoneCtx {
    cwt_server_s *srv;
    int slot;
};

// Host callback after a batch's results reached host memory.
void CUDART_CB on_batch_done(void *arg) {
    DoneCtx *ctx = (DoneCtx *)arg;
    cwt_server_s *srv = ctx->srv;
    const double t = now_s();
    std::lock_guard<std::mutex> lk(srv->mu);
    Slot &sl = srv->slots[ctx->slot];
    for (auto &h : sl.hops) {
        Stream &s = srv->streams[h.first];
        for (auto it = s.inflight.begin(); it != s.inflight.end(); ++it) {
            if (it->e == h.second) {
                Hop hop = *it;
                hop.t_done = t;
                s.inflight.erase(it);
                s.done.push_back(hop);
                srv->latencies.push_back(t - hop.t_ready);
                srv->hops_done++;
                srv->coeffs_done += (long long)s.C * srv->S * s.H;
                srv->last_done = t;
                break;
            }
        }
    }
    sl.busy = false;
    delete ctx;
}

// Index of the bank for fs, generating it if new.  Called without the
// server mutex (it allocates and waits for the generator).
cudaError_t bank_for(cwt_server_s *srv, double fs, int *idx) {
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (size_t i = 0; i < srv->banks.size(); ++i)
            if (srv->banks[i].fs == fs) {
                *idx = (int)i;
                return cudaSuccess;
            }
    }
    Bank b;
    b.fs = fs;
    cudaError_t e = cwtk::dmalloc(&b.bank, sizeof(float) * (size_t)srv->S * kSW);
    if (e == cudaSuccess) e = cwtk::dmalloc(&b.band, sizeof(int) * 2 * (size_t)srv->S);
    if (e == cudaSuccess) {
        // reuse the plan generator through a temporary plan description, on a
        // private stream so that in-flight batches are not waited for
        cwt_plan_s tmp;
        tmp.S = srv->S;
        tmp.fs = fs;
        tmp.wavelet = srv->wavelet;
        tmp.gmw_gamma = srv->opt.gmw_gamma;
        tmp.freqs = srv->freqs;
        tmp.cycles = srv->cycles;
        cudaStream_t bs = nullptr;
        e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = launch_bank_n(&tmp, kSW, b.bank, b.band, bs, nullptr);
        if (bs) cudaStreamDestroy(bs);
    }
    if (e != cudaSuccess) {
        cudaFree(b.bank);
        cudaFree(b.band);
        return e;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->dev_bytes += sizeof(float) * (size_t)srv->S * kSW + sizeof(int) * 2 * (size_t)srv->S;
    srv->banks.push_back(b);
    *idx = (int)srv->banks.size() - 1;
    return cudaSuccess;
}

// Grow both slots' batch buffers to hold `items` work items and `outf`
// output floats.  The new buffers are allocated first, so a failure leaves
// every slot as it was; a slot's batch in flight is waited for before its
// buffers are replaced.  Called at admission, never by cwt_server_step.
cudaError_t grow_slots(cwt_server_s *srv, size_t items, size_t outf) {
    for (Slot &sl : srv->slots) {
        if (sl.items_cap >= items && sl.out_cap >= outf) continue;
        StreamItem *d_items = nullptr, *h_items = nullptr;
        float *d_out = nullptr;
        cudaError_t e = cudaSuccess;
        if (sl.items_cap < items) {
            e = cwtk::dmalloc(&d_items, sizeof(StreamItem) * items);
            if (e == cudaSuccess) e = cwtk::hmalloc(&h_items, sizeof(StreamItem) * items);
        }
        if (e == cudaSuccess && sl.out_cap < outf) e = cwtk::dmalloc(&d_out, sizeof(float) * outf);
        if (e == cudaSuccess && sl.busy) e = cudaEventSynchronize(sl.done);
        if (e != cudaSuccess) {
            cudaFree(d_items);
            if (h_items) cudaFreeHost(h_items);
            cudaFree(d_out);
            return e;
        }
        if (d_items) {
            cudaFree(sl.d_items);
            if (sl.h_items) cudaFreeHost(sl.h_items);
            sl.d_items = d_items;
            sl.h_items = h_items;
            sl.items_cap = items;
        }
        if (d_out) {
            cudaFree(sl.d_out);
            sl.d_out = d_out;
            sl.out_cap = outf;
        }
    }
    return cudaSuccess;
}

size_t stream_dev_bytes(const cwt_server_s *srv, int C, int H) {
    const size_t ring = sizeof(float) * (size_t)C * (kSW + (size_t)kMaxPending * H);
    const size_t outs = sizeof(float) * (size_t)C * srv->S * H * kMaxPending * kSlots;
    return ring + outs;
}

}  // namespace
}  // namespace cwtk

using namespace cwtk;

namespace {
struct Guard {
    int prev = -1;
    bool ok = false;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
cwt_status cuda_fail(cwt_server_s *s, cudaError_t e) {
    if (s) s->last_error = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CWT_ENOMEM : CWT_ECUDA;
}
}  // namespace

extern "C" {

// the Python binding mirrors this layout
static_assert(sizeof(cwt_server_options) == 56 && offsetof(cwt_server_options, gmw_gamma) == 32,
              "cwt_server_options layout");

cwt_status cwt_server_options_init(cwt_server_options *o) {
    if (!o) return CWT_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->max_streams = 32;
    o->mem_budget_bytes = 0;
    o->hop_seconds = 0.05;
    o->window = kSW;
    o->output_kinds = CWT_OUT_POWER;
    o->gmw_gamma = 3.0;
    return CWT_OK;
}

cwt_status cwt_server_create(cwt_server *out, const double *freqs_hz, const double *n_cycles,
                             int n_freqs, int wavelet, const cwt_server_options *opt) {
    if (!out || !freqs_hz || !n_cycles || n_freqs < 1) return CWT_EINVAL;
    for (int i = 0; i < n_freqs; ++i)
        if (!(freqs_hz[i] > 0.0) || !std::isfinite(freqs_hz[i]) || !(n_cycles[i] > 0.0) ||
            !std::isfinite(n_cycles[i]))
            return CWT_EINVAL;
    cwt_server_options o;
    cwt_server_options_init(&o);
    if (opt) o = *opt;
    if (!wavelet_params_ok(wavelet, n_cycles, n_freqs, o.gmw_gamma)) return CWT_EINVAL;
    if (o.max_streams < 1 || !(o.hop_seconds > 0.0) || !std::isfinite(o.hop_seconds)) return CWT_EINVAL;
    if (o.window != kSW) return CWT_EUNSUPPORTED;
    if (o.output_kinds != CWT_OUT_POWER) return CWT_EUNSUPPORTED;
    cwt_server_s *s = new (std::nothrow) cwt_server_s();
    if (!s) return CWT_ENOMEM;
    s->freqs.assign(freqs_hz, freqs_hz + n_freqs);
    s->cycles.assign(n_cycles, n_cycles + n_freqs);
    s->S = n_freqs;
    s->wavelet = wavelet;
    s->opt = o;
    s->streams.resize(o.max_streams);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = device_twiddles(&s->tw);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->pushed, cudaEventDisableTiming);
    static std::atomic<unsigned> attr{0};
    if (e == cudaSuccess) e = ensure_smem_attr(stream_kernel, kStreamSmem, &attr);
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->slots[i].done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cwt_status r = cuda_fail(s, e);
        if (s->st) cudaStreamDestroy(s->st);
        if (s->cst) cudaStreamDestroy(s->cst);
        if (s->pushed) cudaEventDestroy(s->pushed);
        for (auto &sl : s->slots)
            if (sl.done) cudaEventDestroy(sl.done);
        delete s;
        return r;
    }
    *out = s;
    return CWT_OK;
}

cwt_status cwt_server_destroy(cwt_server s) {
    if (!s) return CWT_OK;
    {
        Guard g(s->device);
        cudaStreamSynchronize(s->cst);
        cudaStreamSynchronize(s->st);
        for (auto &st : s->streams) {
            cudaFree(st.d_ring);
            if (st.h_queue) cudaFreeHost(st.h_queue);
        }
        for (auto &b : s->banks) {
            cudaFree(b.bank);
            cudaFree(b.band);
        }
        for (auto &sl : s->slots) {
            cudaFree(sl.d_items);
            cudaFree(sl.d_out);
            if (sl.h_items) cudaFreeHost(sl.h_items);
            if (sl.done) cudaEventDestroy(sl.done);
        }
        cudaStreamDestroy(s->st);
        cudaStreamDestroy(s->cst);
        cudaEventDestroy(s->pushed);
    }
    delete s;
    return CWT_OK;
}

cwt_status cwt_stream_open(cwt_server s, int channels, double fs, int *stream_id) {
    if (!s || !stream_id || channels < 1 || !(fs > 0.0) || !std::isfinite(fs)) return CWT_EINVAL;
    for (double f : s->freqs)
        if (!(f < 0.5 * fs)) return CWT_EINVAL;
    if (!scales_on_grid(s->wavelet, s->freqs.data(), s->cycles.data(), s->S, s->opt.gmw_gamma, fs, kSW))
        return CWT_EINVAL;
    const int H = (int)std::ceil(fs * s->opt.hop_seconds - 1e-9);
    if (H < 1 || H > kSW / 2) return CWT_EINVAL;
    Guard g(s->device);
    if (!g.ok) return CWT_ECUDA;
    const size_t need = stream_dev_bytes(s, channels, H);
    int id = -1;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int i = 0; i < (int)s->streams.size(); ++i)
            if (!s->streams[i].open && !s->streams[i].reserved && s->streams[i].inflight.empty()) {
                id = i;
                break;
            }
        if (id < 0 || (s->opt.mem_budget_bytes && s->dev_bytes + need > s->opt.mem_budget_bytes)) {
            s->refused++;
            return CWT_EBUSY;
        }
        s->streams[id].reserved = true;  // the slot and its bytes are ours from here
        s->dev_bytes += need;
    }
    int b = -1;
    cudaError_t e = bank_for(s, fs, &b);
    Stream st;
    st.id = id;
    st.C = channels;
    st.fs = fs;
    st.H = H;
    st.D = (kSW - H) / 2;
    st.cap = kSW + kMaxPending * H;
    st.bank = b;
    st.next_e = H;
    st.queue_slots = kMaxPending * 2;
    const size_t ring_b = sizeof(float) * (size_t)channels * st.cap;
    const size_t q_b = sizeof(float) * (size_t)channels * s->S * H * st.queue_slots;
    // zeroed on the copy stream, so that the stream's pushes land after it
    if (e == cudaSuccess) e = cwtk::dmalloc(&st.d_ring, ring_b);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.d_ring, 0, ring_b, s->cst);
    if (e == cudaSuccess) e = cwtk::hmalloc(&st.h_queue, q_b);
    const size_t items = s->bound_items + (size_t)channels * kMaxPending;
    const size_t outf = s->bound_out + (size_t)channels * s->S * H * kMaxPending;
    if (e == cudaSuccess) e = grow_slots(s, items, outf);
    if (e != cudaSuccess) {
        cudaFree(st.d_ring);
        if (st.h_queue) cudaFreeHost(st.h_queue);
        std::lock_guard<std::mutex> lk(s->mu);
        s->streams[id] = Stream();
        s->dev_bytes -= need;
        return cuda_fail(s, e);
    }
    s->bound_items = items;
    s->bound_out = outf;
    std::lock_guard<std::mutex> lk(s->mu);
    for (int i = st.queue_slots - 1; i >= 0; --i) st.free_slots.push_back(i);
    st.dev_bytes = need;
    st.open = true;
    s->streams[id] = std::move(st);
    s->admitted++;
    *stream_id = id;
    return CWT_OK;
}

cwt_status cwt_stream_push(cwt_server s, int id, const float *samples, int k) {
    if (!s || id < 0 || id >= (int)s->streams.size() || k < 0 || (k > 0 && !samples)) return CWT_EINVAL;
    Stream &st = s->streams[id];
    if (!st.open) return CWT_EINVAL;
    if (k == 0) return CWT_OK;
    // One thread feeds a stream; the completion callback only moves hops from
    // `inflight` to `done`, so the lock is held just to read those counts.
    const long long end = st.pushed + k;
    long long new_hops = 0;
    for (long long e = st.next_e; e <= end; e += st.H) ++new_hops;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const long long pending = (long long)st.waiting.size() + st.inflight.size() + st.done.size();
        if (pending + new_hops > kMaxPending || k > st.cap - kSW) return CWT_EBUSY;
    }
    Guard g(s->device);
    if (!g.ok) return CWT_ECUDA;
    // copy [C][k] into the ring at (pushed mod cap), in at most two pieces
    const int pos = (int)(st.pushed % st.cap);
    const int first = std::min(k, st.cap - pos);
    cudaError_t e = cudaMemcpy2DAsync(st.d_ring + pos, sizeof(float) * st.cap, samples,
                                      sizeof(float) * k, sizeof(float) * first, st.C,
                                      cudaMemcpyDefault, s->cst);
    if (e == cudaSuccess && first < k)
        e = cudaMemcpy2DAsync(st.d_ring, sizeof(float) * st.cap, samples + first, sizeof(float) * k,
                              sizeof(float) * (k - first), st.C, cudaMemcpyDefault, s->cst);
    if (e != cudaSuccess) return cuda_fail(s, e);
    std::lock_guard<std::mutex> lk(s->mu);
    st.pushed = end;
    const double t = now_s();
    while (st.next_e <= st.pushed) {
        Hop h;
        h.e = st.next_e;
        h.t_ready = t;
        st.waiting.push_back(h);
        st.next_e += st.H;
        if (s->first_ready < 0) s->first_ready = t;
    }
    return CWT_OK;
}

cwt_status cwt_server_step(cwt_server s, int *hops_launched) {
    if (!s) return CWT_EINVAL;
    Guard g(s->device);
    if (!g.ok) return CWT_ECUDA;
    Slot &sl = s->slots[s->next_slot];
    // wait for the slot's previous batch: its event is recorded after the
    // completion callback, so once it has fired the callback has run
    if (sl.busy) {
        cudaError_t e = cudaEventSynchronize(sl.done);
        if (e != cudaSuccess) return cuda_fail(s, e);
    }
    std::vector<StreamItem> items;
    std::vector<std::pair<int, long long>> hops;
    std::vector<std::pair<size_t, size_t>> copies;  // (out offset floats, count) per hop
    std::vector<float *> dsts;
    size_t out_floats = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (sl.busy) return CWT_EAGAIN;
        for (auto &st : s->streams) {
            if (!st.open) continue;
            while (!st.waiting.empty()) {
                Hop h = st.waiting.front();
                if (st.free_slots.empty()) break;
                st.waiting.pop_front();
                h.slot_out = st.free_slots.back();
                st.free_slots.pop_back();
                const size_t blk = (size_t)st.C * s->S * st.H;
                for (int c = 0; c < st.C; ++c) {
                    StreamItem it;
                    it.ring = st.d_ring + (size_t)c * st.cap;
                    it.out = nullptr;  // filled once the buffer exists
                    it.bank = s->banks[st.bank].bank;
                    it.band = s->banks[st.bank].band;
                    it.start = h.e - kSW;
                    it.cap = st.cap;
                    it.H = st.H;
                    it.D = st.D;
                    items.push_back(it);
                    (void)c;
                }
                copies.push_back({out_floats, blk});
                dsts.push_back(st.h_queue + (size_t)h.slot_out * blk);
                out_floats += blk;
                hops.push_back({st.id, h.e});
                st.inflight.push_back(h);
            }
        }
    }
    if (hops_launched) *hops_launched = (int)hops.size();
    if (items.empty()) return CWT_OK;
    // the slot buffers were sized at admission for kMaxPending hops of every
    // open stream, which bounds any batch: nothing is allocated here
    if (items.size() > sl.items_cap || out_floats > sl.out_cap) {
        s->last_error = "batch exceeds the buffers sized at admission";
        return CWT_ECUDA;
    }
    // the batch reads samples pushed on the copy stream
    cudaError_t e = cudaEventRecord(s->pushed, s->cst);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->st, s->pushed, 0);
    if (e != cudaSuccess) return cuda_fail(s, e);
    // per-channel output blocks: hop block base + c * S * H
    {
        size_t i = 0;
        for (size_t h = 0; h < copies.size(); ++h) {
            const Stream &st = s->streams[hops[h].first];
            for (int c = 0; c < st.C; ++c, ++i)
                items[i].out = sl.d_out + copies[h].first + (size_t)c * s->S * st.H;
        }
    }
    std::memcpy(sl.h_items, items.data(), sizeof(StreamItem) * items.size());
    e = cudaMemcpyAsync(sl.d_items, sl.h_items, sizeof(StreamItem) * items.size(),
                        cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) {
        stream_kernel<<<(unsigned)items.size(), kSThreads, kStreamSmem, s->st>>>(sl.d_items, s->tw, s->S);
        e = cudaGetLastError();
    }
    for (size_t h = 0; h < copies.size() && e == cudaSuccess; ++h)
        e = cudaMemcpyAsync(dsts[h], sl.d_out + copies[h].first, sizeof(float) * copies[h].second,
                            cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        sl.hops = hops;
        sl.busy = true;
    }
    if (e == cudaSuccess) e = cudaLaunchHostFunc(s->st, on_batch_done, new DoneCtx{s, s->next_slot});
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, s->st);
    if (e != cudaSuccess) return cuda_fail(s, e);
    s->launches++;
    s->next_slot = (s->next_slot + 1) % kSlots;
    return CWT_OK;
}

cwt_status cwt_server_sync(cwt_server s) {
    if (!s) return CWT_EINVAL;
    Guard g(s->device);
    if (!g.ok) return CWT_ECUDA;
    cudaError_t e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_fail(s, e);
#ifdef CWT_BOUNDS_CHECK
    std::string where;
    if (check_collect(&where)) {
        s->last_error = where;
        return CWT_EDEVICE;
    }
#endif
    return CWT_OK;
}

cwt_status cwt_stream_pull(cwt_server s, int id, float *out, int max_hops, int *n_hops,
                           long long *first_sample) {
    if (!s || id < 0 || id >= (int)s->streams.size() || max_hops < 0 || !n_hops ||
        (max_hops > 0 && !out))
        return CWT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    Stream &st = s->streams[id];
    if (!st.open && st.done.empty()) return CWT_EINVAL;
    if (st.done.empty()) {
        *n_hops = 0;
        return CWT_EAGAIN;
    }
    const size_t blk = (size_t)st.C * s->S * st.H;
    int n = 0;
    if (first_sample) *first_sample = st.done.front().e - st.D - st.H;
    while (n < max_hops && !st.done.empty()) {
        Hop h = st.done.front();
        st.done.pop_front();
        std::memcpy(out + (size_t)n * blk, st.h_queue + (size_t)h.slot_out * blk, sizeof(float) * blk);
        st.free_slots.push_back(h.slot_out);
        ++n;
    }
    *n_hops = n;
    return CWT_OK;
}

cwt_status cwt_stream_close(cwt_server s, int id) {
    if (!s || id < 0 || id >= (int)s->streams.size()) return CWT_EINVAL;
    Guard g(s->device);
    if (!g.ok) return CWT_ECUDA;
    if (!s->streams[id].open) return CWT_EINVAL;
    // let its pushes and launched hops finish (they write its ring and host
    // queue), then free it
    cudaError_t e = cudaStreamSynchronize(s->cst);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_fail(s, e);
    float *ring = nullptr, *queue = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Stream &st = s->streams[id];
        ring = st.d_ring;
        queue = st.h_queue;
        s->dev_bytes -= st.dev_bytes;
        s->bound_items -= (size_t)st.C * kMaxPending;
        s->bound_out -= (size_t)st.C * s->S * st.H * kMaxPending;
        st = Stream();
    }
    cudaFree(ring);
    if (queue) cudaFreeHost(queue);
    return CWT_OK;
}

cwt_status cwt_server_stats(cwt_server s, cwt_server_stats_t *out) {
    if (!s || !out) return CWT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    int open = 0;
    for (auto &st : s->streams) open += st.open;
    out->open_streams = open;
    out->admitted = s->admitted;
    out->refused = s->refused;
    out->hops = s->hops_done;
    out->launches = s->launches;
    out->coefficients = s->coeffs_done;
    out->device_bytes = s->dev_bytes;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = std::min(v.size() - 1, (size_t)std::ceil(p * v.size()) - (p > 0 ? 1 : 0));
            return v[i];
        };
        out->latency_p50_s = pct(0.50);
        out->latency_p99_s = pct(0.99);
        out->latency_max_s = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->latency_mean_s = sum / v.size();
    }
    if (s->first_ready >= 0 && s->last_done > s->first_ready)
        out->span_s = s->last_done - s->first_ready;
    return CWT_OK;
}

cwt_status cwt_server_reset_stats(cwt_server s) {
    if (!s) return CWT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->latencies.clear();
    s->hops_done = s->launches = s->coeffs_done = 0;
    s->admitted = s->refused = 0;
    s->first_ready = s->last_done = -1;
    return CWT_OK;
}

}  // extern "C"
