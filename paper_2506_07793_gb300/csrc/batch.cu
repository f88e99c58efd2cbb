// batch.cu -- many epochs of uneven length in one persistent launch.
//
// The paper loops over recordings in Python (Sections "Comparison between
// devices and software" and "Wavelength and flexibility"); here a batch of
// epochs, each with its own length n_e and hence its own padded length
// N_e = next power of two >= max(n_e, 32) (Section "Fast Fourier transform"),
// is one persistent kernel replayed from a CUDA graph.
//
// Work item = (epoch, group of G channels) with G * N_e = one tile of kTile
// points (G capped by the channel count).  Per item the CTA
//   1. runs the forward FFT of the G channels (Eq. 2, one FFT per channel)
//      and keeps the spectra in shared memory -- they never reach HBM;
//   2. for every (channel, scale) row: band product with the FP64-generated
//      bank of length N_e (Eq. 3), spectral fold by the power-of-two factor f
//      of the decimation, inverse FFT of N_e / f points, crop / decimate /
//      reduce and coalesced stores (Section "Precision").
// CTAs pull items from an atomic counter, largest FFTs first by default.  An
// autotuner times the candidate schedules (inverse radix 16 or 32, item
// order) on the first batch of a given shape and keeps the fastest; every
// candidate computes the same values.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "batch_kernel.cuh"

namespace cwtk {

const void *batch_kernel_ptr_16();
const void *batch_kernel_ptr_32();
const void *batch_kernel_ptr(int ri) { return ri == 16 ? batch_kernel_ptr_16() : batch_kernel_ptr_32(); }

// ---- host side -------------------------------------------------------------

struct BatchState {
    float *bank[kMaxBatchLog2 + 1] = {};
    int *band[kMaxBatchLog2 + 1] = {};
    BatchItem *d_items = nullptr;
    size_t items_cap = 0;
    int *d_counter = nullptr;
    std::vector<BatchItem> h_items_natural, h_items_sorted;
    std::vector<BatchItem> uploaded;
    // CUDA graph: memset(counter) -> batch_kernel
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
    int graph_ri = 0;
    BatchArgs graph_args{};
    // autotuner
    bool tuned = false;
    int ri = 16, order = 0;
    double tune_ms[4] = {0, 0, 0, 0};
    long long launches = 0;
    int grid = 0;
    size_t bytes = 0;
};

void free_batch_state(BatchState *b) {
    if (!b) return;
    for (int i = 0; i <= kMaxBatchLog2; ++i) {
        cudaFree(b->bank[i]);
        cudaFree(b->band[i]);
    }
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

namespace {

template <int RI>
cudaError_t batch_attr() {
    static std::atomic<unsigned> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 32 && (done.load(std::memory_order_acquire) & (1u << dev))) return cudaSuccess;
    e = cudaFuncSetAttribute(batch_kernel_ptr(RI), cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem<RI>());
    if (e == cudaSuccess && dev < 32) done.fetch_or(1u << dev, std::memory_order_acq_rel);
    return e;
}

cudaError_t batch_grid(int ri, int *grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel_ptr(ri), kBThreads,
                                                          ri == 16 ? batch_smem<16>() : batch_smem<32>());
    if (e == cudaSuccess) *grid = sms * std::max(per, 1);
    return e;
}

// (Re)build the graph for radix `ri` with arguments `args`, or update its
// kernel node in place when only the arguments changed.
cudaError_t batch_graph(BatchState *b, int ri, const BatchArgs &args, int grid) {
    cudaKernelNodeParams kp{};
    void *kargs[] = {(void *)&args};
    kp.func = (void *)batch_kernel_ptr(ri);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(kBThreads);
    kp.sharedMemBytes = ri == 16 ? batch_smem<16>() : batch_smem<32>();
    kp.kernelParams = kargs;
    if (b->exec && b->graph_ri == ri) {
        if (std::memcmp(&b->graph_args, &args, sizeof(args)) == 0) return cudaSuccess;
        cudaError_t e = cudaGraphExecKernelNodeSetParams(b->exec, b->knode, &kp);
        if (e == cudaSuccess) b->graph_args = args;
        return e;
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaGraphCreate(&b->graph, 0);
    cudaGraphNode_t mnode;
    cudaMemsetParams mp{};
    mp.dst = b->d_counter;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    mp.value = 0;
    if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&mnode, b->graph, nullptr, 0, &mp);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&b->knode, b->graph, &mnode, 1, &kp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) {
        b->graph_ri = ri;
        b->graph_args = args;
    }
    return e;
}

}  // namespace

cudaError_t batch_execute(cwt_plan_s *p, const cwt_epoch *epochs, int n_epochs, const float *in,
                          float2 *oc, float *op, float *oph, cudaStream_t st, bool prepare_only) {
    if (!p->batch) p->batch = new BatchState();
    BatchState *b = p->batch;
    cudaError_t e = cudaSuccess;
    if (!b->d_counter) {
        e = cwtk::dmalloc(&b->d_counter, sizeof(int));
        if (e != cudaSuccess) return e;
    }
    // banks for every padded length in the batch (generated once per length)
    const int C = p->C, S = p->S;
    std::vector<BatchItem> items;
    for (int ei = 0; ei < n_epochs; ++ei) {
        const cwt_epoch &ep = epochs[ei];
        int N = kMinFft;
        while (N < ep.samples + p->pad_extra) N <<= 1;
        const int L = ilog2c(N);
        if (!b->bank[L]) {
            // a length's bank is published only once it is generated, so a
            // failure here leaves nothing half-built for the next call
            float *bank = nullptr;
            int *band = nullptr;
            e = cwtk::dmalloc(&bank, sizeof(float) * (size_t)S * N);
            if (e == cudaSuccess) e = cwtk::dmalloc(&band, sizeof(int) * 2 * (size_t)S);
            if (e == cudaSuccess) e = launch_bank_n(p, N, bank, band, st, nullptr);
            if (e != cudaSuccess) {
                cudaFree(bank);
                cudaFree(band);
                return e;
            }
            b->bank[L] = bank;
            b->band[L] = band;
            b->bytes += sizeof(float) * (size_t)S * N + sizeof(int) * 2 * (size_t)S;
        }
        const int G = std::max(1, std::min(C, kTile / N));
        const int n_out = (ep.samples + p->d - 1) / p->d;
        for (int c0 = 0; c0 < C; c0 += G) {
            BatchItem it{};
            it.in_off = ep.in_offset + (long long)c0 * ep.samples;
            it.out_off = ep.out_offset + (long long)c0 * S * n_out;
            it.n = ep.samples;
            it.log2n = L;
            it.G = std::min(G, C - c0);
            items.push_back(it);
        }
    }
    if (items.empty()) return cudaSuccess;
    // RI = 16 stages kBThreads * 16 points of inverse rows: only for batches
    // whose every inverse length fits (an 8192-point row at odd d needs RI = 32)
    int max_m = 0;
    for (const BatchItem &it : items) max_m = std::max(max_m, batch_inverse_length(1 << it.log2n, p->d));
    const bool ri16_ok = max_m <= kBThreads * 16;
    // two orders: input order, and largest FFT first (stable)
    std::vector<BatchItem> sorted = items;
    std::stable_sort(sorted.begin(), sorted.end(),
                     [](const BatchItem &x, const BatchItem &y) { return x.log2n > y.log2n; });
    const bool shape_changed =
        items.size() != b->h_items_natural.size() ||
        std::memcmp(items.data(), b->h_items_natural.data(), items.size() * sizeof(BatchItem)) != 0;
    if (shape_changed) {
        if (items.size() > b->items_cap) {
            BatchItem *d = nullptr;
            e = cwtk::dmalloc(&d, sizeof(BatchItem) * items.size());
            if (e != cudaSuccess) return e;  // the previous shape stays intact
            cudaFree(b->d_items);
            b->d_items = d;
            b->items_cap = items.size();
            b->uploaded.clear();
        }
        b->h_items_natural = items;
        b->h_items_sorted = sorted;
        b->tuned = false;
    }
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));  // padding too: the graph compares argument bytes
    a.in = in;
    a.oc = oc;
    a.op = op;
    a.oph = oph;
    a.items = b->d_items;
    a.n_items = (int)items.size();
    a.counter = b->d_counter;
    for (int i = 0; i <= kMaxBatchLog2; ++i) {
        a.bank[i] = b->bank[i];
        a.band[i] = b->band[i];
    }
    a.tw = p->tw;
    a.S = S;
    a.d = p->d;
    e = batch_attr<16>();
    if (e == cudaSuccess) e = batch_attr<32>();
    if (e != cudaSuccess) return e;

    auto upload = [&](int order) -> cudaError_t {
        const std::vector<BatchItem> &v = order == 0 ? b->h_items_sorted : b->h_items_natural;
        if (b->uploaded.size() == v.size() &&
            std::memcmp(b->uploaded.data(), v.data(), v.size() * sizeof(BatchItem)) == 0)
            return cudaSuccess;
        cudaError_t r = cudaMemcpyAsync(b->d_items, v.data(), v.size() * sizeof(BatchItem),
                                        cudaMemcpyHostToDevice, st);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);  // host vector may change later
        if (r == cudaSuccess) b->uploaded = v;
        return r;
    };
    auto run = [&](int ri, int order) -> cudaError_t {
        cudaError_t r = upload(order);
        int grid = 0;
        if (r == cudaSuccess) r = batch_grid(ri, &grid);
        if (r == cudaSuccess) r = batch_graph(b, ri, a, grid);
        if (r == cudaSuccess) r = cudaGraphLaunch(b->exec, st);
        if (r == cudaSuccess) {
            b->grid = grid;
            ++b->launches;
        }
        return r;
    };

    if (!b->tuned) {
        // autotune: time each (radix, order) candidate once on this batch
        const int cands[4][2] = {{16, 0}, {32, 0}, {16, 1}, {32, 1}};
        cudaEvent_t t0, t1;
        e = cudaEventCreate(&t0);
        if (e == cudaSuccess) e = cudaEventCreate(&t1);
        double best = 1e300;
        for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
            if (cands[c][0] == 16 && !ri16_ok) {
                b->tune_ms[c] = -1.f;  // not a candidate for this batch
                continue;
            }
            e = run(cands[c][0], cands[c][1]);  // warm (graph build, upload)
            if (e == cudaSuccess) e = cudaEventRecord(t0, st);
            if (e == cudaSuccess) e = run(cands[c][0], cands[c][1]);
            if (e == cudaSuccess) e = cudaEventRecord(t1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            b->tune_ms[c] = ms;
            if (e == cudaSuccess && ms < best) {
                best = ms;
                b->ri = cands[c][0];
                b->order = cands[c][1];
            }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (e != cudaSuccess) return e;
        b->tuned = true;
    }
    if (prepare_only) return cudaSuccess;
    return run(b->ri, b->order);
}

void batch_stats(const cwt_plan_s *p, cwt_batch_stats *s) {
    std::memset(s, 0, sizeof(*s));
    const BatchState *b = p->batch;
    if (!b) return;
    s->items = (int)b->h_items_natural.size();
    s->grid = b->grid;
    s->inverse_radix = b->ri;
    s->order = b->order;
    s->tuned = b->tuned;
    for (int i = 0; i < 4; ++i) s->tune_ms[i] = b->tune_ms[i];
    s->graph_launches = b->launches;
    s->bank_bytes = b->bytes;
}

}  // namespace cwtk
