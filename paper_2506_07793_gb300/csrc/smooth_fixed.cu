// smooth_fixed.cu -- fixed-length scale-block kernels (smooth_kernel.cuh,
// CWT_MR_FIXED): the row lengths whose whole schedule is compiled in, and the
// host check that the scheduler's schedule for N is exactly that one.
#include "smooth_kernel.cuh"

namespace cwtk {

namespace {

template <class FX>
bool same_schedule(const MrSchedule &s) {
    if (s.N != FX::N || s.T != FX::T || s.np != FX::NP || s.mag0 != FX::mag0) return false;
    for (int q = 0; q < FX::NP; ++q) {
        const MrPass f = FX::pass(q);
        const MrPass &h = s.p[q];
        if (h.R != f.R || h.G != f.G || h.Ns != f.Ns || h.mag != f.mag || h.tws != f.tws) return false;
    }
    return true;
}

template <class FX>
cudaError_t fixed_launch(const MrArgs &a, cudaStream_t st) {
    static_assert(FX::N <= kMaxFft, "one shared-memory row");
    static std::atomic<unsigned> done{0};
    constexpr int smem = FX::ROWS * (FX::N + (FX::N >> 4)) * 8;
    static_assert(smem <= kMrMaxSmem, "shared memory of one CTA");
    cudaError_t e = ensure_smem_attr(mr_fixed_scale_block_kernel<FX>, smem, &done);
    if (e != cudaSuccess) return e;
    const int grid = (a.total_rows + FX::ROWS - 1) / FX::ROWS;
    mr_fixed_scale_block_kernel<FX><<<grid, FX::THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <class FX>
cudaError_t fixed_fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    constexpr int smem = FX::ROWS * (FX::N + (FX::N >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(mr_fixed_forward_kernel<FX>, smem, &done);
    if (e != cudaSuccess) return e;
    const int grid = (p->C + FX::ROWS - 1) / FX::ROWS;
    mr_fixed_forward_kernel<FX><<<grid, FX::THREADS, smem, st>>>(signal, p->io == CWT_DTYPE_F64, p->n,
                                                                 p->spec, p->twN, p->C);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mr_fixed_fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    switch (p->sch.fixed) {
#define CWT_MR_CASE(I, N, T, ROWS, MINB, ...) \
    case I: return fixed_fwd_launch<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(p, signal, st);
        CWT_MR_FIXED(CWT_MR_CASE)
#undef CWT_MR_CASE
        default: return cudaErrorInvalidValue;
    }
}

int mr_fixed_index(const MrSchedule &s) {
#define CWT_MR_CASE(I, N, T, ROWS, MINB, ...) \
    if (same_schedule<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(s)) return I;
    CWT_MR_FIXED(CWT_MR_CASE)
#undef CWT_MR_CASE
    return -1;
}

cudaError_t mr_fixed_sb_launch(const cwt_plan_s *p, const MrArgs &a, cudaStream_t st) {
    switch (p->sch.fixed) {
#define CWT_MR_CASE(I, N, T, ROWS, MINB, ...) \
    case I: return fixed_launch<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(a, st);
        CWT_MR_FIXED(CWT_MR_CASE)
#undef CWT_MR_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwtk
