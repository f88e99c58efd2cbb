// smooth_fixed.cu -- fixed-length scale-block and forward kernels (smooth_kernel.cuh,
// CWT_MR_FIXED): the row lengths whose whole schedule is compiled in (list A
// here, list B in smooth_fixed_b.cu), the dispatch over both lists, and the
// host check that the scheduler's schedule for N is exactly that one.
#include "smooth_fixed.cuh"

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

}  // namespace

CWT_MR_FIXED_A(CWT_MR_FIXED_DEFINE)

cudaError_t mr_fixed_fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    switch (p->sch.fixed) {
#define CWT_MR_CASE(I, ...) \
    case I: return mr_fixed_fwd<I>(p, signal, st);
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
#define CWT_MR_CASE(I, ...) \
    case I: return mr_fixed_sb<I>(p, a, st);
        CWT_MR_FIXED(CWT_MR_CASE)
#undef CWT_MR_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwtk
