// smooth_cluster_fixed.cu -- the dispatch to the cluster kernels of
// smooth_cluster.cuh for the local lengths whose schedule is compiled in
// (CWT_CL_MR_FIXED; the kernels themselves are in smooth_cluster_fixed_<I>.cu),
// and the host check that the scheduler's schedule for NL is exactly that one.
#include "smooth_cluster.cuh"

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

int cl_mr_fixed_index(const MrSchedule &s, int cl) {
    if (cl < 2 || cl > kMaxClusterCtas) return -1;
#define CWT_CL_CASE(I, MASK, N, T, ROWS, MINB, ...) \
    if ((((MASK) >> cl) & 1u) && same_schedule<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(s)) return I;
    CWT_CL_MR_FIXED(CWT_CL_CASE)
#undef CWT_CL_CASE
    return -1;
}

int cl_mr_fixed_minb(int I) {
#define CWT_CL_CASE(J, MASK, N, T, ROWS, MINB, ...) \
    if (I == J) return MINB;
    CWT_CL_MR_FIXED(CWT_CL_CASE)
#undef CWT_CL_CASE
    return 0;
}

cudaError_t cl_mr_fixed_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st, int rows) {
    switch (p->sch.fixed_cl) {
#define CWT_CL_CASE(I, ...) \
    case I: return cl_fixed_sb<I>(p, a, st, rows);
        CWT_CL_MR_FIXED(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t cl_mr_fixed_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    switch (p->sch.fixed_cl) {
#define CWT_CL_CASE(I, ...) \
    case I: return cl_fixed_fwd<I>(p, signal, st);
        CWT_CL_MR_FIXED(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwtk
