// smooth_cluster_wide.cu -- the runtime-schedule cluster kernels of
// smooth_cluster.cuh on 5 ... 8 CTAs (a translation unit of its own so that
// the kernels compile in parallel with smooth_cluster.cu).
#include "smooth_cluster.cuh"

namespace cwtk {

cudaError_t cl_mr_wide_sb(const cwt_plan_s *p, const ClMrArgs &a, cudaStream_t st) {
    switch (p->cl) {
#define CWT_CL_CASE(CL) \
    case CL: return cl_mr::sb_launch<CL, void>(p, a, st);
        CWT_CL_SIZES_WIDE(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t cl_mr_wide_fwd(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    switch (p->cl) {
#define CWT_CL_CASE(CL) \
    case CL: return cl_mr::fwd_launch<CL, void>(p, signal, st);
        CWT_CL_SIZES_WIDE(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwtk
