// smooth_fwd.cu -- forward FFT of each zero-padded channel for 2,3,5,7-smooth
// padded lengths (Section "Fast Fourier transform"; Eq. 2: one forward FFT per
// channel): the generic kernel of smooth_kernel.cuh, and the dispatch to the
// fixed-length kernels (smooth_fixed.cu) and the inlined radix pairs
// (instantiated in smooth_fast_*.cu).  Kept apart from
// smooth.cu (the scale block and the schedule) so that the two compile in
// parallel.
#include <cuda_runtime.h>

#include "smooth_kernel.cuh"

namespace cwtk {

cudaError_t launch_forward_mr(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    if (p->cl > 1) return launch_forward_mr_cluster(p, signal, st);
    if (p->jit) return jit_fwd_launch(p, signal, st);
    if (p->sch.fixed >= 0) return mr_fixed_fwd_launch(p, signal, st);
    switch (p->sch.fast) {
#define CWT_MR_CASE(I, A, B) \
    case I: return mr_fwd_launch<A, B>(p, signal, st);
        CWT_MR_FAST_PAIRS(CWT_MR_CASE)
#undef CWT_MR_CASE
        default: return mr_fwd_launch<0, 0>(p, signal, st);
    }
}

}  // namespace cwtk
