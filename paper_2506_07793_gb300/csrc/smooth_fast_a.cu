// smooth_fast_a.cu -- inlined mixed-radix forward and scale-block kernels for the radix
// pairs (16, 25), (20, 25) (smooth_kernel.cuh).
#include "smooth_kernel.cuh"

namespace cwtk {

template cudaError_t mr_sb_launch<16, 25>(const cwt_plan_s *, const MrArgs &, cudaStream_t);
template cudaError_t mr_sb_launch<20, 25>(const cwt_plan_s *, const MrArgs &, cudaStream_t);
template cudaError_t mr_fwd_launch<16, 25>(const cwt_plan_s *, const void *, cudaStream_t);
template cudaError_t mr_fwd_launch<20, 25>(const cwt_plan_s *, const void *, cudaStream_t);

}  // namespace cwtk
