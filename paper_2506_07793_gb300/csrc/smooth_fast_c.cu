// smooth_fast_c.cu -- inlined mixed-radix forward and scale-block kernels for the radix
// pairs (8, 25), (10, 32) (smooth_kernel.cuh).
#include "smooth_kernel.cuh"

namespace cwtk {

template cudaError_t mr_sb_launch<8, 25>(const cwt_plan_s *, const MrArgs &, cudaStream_t);
template cudaError_t mr_sb_launch<10, 32>(const cwt_plan_s *, const MrArgs &, cudaStream_t);
template cudaError_t mr_fwd_launch<8, 25>(const cwt_plan_s *, const void *, cudaStream_t);
template cudaError_t mr_fwd_launch<10, 32>(const cwt_plan_s *, const void *, cudaStream_t);

}  // namespace cwtk
