// smooth_fixed_b.cu -- the fixed-length kernels of list B (CWT_MR_FIXED_B in
// smooth_kernel.cuh); a translation unit of its own so that the two lists
// compile in parallel.
#include "smooth_fixed.cuh"

namespace cwtk {

CWT_MR_FIXED_B(CWT_MR_FIXED_DEFINE)

}  // namespace cwtk
