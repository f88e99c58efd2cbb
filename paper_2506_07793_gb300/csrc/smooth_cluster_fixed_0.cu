// smooth_cluster_fixed_0.cu -- the cluster kernels of smooth_cluster.cuh on
// the compiled-in local schedule 15360 = 16 x 30 x 32 (entry 0 of
// CWT_CL_MR_FIXED), for the cluster sizes of its mask; a translation unit of
// its own so that the entries compile in parallel.
#include "smooth_cluster.cuh"

namespace cwtk {

CWT_CL_MR_FIXED_0(CWT_CL_FIXED_DEFINE)

}  // namespace cwtk
