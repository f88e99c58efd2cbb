// smooth_cluster_fixed_2.cu -- the cluster kernels of smooth_cluster.cuh on
// the compiled-in local schedule 10000 = 16 x 25 x 25 (entry 2 of
// CWT_CL_MR_FIXED), for the cluster sizes of its mask; a translation unit of
// its own so that the entries compile in parallel.
#include "smooth_cluster.cuh"

namespace cwtk {

CWT_CL_MR_FIXED_2(CWT_CL_FIXED_DEFINE)

}  // namespace cwtk
