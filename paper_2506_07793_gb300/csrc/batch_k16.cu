// batch_k16.cu -- the persistent batch kernel with 16 points per thread in
// the inverse FFTs (batch_kernel.cuh; design in batch.cu).
#define CWT_BATCH_KERNELS
#include "batch_kernel.cuh"

namespace cwtk {

const void *batch_kernel_ptr_16() { return (const void *)batch_kernel<16>; }

}  // namespace cwtk
