// batch_k32.cu -- the persistent batch kernel with 32 points per thread in
// the inverse FFTs (batch_kernel.cuh; design in batch.cu).
#define CWT_BATCH_KERNELS
#include "batch_kernel.cuh"

namespace cwtk {

const void *batch_kernel_ptr_32() { return (const void *)batch_kernel<32>; }

}  // namespace cwtk
