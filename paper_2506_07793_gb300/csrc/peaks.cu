// peaks.cu -- measured compute peaks of this GPU, the denominators of the
// FP32-side and tensor-side roofline fractions that the benchmark reports.
//
//  * FP32: every thread runs 8 independent chains of fma.rn.f32 (so issue,
//    not latency, bounds it) on a grid of 8 CTAs of 256 threads per SM;
//    flops = 2 per FMA.
//  * Tensor (legacy path): every warp runs 4 independent accumulators of
//    mma.sync.m16n8k16 with FP16 or BF16 operands and FP32 accumulation, the
//    instruction the tensor-core inverse FFTs issue; flops = 2 * 16 * 8 * 16
//    per MMA.
// Both time one launch with CUDA events after one warm-up launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cwt.h"

namespace {

__global__ void __launch_bounds__(256) fma_peak_kernel(float *out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live
}

template <bool BF16>
__global__ void __launch_bounds__(256) mma_peak_kernel(float *out, int iters) {
    uint32_t a0 = 0x3c003c00u ^ threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    uint32_t b0 = 0x3c003c00u ^ (threadIdx.x * 7), b1 = b0 + 5;
    float d[4][4] = {};
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (BF16)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
                        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(d[j][0]), "+f"(d[j][1]), "+f"(d[j][2]), "+f"(d[j][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                else
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
                        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(d[j][0]), "+f"(d[j][1]), "+f"(d[j][2]), "+f"(d[j][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += d[j][0] + d[j][1] + d[j][2] + d[j][3];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" cwt_status cwt_measure_peak(int what, double *tflops) {
    if (!tflops || what < 0 || what > 2) return CWT_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CWT_ECUDA;
    const int grid = sms * 8;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(float) * grid);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int iters = 20000;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // rep 0 warms up
        e = cudaEventRecord(e0, 0);
        if (what == 0)
            fma_peak_kernel<<<grid, 256>>>(out, iters, 0.999f, 0.001f);
        else if (what == 1)
            mma_peak_kernel<false><<<grid, 256>>>(out, iters);
        else
            mma_peak_kernel<true><<<grid, 256>>>(out, iters);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CWT_ENOMEM : CWT_ECUDA;
    const double threads = (double)grid * 256.0;
    double flops;
    if (what == 0)
        flops = threads * iters * 16.0 * 8.0 * 2.0;
    else
        flops = (threads / 32.0) * iters * 16.0 * (2.0 * 16 * 8 * 16);
    *tflops = flops / (ms * 1e-3) / 1e12;
    return CWT_OK;
}
