// smooth_fixed.cuh -- the launches of the fixed-length kernels of
// smooth_kernel.cuh, shared by the two translation units that instantiate
// them (smooth_fixed.cu: CWT_MR_FIXED_A; smooth_fixed_b.cu: CWT_MR_FIXED_B).
#pragma once

#include "smooth_kernel.cuh"

namespace cwtk {

namespace fixed_detail {

template <class FX>
cudaError_t sb_launch(const MrArgs &a, cudaStream_t st) {
    static_assert(FX::N <= kMaxFft, "one shared-memory row");
    static std::atomic<unsigned> done{0};
    constexpr int smem = FX::ROWS * (FX::N + (FX::N >> 4)) * 8;
    static_assert(smem <= kMrMaxSmem, "shared memory of one CTA");
    cudaError_t e = ensure_smem_attr(mr_fixed_scale_block_kernel<FX>, smem, &done);
    if (e != cudaSuccess) return e;
    const int grid = (a.total_rows + FX::ROWS - 1) / FX::ROWS;
    mr_fixed_scale_block_kernel<FX><<<grid, FX::THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <class FX>
cudaError_t fwd_launch(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    static std::atomic<unsigned> done{0};
    constexpr int smem = FX::ROWS * (FX::N + (FX::N >> 4)) * 8;
    cudaError_t e = ensure_smem_attr(mr_fixed_forward_kernel<FX>, smem, &done);
    if (e != cudaSuccess) return e;
    const int grid = (p->C + FX::ROWS - 1) / FX::ROWS;
    mr_fixed_forward_kernel<FX><<<grid, FX::THREADS, smem, st>>>(signal, p->io == CWT_DTYPE_F64, p->n,
                                                                 p->spec, p->twN, p->C);
    return cudaGetLastError();
}

}  // namespace fixed_detail

// The definitions of mr_fixed_sb<I> / mr_fixed_fwd<I> for one list entry.
#define CWT_MR_FIXED_DEFINE(I, N, T, ROWS, MINB, ...)                                              \
    template <>                                                                                    \
    cudaError_t mr_fixed_sb<I>(const cwt_plan_s *, const MrArgs &a, cudaStream_t st) {             \
        return fixed_detail::sb_launch<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(a, st);             \
    }                                                                                              \
    template <>                                                                                    \
    cudaError_t mr_fixed_fwd<I>(const cwt_plan_s *p, const void *signal, cudaStream_t st) {        \
        return fixed_detail::fwd_launch<MrFixed<N, T, ROWS, MINB, __VA_ARGS__>>(p, signal, st);    \
    }

}  // namespace cwtk
