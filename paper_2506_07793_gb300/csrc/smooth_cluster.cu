// smooth_cluster.cu -- the runtime-schedule cluster kernels for smooth
// lengths one CTA does not run (smooth_cluster.cuh) on 2 ... 4 CTAs, the
// dispatch over every cluster kernel, and the host's choice of the cluster
// split N = CL NL.
#include "smooth_cluster.cuh"

namespace cwtk {

cudaError_t launch_forward_mr_cluster(const cwt_plan_s *p, const void *signal, cudaStream_t st) {
    if (p->jit) return jit_fwd_launch(p, signal, st);
    if (p->sch.fixed_cl >= 0) return cl_mr_fixed_fwd(p, signal, st);
    switch (p->cl) {
#define CWT_CL_CASE(CL) \
    case CL: return cl_mr::fwd_launch<CL, void>(p, signal, st);
        CWT_CL_SIZES_NARROW(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cl_mr_wide_fwd(p, signal, st);
    }
}

cudaError_t launch_scale_block_mr_cluster(const cwt_plan_s *p, void *out_c, void *out_p, void *out_ph,
                                          cudaStream_t st) {
    ClMrArgs a;
    a.spec = p->spec;
    a.bank = p->bank;
    a.band = p->band;
    a.twL = p->twL;
    a.twN = p->twN;
    a.out_c = out_c;
    a.out_p = out_p;
    a.out_ph = out_ph;
    a.S = p->S;
    a.n_out = p->n_out;
    a.sub = p->d;
    a.f64 = p->io == CWT_DTYPE_F64;
    if (p->jit) return jit_cl_sb_launch(p, a, st);
    if (p->sch.fixed_cl >= 0) return cl_mr_fixed_sb(p, a, st);
    switch (p->cl) {
#define CWT_CL_CASE(CL) \
    case CL: return cl_mr::sb_launch<CL, void>(p, a, st);
        CWT_CL_SIZES_NARROW(CWT_CL_CASE)
#undef CWT_CL_CASE
        default: return cl_mr_wide_sb(p, a, st);
    }
}

// The cluster split of a smooth length N that one CTA does not run: the
// smallest CL in 2 ... 8 with N = CL NL and NL <= 16384 a length the
// scheduler covers (false when there is none, e.g. 5^7).  sch receives NL's
// schedule.
bool mr_cluster_split(int N, int *cl, MrSchedule *sch) {
    for (int c = 2; c <= 8; ++c) {
        if (N % c || N / c > kMaxFft) continue;
        if (mr_schedule(N / c, sch)) {
            sch->fixed_cl = cl_mr_fixed_index(*sch);
            *cl = c;
            return true;
        }
    }
    return false;
}

}  // namespace cwtk
