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

// Two CTAs of an NL-point local row share an SM when its padded staging
// (NL + NL / 16 float2) and the 1 KB each CTA reserves fit half of the 227 KB.
static bool two_per_sm(int NL) { return (227 * 1024) / ((NL + (NL >> 4)) * 8 + 1024) >= 2; }

// The cluster split of a smooth length N that one CTA does not run: N = CL NL
// with NL <= 16384 a length the scheduler covers (false when there is none,
// e.g. 5^7).  Preferred are local rows two CTAs per SM hold on kernels
// compiled for that (a compiled-in entry with two CTAs per SM, or -- jit --
// any schedule compiled at plan creation): fewest passes, then the smallest
// CL.  Measured on 8 channels x 100 scales: 30000 on 3 x 10000 0.162 ms
// against 0.225 on 2 x 15000, 60000 on 5 x 12000 0.323 against 0.454 on
// 4 x 15000, 120000 on 10 x 12000 0.760 against 1.119 on 8 x 15000, 100000 on
// 10 x 10000 (three passes) 0.586 against 0.723 on 8 x 12500 (four).  Else
// the smallest CL up to 8.  Cluster sizes above 8 need such kernels.  sch
// receives NL's schedule, fixed_cl its compiled-in entry for CL (or -1).
bool mr_cluster_split(int N, int *cl, MrSchedule *sch, bool jit) {
    int first = 0, best = 0;
    MrSchedule s_first, s_best;
    for (int c = 2; c <= kMaxClusterCtas; ++c) {
        if (N % c || N / c > kMaxFft) continue;
        MrSchedule s;
        if (!mr_schedule(N / c, &s)) continue;
        s.fixed_cl = cl_mr_fixed_index(s, c);
        if (c > 8 && !jit && s.fixed_cl < 0) continue;  // no kernel for this cluster size
        if (!first && c <= 8) {
            first = c;
            s_first = s;
        }
        const bool fast = two_per_sm(N / c) && (jit || (s.fixed_cl >= 0 && cl_mr_fixed_minb(s.fixed_cl) >= 2));
        if (fast && (!best || s.np < s_best.np)) {
            best = c;
            s_best = s;
        }
    }
    if (best) {
        *cl = best;
        *sch = s_best;
        return true;
    }
    if (first) {
        *cl = first;
        *sch = s_first;
        return true;
    }
    return false;
}

}  // namespace cwtk
