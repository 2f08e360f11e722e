// Degridder variants for L = 32 (the LOFAR-like workload), kept in their own
// translation unit so they compile in parallel with the rest.
#include "degridder_impl.cuh"

namespace idg {
namespace {

using namespace dev;

#define DV_RT(L, NV, NT) {"nv" #NV "_nt" #NT "_pg_runtime", degrid_launch_kernel<L, NV, 0, NT, 1>}
#define DV_ST(L, NV, NT, MINB) {"nv" #NV "_nt" #NT "_minb" #MINB "_pg_static", degrid_launch_static<L, NV, NT, MINB>}

#define DV_RTM(L, NV, NT, MINB) {"nv" #NV "_nt" #NT "_minb" #MINB "_pg_runtime", degrid_launch_kernel<L, NV, 0, NT, MINB>}
#define DV_F2(L, NV, NT, MINB) {"f32x2_nv" #NV "_nt" #NT "_minb" #MINB "_pg_static", degrid_f2_launch_static<L, NV, NT, MINB>}

idg_status launch_tcw(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                      const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    return launch_degridder_tcw(g, set, sub, flags, aterms, taper, vis_out, (void *)s);
}

// One kernel family per call: the tensor-core form unless most of the call's
// visibilities sit in subgrids of fewer than KPMIN, where its fixed cost per
// subgrid (the split image operand, filling and draining the pipeline, padding to
// 128 visibilities) outweighs its faster sum; splitting one call across both
// kernels by K_p was measured slower (launch tails).
template <int KPMIN>
idg_status launch_tcw_auto(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                           const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    if (!set.kp_host) return fail(IDG_ERR_INVALID_ARG, "degridder: K_p of the subgrid set is required");
    int64_t small = 0, all = 0;
    for (int64_t i = 0; i < set.count; ++i) {
        all += set.kp_host[i];
        if (set.kp_host[i] < KPMIN) small += set.kp_host[i];
    }
    if (2 * small > all) return degrid_f2_launch_static<32, 4, 128, 3>(g, set, sub, flags, aterms, taper, vis_out, s);
    return launch_tcw(g, set, sub, flags, aterms, taper, vis_out, s);
}

// separable tensor-core form where the plan allows it (by the same K_p rule), else the above
idg_status launch_sep_auto(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                           const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    if (!g.separable) return launch_tcw_auto<512>(g, set, sub, flags, aterms, taper, vis_out, s);
    if (!set.kp_host) return fail(IDG_ERR_INVALID_ARG, "degridder: K_p of the subgrid set is required");
    int64_t small = 0, all = 0;
    for (int64_t i = 0; i < set.count; ++i) {
        all += set.kp_host[i];
        if (set.kp_host[i] < kSepFusedKpMin) small += set.kp_host[i];
    }
    if (2 * small > all) return degrid_f2_launch_static<32, 4, 128, 3>(g, set, sub, flags, aterms, taper, vis_out, s);
    return launch_degridder_sep(g, set, sub, flags, aterms, taper, vis_out, (void *)s);
}

idg_status launch_sep(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                      const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    if (!g.separable) return launch_tcw(g, set, sub, flags, aterms, taper, vis_out, s);
    return launch_degridder_sep(g, set, sub, flags, aterms, taper, vis_out, (void *)s);
}

const DegridVariant kD32[] = {{"tcgen05_separable_auto512", launch_sep_auto},
                              {"tcgen05_separable", launch_sep},
                              {"tcgen05_tmemA_ws_nt288_auto512", launch_tcw_auto<512>},
                              DV_F2(32, 4, 128, 3),      {"tcgen05_tmemA_ws_nt288", launch_tcw},
                              DV_RT(32, 4, 256),         DV_ST(32, 4, 256, 3),
                              DV_ST(32, 4, 128, 5),      DV_ST(32, 4, 128, 6), DV_ST(32, 2, 256, 4),
                              DV_RTM(32, 4, 256, 3),     DV_F2(32, 4, 128, 4), DV_F2(32, 2, 128, 4),
                              DV_F2(32, 4, 256, 2)};
#undef DV_F2
#undef DV_RTM

#undef DV_RT
#undef DV_ST

}  // namespace

bool degridder_table_l32(const DegridVariant **v, int *n) {
    *v = kD32;
    *n = (int)(sizeof(kD32) / sizeof(DegridVariant));
    return true;
}

}  // namespace idg
