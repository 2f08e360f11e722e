// Degridder dispatch and the variants for L != 32 (kernels in degridder_impl.cuh).
#include "degridder_impl.cuh"

namespace idg {
namespace {

using namespace dev;

// runtime-PG form (one launch for any K_p) and the static-PG forms
#define DV_RT(L, NV, NT) {"nv" #NV "_nt" #NT "_pg_runtime", degrid_launch_kernel<L, NV, 0, NT, 1>}
#define DV_ST(L, NV, NT, MINB) {"nv" #NV "_nt" #NT "_minb" #MINB "_pg_static", degrid_launch_static<L, NV, NT, MINB>}

#define DV_F2(L, NV, NT, MINB) {"f32x2_nv" #NV "_nt" #NT "_minb" #MINB "_pg_static", degrid_f2_launch_static<L, NV, NT, MINB>}
const DegridVariant kD8[] = {DV_F2(8, 4, 128, 4), DV_RT(8, 4, 256), DV_ST(8, 4, 256, 3), DV_ST(8, 4, 128, 5)};
const DegridVariant kD16[] = {DV_F2(16, 4, 128, 3), DV_RT(16, 4, 256), DV_ST(16, 4, 256, 3), DV_ST(16, 4, 128, 5)};
const DegridVariant kD24[] = {DV_F2(24, 4, 128, 3), DV_RT(24, 4, 256), DV_ST(24, 4, 256, 3), DV_ST(24, 4, 128, 5)};
const DegridVariant kD48[] = {DV_F2(48, 4, 128, 2), DV_RT(48, 4, 256), DV_ST(48, 4, 256, 2), DV_ST(48, 4, 128, 4)};
// L = 64: the packed form would need 64^2 x 68 B of shared memory (> 227 KB)
const DegridVariant kD64[] = {DV_RT(64, 4, 256), DV_ST(64, 4, 256, 1), DV_ST(64, 4, 128, 2)};
#undef DV_F2

#undef DV_RT
#undef DV_ST

}  // namespace

bool degridder_table(int L, const DegridVariant **v, int *n) {
    switch (L) {
#define T(X) case X: *v = kD##X; *n = (int)(sizeof(kD##X) / sizeof(DegridVariant)); return true;
        T(8) T(16) T(24) T(48) T(64)
#undef T
    case 32: return degridder_table_l32(v, n);
    }
    return false;
}

int degridder_variant_count(int L) {
    const DegridVariant *v;
    int n;
    return degridder_table(L, &v, &n) ? n : 0;
}

const char *degridder_variant_name(int L, int i) {
    const DegridVariant *v;
    int n;
    if (!degridder_table(L, &v, &n) || i < 0 || i >= n) return nullptr;
    return v[i].name;
}

idg_status launch_degridder(const Geometry &g, const SubgridSet &set, int variant, const void *sub,
                            const uint8_t *flags, const void *aterms, const float *taper, void *vis_out,
                            void *stream) {
    const DegridVariant *v;
    int n;
    if (!degridder_table(g.L, &v, &n)) return fail(IDG_ERR_UNSUPPORTED, "subgrid size not compiled in");
    if (set.count <= 0) return IDG_OK;
    if (g.recurrence) return launch_degridder_rec(g, set, sub, flags, aterms, taper, vis_out, stream);
    if (variant < 0) variant = get_variant(IDG_KERNEL_DEGRIDDER, g.L);
    if (variant >= n) variant = 0;
    return v[variant].fn(g, set, sub, flags, aterms, taper, vis_out, (cudaStream_t)stream);
}

}  // namespace idg
