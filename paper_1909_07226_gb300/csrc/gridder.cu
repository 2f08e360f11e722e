// Gridder: subgrid images by direct summation (Algorithm 1, inner loops;
// Eq. ShiftedDirectImaging), followed by the image-domain kernel
// taper * A_p^H . I_p . A_q (Sect. 3.4).
//
// One CTA per subgrid.  Each thread owns NPX consecutive pixels of one row and
// keeps their 4-pol complex accumulators in registers; visibilities are staged
// in shared memory in batches of VB (FP32 phase coefficients and the 2x2
// visibility) and read back as block-wide broadcasts.  Per visibility and pixel
// the inner loop issues 2 FFMA for the phase, sin and cos on the SFU, and 16
// FFMA for the four complex multiply-adds.
//
// With PREFETCH the next batch is fetched from global memory into registers
// while the current one is summed, then converted and stored into the other
// half of a double buffer: one barrier per batch, global latency hidden.
#include <cuda_runtime.h>

#include "gridder_impl.cuh"

namespace idg {
namespace {

using namespace dev;

template <int L, int NPX, int VB, int MINB>
__global__ void __launch_bounds__(L * L / NPX, MINB)
gridder_f2_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                  const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                  const float *__restrict__ taper, float4 *__restrict__ out) {
    constexpr int NT = L * L / NPX;
    constexpr int TPR = L / NPX;
    __shared__ float4 s_coef[VB];
    __shared__ float4 s_v01[VB];
    __shared__ float4 s_v23[VB];
    __shared__ float4 s_iv01[VB];
    __shared__ float4 s_iv23[VB];

    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int tid = threadIdx.x;
    const int y = tid / TPR;
    const int x0 = (tid % TPR) * NPX;
    const float Y = (float)(y - L / 2);
    float X[NPX], NP[NPX];
#pragma unroll
    for (int j = 0; j < NPX; ++j) {
        X[j] = (float)(x0 + j - L / 2);
        NP[j] = g.nprime[y * L + x0 + j];
    }
    f2_t acc[NPX][4];
#pragma unroll
    for (int j = 0; j < NPX; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = f2_pack(0.0f, 0.0f);

    for (int k0 = 0; k0 < d.kp; k0 += VB) {
        const int nb = min(VB, d.kp - k0);
        for (int i = tid; i < nb; i += NT) {
            RawVis r;
            fetch_raw(g, d, k0 + i, vis, flags, r);
            store_raw(g, d, r, s_coef, s_v01, s_v23, i);
            const float4 a = s_v01[i], b = s_v23[i];
            s_iv01[i] = make_float4(-a.y, a.x, -a.w, a.z);
            s_iv23[i] = make_float4(-b.y, b.x, -b.w, b.z);
        }
        __syncthreads();
        sum_batch_f2<NPX>(s_coef, s_v01, s_v23, s_iv01, s_iv23, nb, Y, X, NP, acc);
        __syncthreads();
    }

    float4 *o = out + (size_t)blockIdx.x * L * L * 2;
#pragma unroll
    for (int j = 0; j < NPX; ++j) {
        const int pix = y * L + x0 + j;
        M22 P;
        f2_unpack(acc[j][0], P.m[0].x, P.m[0].y);
        f2_unpack(acc[j][1], P.m[1].x, P.m[1].y);
        f2_unpack(acc[j][2], P.m[2].x, P.m[2].y);
        f2_unpack(acc[j][3], P.m[3].x, P.m[3].y);
        if (aterms) {
            const size_t base = ((size_t)d.slot * g.n_stations) * L * L;
            const M22 Ap = load_m22(aterms + 2 * (base + (size_t)d.st_p * L * L + pix));
            const M22 Aq = load_m22(aterms + 2 * (base + (size_t)d.st_q * L * L + pix));
            P = herm_mul_mul(Ap, P, Aq);
        }
        const float tw = taper[pix];
        o[2 * pix] = make_float4(tw * P.m[0].x, tw * P.m[0].y, tw * P.m[1].x, tw * P.m[1].y);
        o[2 * pix + 1] = make_float4(tw * P.m[2].x, tw * P.m[2].y, tw * P.m[3].x, tw * P.m[3].y);
    }
}

template <int L, int NPX, int VB, int MINB, bool PREFETCH>
__global__ void __launch_bounds__(L * L / NPX, MINB)
gridder_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
               const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
               const float *__restrict__ taper, float4 *__restrict__ out) {
    constexpr int NT = L * L / NPX;
    constexpr int TPR = L / NPX;
    constexpr int NBUF = PREFETCH ? 2 : 1;
    constexpr int NS = (VB + NT - 1) / NT;   // visibilities staged per thread per batch
    static_assert(L % NPX == 0, "pixels per thread must divide L");

    __shared__ float4 s_coef[NBUF][VB];
    __shared__ float4 s_v01[NBUF][VB];
    __shared__ float4 s_v23[NBUF][VB];

    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int tid = threadIdx.x;
    const int y = tid / TPR;
    const int x0 = (tid % TPR) * NPX;
    const float Y = (float)(y - L / 2);

    float X[NPX], NP[NPX];
#pragma unroll
    for (int j = 0; j < NPX; ++j) {
        X[j] = (float)(x0 + j - L / 2);
        NP[j] = g.nprime[y * L + x0 + j];
    }
    float acc[NPX][8];
#pragma unroll
    for (int j = 0; j < NPX; ++j)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[j][q] = 0.0f;

    if (PREFETCH) {
        {   // stage batch 0
            const int nb = min(VB, d.kp);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int i = tid + s * NT;
                if (i < nb) {
                    RawVis r;
                    fetch_raw(g, d, i, vis, flags, r);
                    store_raw(g, d, r, s_coef[0], s_v01[0], s_v23[0], i);
                }
            }
        }
        __syncthreads();
        for (int k0 = 0, b = 0; k0 < d.kp; k0 += VB, ++b) {
            const int cur = b & 1;
            const int nb = min(VB, d.kp - k0);
            const int nbn = min(VB, d.kp - k0 - VB);   // next batch (<= 0: none)
            RawVis raw[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int i = tid + s * NT;
                if (i < nbn) fetch_raw(g, d, k0 + VB + i, vis, flags, raw[s]);
            }
            sum_batch<NPX>(s_coef[cur], s_v01[cur], s_v23[cur], nb, Y, X, NP, acc);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int i = tid + s * NT;
                if (i < nbn) store_raw(g, d, raw[s], s_coef[cur ^ (NBUF - 1)], s_v01[cur ^ (NBUF - 1)],
                                       s_v23[cur ^ (NBUF - 1)], i);
            }
            __syncthreads();
        }
    } else {
        for (int k0 = 0; k0 < d.kp; k0 += VB) {
            const int nb = min(VB, d.kp - k0);
            for (int i = tid; i < nb; i += NT) {
                RawVis r;
                fetch_raw(g, d, k0 + i, vis, flags, r);
                store_raw(g, d, r, s_coef[0], s_v01[0], s_v23[0], i);
            }
            __syncthreads();
            sum_batch<NPX>(s_coef[0], s_v01[0], s_v23[0], nb, Y, X, NP, acc);
            __syncthreads();
        }
    }

    // image-domain kernel: taper * A_p^H . I . A_q, then store [L][L][4]
    float4 *o = out + (size_t)blockIdx.x * L * L * 2;
#pragma unroll
    for (int j = 0; j < NPX; ++j) {
        const int pix = y * L + x0 + j;
        M22 P;
        P.m[0] = make_float2(acc[j][0], acc[j][1]);
        P.m[1] = make_float2(acc[j][2], acc[j][3]);
        P.m[2] = make_float2(acc[j][4], acc[j][5]);
        P.m[3] = make_float2(acc[j][6], acc[j][7]);
        if (aterms) {
            const size_t base = ((size_t)d.slot * g.n_stations) * L * L;
            const M22 Ap = load_m22(aterms + 2 * (base + (size_t)d.st_p * L * L + pix));
            const M22 Aq = load_m22(aterms + 2 * (base + (size_t)d.st_q * L * L + pix));
            P = herm_mul_mul(Ap, P, Aq);
        }
        const float tw = taper[pix];
        o[2 * pix] = make_float4(tw * P.m[0].x, tw * P.m[0].y, tw * P.m[1].x, tw * P.m[1].y);
        o[2 * pix + 1] = make_float4(tw * P.m[2].x, tw * P.m[2].y, tw * P.m[3].x, tw * P.m[3].y);
    }
}

using LaunchFn = idg_status (*)(const Geometry &, const SubgridSet &, const void *, const uint8_t *, const void *,
                                const float *, void *, cudaStream_t);

template <int L, int NPX, int VB, int MINB, bool PF>
idg_status launch_one(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                      const void *aterms, const float *taper, void *out, cudaStream_t s) {
    constexpr int NT = L * L / NPX;
    gridder_kernel<L, NPX, VB, MINB, PF><<<(unsigned)set.count, NT, 0, s>>>(
        g, set.idx, set.first, (const float4 *)vis, flags, (const float4 *)aterms, taper, (float4 *)out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gridder launch");
    return IDG_OK;
}

template <int L, int NPX, int VB, int MINB>
idg_status launch_f2(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                     const void *aterms, const float *taper, void *out, cudaStream_t s) {
    constexpr int NT = L * L / NPX;
    gridder_f2_kernel<L, NPX, VB, MINB><<<(unsigned)set.count, NT, 0, s>>>(
        g, set.idx, set.first, (const float4 *)vis, flags, (const float4 *)aterms, taper, (float4 *)out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gridder launch");
    return IDG_OK;
}

idg_status launch_tcw(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                      const void *aterms, const float *taper, void *out, cudaStream_t s) {
    return launch_gridder_tcw(g, set, vis, flags, aterms, taper, out, (void *)s);
}

// separable tensor-core form where the plan allows it, else the direct one
idg_status launch_sep(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                      const void *aterms, const float *taper, void *out, cudaStream_t s) {
    if (!g.separable) return launch_gridder_tcw(g, set, vis, flags, aterms, taper, out, (void *)s);
    return launch_gridder_sep(g, set, vis, flags, aterms, taper, out, (void *)s);
}

struct Variant {
    const char *name;
    LaunchFn fn;
};

#define GV(L, NPX, VB, MINB, PF) {"npx" #NPX "_vb" #VB "_minb" #MINB "_prefetch_" #PF, launch_one<L, NPX, VB, MINB, PF>}

#define GF(L, NPX, VB, MINB) {"f32x2_npx" #NPX "_vb" #VB "_minb" #MINB, launch_f2<L, NPX, VB, MINB>}
const Variant kV8[] = {GF(8, 1, 128, 4), GV(8, 1, 128, 4, false), GV(8, 2, 256, 8, true)};
const Variant kV16[] = {GF(16, 2, 128, 3), GV(16, 2, 128, 3, false), GV(16, 2, 256, 3, true),
                        GV(16, 4, 256, 6, true), GF(16, 4, 128, 2)};
const Variant kV24[] = {GF(24, 3, 128, 3), GV(24, 3, 128, 3, false), GV(24, 3, 256, 3, true),
                        GV(24, 6, 256, 6, true), GF(24, 6, 128, 2)};
const Variant kV32[] = {{"tcgen05_separable", launch_sep}, {"tcgen05_tmemA_ws_nt288", launch_tcw}, GF(32, 4, 128, 2), GV(32, 4, 128, 3, false),
                        GV(32, 4, 256, 3, true),
                        GV(32, 4, 256, 4, true),  GV(32, 8, 256, 4, true),  GV(32, 2, 256, 2, true),
                        GF(32, 4, 128, 3),        GF(32, 2, 128, 3),        GF(32, 8, 128, 4)};
const Variant kV48[] = {GF(48, 4, 128, 1), GV(48, 6, 128, 2, false), GV(48, 6, 256, 2, true),
                        GV(48, 4, 256, 1, true), GF(48, 6, 128, 1)};
const Variant kV64[] = {GF(64, 4, 128, 1), GV(64, 8, 128, 1, false), GV(64, 8, 256, 1, true),
                        GV(64, 4, 256, 1, true)};

#undef GV
#undef GF

bool table(int L, const Variant **v, int *n) {
    switch (L) {
#define T(X) case X: *v = kV##X; *n = (int)(sizeof(kV##X) / sizeof(Variant)); return true;
        T(8) T(16) T(24) T(32) T(48) T(64)
#undef T
    }
    return false;
}

}  // namespace

bool gridder_supported(int L) {
    const Variant *v;
    int n;
    return table(L, &v, &n);
}

int gridder_variant_count(int L) {
    const Variant *v;
    int n;
    return table(L, &v, &n) ? n : 0;
}

const char *gridder_variant_name(int L, int i) {
    const Variant *v;
    int n;
    if (!table(L, &v, &n) || i < 0 || i >= n) return nullptr;
    return v[i].name;
}

idg_status launch_gridder(const Geometry &g, const SubgridSet &set, int variant, const void *vis,
                          const uint8_t *flags, const void *aterms, const float *taper, void *out, void *stream) {
    const Variant *v;
    int n;
    if (!table(g.L, &v, &n)) return fail(IDG_ERR_UNSUPPORTED, "subgrid size not compiled in");
    if (set.count <= 0) return IDG_OK;
    if (g.recurrence) return launch_gridder_rec(g, set, vis, flags, aterms, taper, out, stream);
    if (variant < 0) variant = get_variant(IDG_KERNEL_GRIDDER, g.L);
    if (variant >= n) variant = 0;
    return v[variant].fn(g, set, vis, flags, aterms, taper, out, (cudaStream_t)stream);
}

}  // namespace idg
