// Gridder building blocks shared by the per-job kernels (gridder.cu) and the
// batched persistent kernels (batch.cu): staging of a visibility batch in
// shared memory and the summation of a batch into per-pixel accumulators.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace idg {
namespace dev {

struct RawVis {
    float4 v01, v23;
    PairCoords x;
    int ok;
};

__device__ __forceinline__ void fetch_raw(const Geometry &g, const DevSubgrid &d, int k, const float4 *vis,
                                          const uint8_t *flags, RawVis &r) {
    int t, c;
    const size_t vi = vis_index(g, d, k, t, c);
    r.x = pair_coords(g, d, t, c);
    r.v01 = vis[2 * vi];
    r.v23 = vis[2 * vi + 1];
    r.ok = !(flags && flags[vi]);
}

__device__ __forceinline__ void store_raw(const Geometry &g, const DevSubgrid &d, const RawVis &r, float4 *s_coef,
                                          float4 *s_v01, float4 *s_v23, int i) {
    const PhaseCoef pc = pair_phase_coef(d, r.x);
    s_coef[i] = make_float4(pc.a, pc.b, pc.c, 0.0f);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    s_v01[i] = r.ok ? r.v01 : z;     // flagged: weight 0
    s_v23[i] = r.ok ? r.v23 : z;
}

template <int NPX>
__device__ __forceinline__ void sum_batch(const float4 *s_coef, const float4 *s_v01, const float4 *s_v23, int nb,
                                          float Y, const float (&X)[NPX], const float (&NP)[NPX],
                                          float (&acc)[NPX][8]) {
#pragma unroll 2
    for (int i = 0; i < nb; ++i) {
        const float4 cf = s_coef[i];
        const float4 v01 = s_v01[i];
        const float4 v23 = s_v23[i];
        const float bY = cf.y * Y;
#pragma unroll
        for (int j = 0; j < NPX; ++j) {
            const float phase = fmaf(cf.x, X[j], fmaf(cf.z, NP[j], bY));
            float sn, cs;
            __sincosf(phase, &sn, &cs);
            // acc += V * (cs + i sn)
            acc[j][0] = fmaf(v01.x, cs, acc[j][0]); acc[j][0] = fmaf(-v01.y, sn, acc[j][0]);
            acc[j][1] = fmaf(v01.x, sn, acc[j][1]); acc[j][1] = fmaf(v01.y, cs, acc[j][1]);
            acc[j][2] = fmaf(v01.z, cs, acc[j][2]); acc[j][2] = fmaf(-v01.w, sn, acc[j][2]);
            acc[j][3] = fmaf(v01.z, sn, acc[j][3]); acc[j][3] = fmaf(v01.w, cs, acc[j][3]);
            acc[j][4] = fmaf(v23.x, cs, acc[j][4]); acc[j][4] = fmaf(-v23.y, sn, acc[j][4]);
            acc[j][5] = fmaf(v23.x, sn, acc[j][5]); acc[j][5] = fmaf(v23.y, cs, acc[j][5]);
            acc[j][6] = fmaf(v23.z, cs, acc[j][6]); acc[j][6] = fmaf(-v23.w, sn, acc[j][6]);
            acc[j][7] = fmaf(v23.z, sn, acc[j][7]); acc[j][7] = fmaf(v23.w, cs, acc[j][7]);
        }
    }
}

// Packed form: acc (re, im) += c (vr, vi) + s (-vi, vr) as two f32x2 fmas per
// polarisation; (vr, vi) and i V = (-vi, vr) are staged in shared memory.
template <int NPX>
__device__ __forceinline__ void sum_batch_f2(const float4 *s_coef, const float4 *s_v01, const float4 *s_v23,
                                             const float4 *s_iv01, const float4 *s_iv23, int nb, float Y,
                                             const float (&X)[NPX], const float (&NP)[NPX], f2_t (&acc)[NPX][4]) {
#pragma unroll 2
    for (int i = 0; i < nb; ++i) {
        const float4 cf = s_coef[i];
        const ulonglong2 v01 = *reinterpret_cast<const ulonglong2 *>(s_v01 + i);
        const ulonglong2 v23 = *reinterpret_cast<const ulonglong2 *>(s_v23 + i);
        const ulonglong2 w01 = *reinterpret_cast<const ulonglong2 *>(s_iv01 + i);
        const ulonglong2 w23 = *reinterpret_cast<const ulonglong2 *>(s_iv23 + i);
        const float bY = cf.y * Y;
#pragma unroll
        for (int j = 0; j < NPX; ++j) {
            const float phase = fmaf(cf.x, X[j], fmaf(cf.z, NP[j], bY));
            float sn, cs;
            __sincosf(phase, &sn, &cs);
            const f2_t cc = f2_pack(cs, cs), ss = f2_pack(sn, sn);
            acc[j][0] = f2_fma(ss, w01.x, f2_fma(cc, v01.x, acc[j][0]));
            acc[j][1] = f2_fma(ss, w01.y, f2_fma(cc, v01.y, acc[j][1]));
            acc[j][2] = f2_fma(ss, w23.x, f2_fma(cc, v23.x, acc[j][2]));
            acc[j][3] = f2_fma(ss, w23.y, f2_fma(cc, v23.y, acc[j][3]));
        }
    }
}

}  // namespace dev
}  // namespace idg
