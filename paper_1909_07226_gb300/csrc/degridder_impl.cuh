// Degridder kernels: image-domain kernel taper * A_p . I_p . A_q^H (Sect. 3.4)
// and the degridding sum of Algorithm 2,
//   y_k = sum_{y,x} I_p[y][x] exp(-2 pi i (du l + dv m + dw n')).
//
// One CTA of NT threads per subgrid.  The corrected subgrid image is staged in
// shared memory; every thread owns NV visibilities with their accumulators in
// registers and sweeps the pixels.  When a subgrid has few visibilities the 32
// lanes of a warp are split into PG pixel groups (group g takes the columns
// x = g mod PG, so a warp's shared-memory reads hit PG consecutive pixels) and
// the partial sums are combined with warp shuffles (__shfl_xor_sync).
//
// Two forms: PG chosen per subgrid at run time (any K_p in one launch), or PG
// fixed at compile time, which unrolls the column loop so pixel offsets and
// the coordinates x - L/2 become immediates; the launcher then splits a set of
// subgrids sorted by K_p into runs of equal PG.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace idg {
namespace dev {

// Pixel groups per warp for a subgrid of kp visibilities: as many as keep all
// its visibilities in one pass of the CTA's visibility lanes.
__host__ __device__ constexpr int degrid_pg(int kp, int nt, int nv) {
    int pg = 1;
    while (pg < 8 && (nt * nv) / (2 * pg) >= kp) pg *= 2;
    return pg;
}

template <int L>
__device__ __forceinline__ void degrid_stage_image(const Geometry &g, const DevSubgrid &d, const float4 *src,
                                                   const float4 *aterms, const float *taper, float4 *s_p01,
                                                   float4 *s_p23, float *s_np, int tid, int nt) {
    for (int pix = tid; pix < L * L; pix += nt) {
        M22 P = load_m22(src + 2 * pix);
        if (aterms) {
            const size_t base = ((size_t)d.slot * g.n_stations) * L * L;
            const M22 Ap = load_m22(aterms + 2 * (base + (size_t)d.st_p * L * L + pix));
            const M22 Aq = load_m22(aterms + 2 * (base + (size_t)d.st_q * L * L + pix));
            P = mul_mul_herm(Ap, P, Aq);
        }
        const float tw = taper[pix];
        s_p01[pix] = make_float4(tw * P.m[0].x, tw * P.m[0].y, tw * P.m[1].x, tw * P.m[1].y);
        s_p23[pix] = make_float4(tw * P.m[2].x, tw * P.m[2].y, tw * P.m[3].x, tw * P.m[3].y);
        s_np[pix] = g.nprime[pix];
    }
}

// acc += P * (cs - i sn) for one pixel and NV visibilities
template <int NV>
__device__ __forceinline__ void degrid_pixel(const float4 p01, const float4 p23, float np, float X,
                                             const float (&ca)[NV], const float (&cc)[NV], const float (&bY)[NV],
                                             float (&acc)[NV][8]) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const float phase = fmaf(ca[j], X, fmaf(cc[j], np, bY[j]));
        float sn, cs;
        __sincosf(phase, &sn, &cs);
        acc[j][0] = fmaf(p01.x, cs, acc[j][0]); acc[j][0] = fmaf(p01.y, sn, acc[j][0]);
        acc[j][1] = fmaf(p01.y, cs, acc[j][1]); acc[j][1] = fmaf(-p01.x, sn, acc[j][1]);
        acc[j][2] = fmaf(p01.z, cs, acc[j][2]); acc[j][2] = fmaf(p01.w, sn, acc[j][2]);
        acc[j][3] = fmaf(p01.w, cs, acc[j][3]); acc[j][3] = fmaf(-p01.z, sn, acc[j][3]);
        acc[j][4] = fmaf(p23.x, cs, acc[j][4]); acc[j][4] = fmaf(p23.y, sn, acc[j][4]);
        acc[j][5] = fmaf(p23.y, cs, acc[j][5]); acc[j][5] = fmaf(-p23.x, sn, acc[j][5]);
        acc[j][6] = fmaf(p23.z, cs, acc[j][6]); acc[j][6] = fmaf(p23.w, sn, acc[j][6]);
        acc[j][7] = fmaf(p23.w, cs, acc[j][7]); acc[j][7] = fmaf(-p23.z, sn, acc[j][7]);
    }
}

template <int NV>
__device__ __forceinline__ void degrid_coefs(const Geometry &g, const DevSubgrid &d, int kbase, float (&ca)[NV],
                                             float (&cb)[NV], float (&cc)[NV]) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int k = kbase + j;
        ca[j] = cb[j] = cc[j] = 0.0f;
        if (k < d.kp) {
            int t, c;
            vis_index(g, d, k, t, c);
            const PhaseCoef pc = phase_coef(g, d, t, c);
            ca[j] = pc.a;
            cb[j] = pc.b;
            cc[j] = pc.c;
        }
    }
}

template <int NV>
__device__ __forceinline__ void degrid_write(const Geometry &g, const DevSubgrid &d, int kbase, const uint8_t *flags,
                                             const float (&acc)[NV][8], float4 *vis_out) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int k = kbase + j;
        if (k < d.kp) {
            int t, c;
            const size_t vi = vis_index(g, d, k, t, c);
            float4 o01 = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
            float4 o23 = make_float4(acc[j][4], acc[j][5], acc[j][6], acc[j][7]);
            if (flags && flags[vi]) {   // flagged visibilities are output as 0
                o01 = make_float4(0.f, 0.f, 0.f, 0.f);
                o23 = o01;
            }
            vis_out[2 * vi] = o01;
            vis_out[2 * vi + 1] = o23;
        }
    }
}

// PGS = 0: pixel groups chosen per subgrid at run time; PGS in {1,2,4,8}: fixed.
template <int L, int NV, int PGS, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
degridder_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ sub,
                 const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                 const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    extern __shared__ float4 smem[];
    float4 *s_p01 = smem;                  // [L*L]
    float4 *s_p23 = smem + L * L;          // [L*L]
    float *s_np = (float *)(smem + 2 * L * L);

    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int tid = threadIdx.x;
    degrid_stage_image<L>(g, d, sub + (size_t)blockIdx.x * L * L * 2, aterms, taper, s_p01, s_p23, s_np, tid, NT);
    __syncthreads();

    const int PG = PGS ? PGS : degrid_pg(d.kp, NT, NV);
    const int lane = tid & 31, warp = tid >> 5;
    const int grp = lane % PG;
    const int vlane = warp * (32 / PG) + lane / PG;          // visibility lane in the CTA
    const int per_pass = (NT / PG) * NV;

    for (int kb = 0; kb < d.kp; kb += per_pass) {
        float ca[NV], cb[NV], cc[NV];
        degrid_coefs<NV>(g, d, kb + vlane * NV, ca, cb, cc);
        float acc[NV][8];
#pragma unroll
        for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[j][q] = 0.0f;

        for (int y = 0; y < L; ++y) {
            const float Y = (float)(y - L / 2);
            float bY[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) bY[j] = cb[j] * Y;
            if (PGS) {
                // compile-time columns: x = xi * PGS + grp
                const float4 *r01 = s_p01 + y * L + grp;
                const float4 *r23 = s_p23 + y * L + grp;
                const float *rnp = s_np + y * L + grp;
                const float X0 = (float)(grp - L / 2);
#pragma unroll 8
                for (int xi = 0; xi < L / (PGS ? PGS : 1); ++xi)
                    degrid_pixel<NV>(r01[xi * PGS], r23[xi * PGS], rnp[xi * PGS], X0 + (float)(xi * PGS), ca, cc,
                                     bY, acc);
            } else {
                const int ncol = L / PG;
#pragma unroll 4
                for (int xi = 0; xi < ncol; ++xi) {
                    const int x = xi * PG + grp;
                    const int pix = y * L + x;
                    degrid_pixel<NV>(s_p01[pix], s_p23[pix], s_np[pix], (float)(x - L / 2), ca, cc, bY, acc);
                }
            }
        }
        // combine the pixel groups (adjacent lanes)
#pragma unroll
        for (int off = 1; off < (PGS ? PGS : 8); off <<= 1) {
            if (!PGS && off >= PG) break;
#pragma unroll
            for (int j = 0; j < NV; ++j)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[j][q] += __shfl_xor_sync(0xffffffffu, acc[j][q], off);
        }
        if (grp == 0) degrid_write<NV>(g, d, kb + vlane * NV, flags, acc, vis_out);
    }
}

using DegridLaunchFn = idg_status (*)(const Geometry &, const SubgridSet &, const void *, const uint8_t *,
                                      const void *, const float *, void *, cudaStream_t);

template <int L, int NV, int PGS, int NT, int MINB>
idg_status degrid_launch_kernel(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    const size_t smem = (size_t)L * L * (2 * sizeof(float4) + sizeof(float));
    auto kern = degridder_kernel<L, NV, PGS, NT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "degridder smem attribute");
    kern<<<(unsigned)set.count, NT, smem, s>>>(g, set.idx, set.first, (const float4 *)sub, flags,
                                               (const float4 *)aterms, taper, (float4 *)vis_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "degridder launch");
    return IDG_OK;
}

// Static-PG form: split the set into runs of equal PG (few runs when the set
// is sorted by K_p) and launch the matching instantiation for each run.
template <int L, int NV, int NT, int MINB>
idg_status degrid_launch_static(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    if (!set.kp_host) return fail(IDG_ERR_INVALID_ARG, "degridder: K_p of the subgrid set is required");
    int64_t b = 0;
    while (b < set.count) {
        const int pg = degrid_pg(set.kp_host[b], NT, NV);
        int64_t e = b + 1;
        while (e < set.count && degrid_pg(set.kp_host[e], NT, NV) == pg) ++e;
        SubgridSet run{set.idx ? set.idx + b : nullptr, set.first + b, e - b, set.kp_host + b};
        const void *rsub = (const float4 *)sub + (size_t)b * L * L * 2;
        idg_status st;
        switch (pg) {
        case 1: st = degrid_launch_kernel<L, NV, 1, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        case 2: st = degrid_launch_kernel<L, NV, 2, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        case 4: st = degrid_launch_kernel<L, NV, 4, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        default: st = degrid_launch_kernel<L, NV, 8, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        }
        if (st != IDG_OK) return st;
        b = e;
    }
    return IDG_OK;
}

// Packed form: y (re, im) += c (pr, pi) + s (pi, -pr) as two f32x2 fmas per
// polarisation.  Shared memory holds P, -i P and n' per pixel; the pixel
// groups are fixed at compile time (PGS in {1,2,4,8}).
template <int L, int NV, int PGS, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
degridder_f2_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ sub,
                    const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                    const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    extern __shared__ float4 smem[];
    float4 *s_p01 = smem;                  // [L*L] (pr, pi) pairs, pols 0 and 1
    float4 *s_p23 = smem + L * L;          // pols 2 and 3
    float4 *s_q01 = smem + 2 * L * L;      // -i P = (pi, -pr)
    float4 *s_q23 = smem + 3 * L * L;
    float *s_np = (float *)(smem + 4 * L * L);

    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int tid = threadIdx.x;
    degrid_stage_image<L>(g, d, sub + (size_t)blockIdx.x * L * L * 2, aterms, taper, s_p01, s_p23, s_np, tid, NT);
    __syncthreads();
    for (int pix = tid; pix < L * L; pix += NT) {
        const float4 a = s_p01[pix], b = s_p23[pix];
        s_q01[pix] = make_float4(a.y, -a.x, a.w, -a.z);
        s_q23[pix] = make_float4(b.y, -b.x, b.w, -b.z);
    }
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    const int grp = lane % PGS;
    const int vlane = warp * (32 / PGS) + lane / PGS;
    const int per_pass = (NT / PGS) * NV;

    for (int kb = 0; kb < d.kp; kb += per_pass) {
        float ca[NV], cb[NV], cc[NV];
        degrid_coefs<NV>(g, d, kb + vlane * NV, ca, cb, cc);
        f2_t acc[NV][4];
#pragma unroll
        for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = f2_pack(0.0f, 0.0f);
        for (int y = 0; y < L; ++y) {
            const float Y = (float)(y - L / 2);
            float bY[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) bY[j] = cb[j] * Y;
            const int row = y * L + grp;
            const float X0 = (float)(grp - L / 2);
#pragma unroll 4
            for (int xi = 0; xi < L / PGS; ++xi) {
                const int pix = row + xi * PGS;
                const ulonglong2 p01 = *reinterpret_cast<const ulonglong2 *>(s_p01 + pix);
                const ulonglong2 p23 = *reinterpret_cast<const ulonglong2 *>(s_p23 + pix);
                const ulonglong2 q01 = *reinterpret_cast<const ulonglong2 *>(s_q01 + pix);
                const ulonglong2 q23 = *reinterpret_cast<const ulonglong2 *>(s_q23 + pix);
                const float np = s_np[pix];
                const float X = X0 + (float)(xi * PGS);
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    const float phase = fmaf(ca[j], X, fmaf(cc[j], np, bY[j]));
                    float sn, cs;
                    __sincosf(phase, &sn, &cs);
                    const f2_t c2 = f2_pack(cs, cs), s2 = f2_pack(sn, sn);
                    acc[j][0] = f2_fma(s2, q01.x, f2_fma(c2, p01.x, acc[j][0]));
                    acc[j][1] = f2_fma(s2, q01.y, f2_fma(c2, p01.y, acc[j][1]));
                    acc[j][2] = f2_fma(s2, q23.x, f2_fma(c2, p23.x, acc[j][2]));
                    acc[j][3] = f2_fma(s2, q23.y, f2_fma(c2, p23.y, acc[j][3]));
                }
            }
        }
        float facc[NV][8];
#pragma unroll
        for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) f2_unpack(acc[j][q], facc[j][2 * q], facc[j][2 * q + 1]);
#pragma unroll
        for (int off = 1; off < PGS; off <<= 1)
#pragma unroll
            for (int j = 0; j < NV; ++j)
#pragma unroll
                for (int q = 0; q < 8; ++q) facc[j][q] += __shfl_xor_sync(0xffffffffu, facc[j][q], off);
        if (grp == 0) degrid_write<NV>(g, d, kb + vlane * NV, flags, facc, vis_out);
    }
}

template <int L, int NV, int PGS, int NT, int MINB>
idg_status degrid_f2_launch_kernel(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                   const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    const size_t smem = (size_t)L * L * (4 * sizeof(float4) + sizeof(float));
    auto kern = degridder_f2_kernel<L, NV, PGS, NT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "degridder smem attribute");
    kern<<<(unsigned)set.count, NT, smem, s>>>(g, set.idx, set.first, (const float4 *)sub, flags,
                                               (const float4 *)aterms, taper, (float4 *)vis_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "degridder launch");
    return IDG_OK;
}

template <int L, int NV, int NT, int MINB>
idg_status degrid_f2_launch_static(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                   const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    if (!set.kp_host) return fail(IDG_ERR_INVALID_ARG, "degridder: K_p of the subgrid set is required");
    int64_t b = 0;
    while (b < set.count) {
        const int pg = degrid_pg(set.kp_host[b], NT, NV);
        int64_t e = b + 1;
        while (e < set.count && degrid_pg(set.kp_host[e], NT, NV) == pg) ++e;
        SubgridSet run{set.idx ? set.idx + b : nullptr, set.first + b, e - b, set.kp_host + b};
        const void *rsub = (const float4 *)sub + (size_t)b * L * L * 2;
        idg_status st;
        switch (pg) {
        case 1: st = degrid_f2_launch_kernel<L, NV, 1, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        case 2: st = degrid_f2_launch_kernel<L, NV, 2, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        case 4: st = degrid_f2_launch_kernel<L, NV, 4, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        default: st = degrid_f2_launch_kernel<L, NV, 8, NT, MINB>(g, run, rsub, flags, aterms, taper, vis_out, s); break;
        }
        if (st != IDG_OK) return st;
        b = e;
    }
    return IDG_OK;
}

struct DegridVariant {
    const char *name;
    DegridLaunchFn fn;
};

}  // namespace dev

// tables of variants per L, defined in degridder_l32.cu and degridder.cu
bool degridder_table(int L, const dev::DegridVariant **v, int *n);
bool degridder_table_l32(const dev::DegridVariant **v, int *n);

}  // namespace idg
