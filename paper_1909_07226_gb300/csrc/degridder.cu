// Degridder: image-domain kernel taper * A_p . I_p . A_q^H (Sect. 3.4) and the
// degridding sum of Algorithm 2,
//   y_k = sum_{y,x} I_p[y][x] exp(-2 pi i (du l + dv m + dw n')).
//
// One CTA (256 threads) per subgrid.  The corrected subgrid image is staged in
// shared memory; every thread owns NV visibilities with their accumulators in
// registers and sweeps the pixels.  When a subgrid has few visibilities the
// 32 lanes of a warp are split into PG pixel groups (group g takes the columns
// x = g mod PG, so a warp's shared-memory reads hit PG consecutive pixels) and
// the partial sums are combined with warp shuffles.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace idg {
namespace {

using namespace dev;

constexpr int kThreads = 256;

template <int L, int NV>
__global__ void __launch_bounds__(kThreads)
degridder_kernel(Geometry g, int64_t first, int use_order, const float4 *__restrict__ sub,
                 const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                 const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    extern __shared__ float4 smem[];
    float4 *s_p01 = smem;                  // [L*L]
    float4 *s_p23 = smem + L * L;          // [L*L]
    float *s_np = (float *)(smem + 2 * L * L);

    const int64_t slot = first + blockIdx.x;
    const int sid = use_order ? g.order[slot] : (int)slot;
    const DevSubgrid d = g.sub[sid];
    const int tid = threadIdx.x;

    // stage taper * A_p . I . A_q^H
    const float4 *src = sub + (size_t)blockIdx.x * L * L * 2;
    for (int pix = tid; pix < L * L; pix += kThreads) {
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
    __syncthreads();

    // pixel groups per warp: as many as keep all visibilities in one pass
    int PG = 1;
    while (PG < 8 && (kThreads * NV) / (2 * PG) >= d.kp) PG *= 2;
    const int lane = tid & 31, warp = tid >> 5;
    const int grp = lane % PG;
    const int vlane = warp * (32 / PG) + lane / PG;          // visibility lane in the CTA
    const int per_pass = (kThreads / PG) * NV;
    const int ncol = L / PG;

    for (int kb = 0; kb < d.kp; kb += per_pass) {
        float ca[NV], cb[NV], cc[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int k = kb + vlane * NV + j;
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
#pragma unroll 4
            for (int xi = 0; xi < ncol; ++xi) {
                const int x = xi * PG + grp;
                const int pix = y * L + x;
                const float X = (float)(x - L / 2);
                const float4 p01 = s_p01[pix];
                const float4 p23 = s_p23[pix];
                const float np = s_np[pix];
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    const float phase = fmaf(ca[j], X, fmaf(cc[j], np, bY[j]));
                    float sn, cs;
                    __sincosf(phase, &sn, &cs);
                    // acc += P * (cs - i sn)
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
        }
        // combine the pixel groups (adjacent lanes)
        for (int off = 1; off < PG; off <<= 1)
#pragma unroll
            for (int j = 0; j < NV; ++j)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[j][q] += __shfl_xor_sync(0xffffffffu, acc[j][q], off);
        if (grp == 0) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const int k = kb + vlane * NV + j;
                if (k < d.kp) {
                    int t, c;
                    const size_t vi = vis_index(g, d, k, t, c);
                    float4 o01 = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
                    float4 o23 = make_float4(acc[j][4], acc[j][5], acc[j][6], acc[j][7]);
                    if (flags && flags[vi]) {
                        o01 = make_float4(0.f, 0.f, 0.f, 0.f);
                        o23 = o01;
                    }
                    vis_out[2 * vi] = o01;
                    vis_out[2 * vi + 1] = o23;
                }
            }
        }
    }
}

template <int L, int NV>
idg_status launch(const Geometry &g, int64_t first, int64_t count, bool use_order, const void *sub,
                  const uint8_t *flags, const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    const size_t smem = (size_t)L * L * (2 * sizeof(float4) + sizeof(float));
    auto kern = degridder_kernel<L, NV>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "degridder smem attribute");
    kern<<<(unsigned)count, kThreads, smem, s>>>(g, first, use_order ? 1 : 0, (const float4 *)sub, flags,
                                                 (const float4 *)aterms, taper, (float4 *)vis_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "degridder launch");
    return IDG_OK;
}

}  // namespace

idg_status launch_degridder(const Geometry &g, int64_t first, int64_t count, bool use_order, const void *sub,
                            const uint8_t *flags, const void *aterms, const float *taper, void *vis_out,
                            void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (g.L) {
    case 8: return launch<8, 4>(g, first, count, use_order, sub, flags, aterms, taper, vis_out, s);
    case 16: return launch<16, 4>(g, first, count, use_order, sub, flags, aterms, taper, vis_out, s);
    case 24: return launch<24, 4>(g, first, count, use_order, sub, flags, aterms, taper, vis_out, s);
    case 32: return launch<32, 4>(g, first, count, use_order, sub, flags, aterms, taper, vis_out, s);
    case 48: return launch<48, 4>(g, first, count, use_order, sub, flags, aterms, taper, vis_out, s);
    case 64: return launch<64, 4>(g, first, count, use_order, sub, flags, aterms, taper, vis_out, s);
    }
    return fail(IDG_ERR_UNSUPPORTED, "subgrid size not compiled in");
}

}  // namespace idg
