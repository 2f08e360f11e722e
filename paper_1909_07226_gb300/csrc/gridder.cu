// Gridder: subgrid images by direct summation (Algorithm 1, inner loops;
// Eq. ShiftedDirectImaging), followed by the image-domain kernel
// taper * A_p^H . I_p . A_q (Sect. 3.4).
//
// One CTA per subgrid.  Each thread owns NPX consecutive pixels of one row and
// keeps their 4-pol complex accumulators in registers; visibilities are staged
// in shared memory in batches of VB (phase coefficients and the 2x2 visibility)
// and read back as block-wide broadcasts.  Per visibility and pixel the inner
// loop issues 2 FFMA for the phase, sin and cos on the SFU, and 16 FFMA for the
// four complex multiply-adds.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace idg {
namespace {

using namespace dev;

template <int L, int NPX, int VB>
__global__ void __launch_bounds__(L * L / NPX)
gridder_kernel(Geometry g, int64_t first, int use_order, const float4 *__restrict__ vis,
               const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
               const float *__restrict__ taper, float4 *__restrict__ out) {
    constexpr int NT = L * L / NPX;
    constexpr int TPR = L / NPX;
    static_assert(L % NPX == 0, "pixels per thread must divide L");

    __shared__ float4 s_coef[VB];
    __shared__ float4 s_v01[VB];
    __shared__ float4 s_v23[VB];

    const int64_t slot = first + blockIdx.x;
    const int sid = use_order ? g.order[slot] : (int)slot;
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

    for (int k0 = 0; k0 < d.kp; k0 += VB) {
        const int nb = min(VB, d.kp - k0);
        for (int i = tid; i < nb; i += NT) {
            int t, c;
            const size_t vi = vis_index(g, d, k0 + i, t, c);
            const PhaseCoef pc = phase_coef(g, d, t, c);
            float4 v01 = vis[2 * vi], v23 = vis[2 * vi + 1];
            if (flags && flags[vi]) {   // zero weight (flags)
                v01 = make_float4(0.f, 0.f, 0.f, 0.f);
                v23 = v01;
            }
            s_coef[i] = make_float4(pc.a, pc.b, pc.c, 0.0f);
            s_v01[i] = v01;
            s_v23[i] = v23;
        }
        __syncthreads();
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
        __syncthreads();
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

template <int L, int NPX, int VB>
idg_status launch(const Geometry &g, int64_t first, int64_t count, bool use_order, const void *vis,
                  const uint8_t *flags, const void *aterms, const float *taper, void *out, cudaStream_t s) {
    constexpr int NT = L * L / NPX;
    int64_t done = 0;
    while (done < count) {   // grid-size limit of one launch
        const int64_t n = count - done < 2147483647 ? count - done : 2147483647;
        gridder_kernel<L, NPX, VB><<<(unsigned)n, NT, 0, s>>>(
            g, first + done, use_order ? 1 : 0, (const float4 *)vis, flags, (const float4 *)aterms, taper,
            (float4 *)out + (size_t)done * L * L * 2);
        done += n;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gridder launch");
    return IDG_OK;
}

}  // namespace

bool gridder_supported(int L) { return L == 8 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64; }

idg_status launch_gridder(const Geometry &g, int64_t first, int64_t count, bool use_order, const void *vis,
                          const uint8_t *flags, const void *aterms, const float *taper, void *out,
                          void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (g.L) {
    case 8: return launch<8, 1, 128>(g, first, count, use_order, vis, flags, aterms, taper, out, s);
    case 16: return launch<16, 2, 128>(g, first, count, use_order, vis, flags, aterms, taper, out, s);
    case 24: return launch<24, 3, 128>(g, first, count, use_order, vis, flags, aterms, taper, out, s);
    case 32: return launch<32, 4, 128>(g, first, count, use_order, vis, flags, aterms, taper, out, s);
    case 48: return launch<48, 6, 128>(g, first, count, use_order, vis, flags, aterms, taper, out, s);
    case 64: return launch<64, 8, 128>(g, first, count, use_order, vis, flags, aterms, taper, out, s);
    }
    return fail(IDG_ERR_UNSUPPORTED, "subgrid size not compiled in");
}

}  // namespace idg
