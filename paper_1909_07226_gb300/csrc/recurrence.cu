// Channel-recurrence forms of the gridder and degridder
// (precision_mode = IDG_PHASOR_RECURRENCE).
//
// With uniformly spaced channels (scale s_c = s_0 + c ds) the phase of
// visibility (t, c) at subgrid pixel (y, x) is affine in the channel index:
//   phi(t, c + j) = phi(t, c) + j delta(t, y, x),
//   delta = 2 pi ds (u_m l + v_m m + w_m n'),
// so exp(i phi) advances along the channels of a timestep by one complex
// multiply with exp(i delta).  sin/cos are evaluated only at the anchor
// channel of each run of R consecutive channels and for the step; runs start
// afresh every R channels so the FP32 drift of the product stays bounded.
// Per visibility-pixel this costs 16 FFMA (4 complex multiply-adds) + 4 for
// the phasor update, and 2 sin/cos per run of R instead of 2 per visibility.
// Anchor and step coefficients are formed in FP64 like the direct form's.
#include <cuda_runtime.h>

#include "degridder_impl.cuh"

namespace idg {
namespace {

using namespace dev;

// phase coefficients of the anchor channel c and of the per-channel step
__device__ __forceinline__ void run_coefs(const Geometry &g, const DevSubgrid &d, int t, int c, float4 &anc,
                                          float4 &stp) {
    const double *x = g.uvw + ((size_t)d.bl * g.n_t + t) * 3;
    const double sc = g.scale[c];
    anc = make_float4((float)((x[0] * sc - d.u0) * g.k_uv), (float)((x[1] * sc - d.v0) * g.k_uv),
                      (float)((x[2] * sc - d.w0) * 6.283185307179586476925286766559), 0.0f);
    stp = make_float4((float)(x[0] * g.ds * g.k_uv), (float)(x[1] * g.ds * g.k_uv),
                      (float)(x[2] * g.ds * 6.283185307179586476925286766559), 0.0f);
}

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// ---------------------------------------------------------------------------
// gridder: one CTA per subgrid, NPX pixels of a row per thread; a batch holds
// RB runs (R channels each) of visibilities plus their anchor/step coefficients

template <int L, int NPX, int R, int RB, int MINB>
__global__ void __launch_bounds__(L * L / NPX, MINB)
gridder_rec_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                   const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                   const float *__restrict__ taper, float4 *__restrict__ out) {
    constexpr int NT = L * L / NPX;
    constexpr int TPR = L / NPX;
    constexpr int VB = RB * R;
    __shared__ float4 s_v01[VB];
    __shared__ float4 s_v23[VB];
    __shared__ float4 s_anc[RB];
    __shared__ float4 s_stp[RB];
    __shared__ int s_n[RB];

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

    const int nc = d.nc;
    const int ng = (nc + R - 1) / R;        // runs per timestep
    const int nruns = d.nt * ng;
    for (int r0 = 0; r0 < nruns; r0 += RB) {
        const int nrb = min(RB, nruns - r0);
        // stage the runs: coefficients (one thread per run) and visibilities
        for (int q = tid; q < nrb; q += NT) {
            const int r = r0 + q;
            const int tt = r / ng, gg = r - (r / ng) * ng;
            float4 a, s;
            run_coefs(g, d, d.t0 + tt, d.c0 + gg * R, a, s);
            s_anc[q] = a;
            s_stp[q] = s;
            s_n[q] = min(R, nc - gg * R);
        }
        for (int i = tid; i < nrb * R; i += NT) {
            const int q = i / R, j = i - (i / R) * R;
            const int r = r0 + q;
            const int tt = r / ng, gg = r - (r / ng) * ng;
            const int c = gg * R + j;
            if (c < nc) {
                const size_t vi = ((size_t)d.bl * g.n_t + d.t0 + tt) * g.n_chan + d.c0 + c;
                float4 v01 = vis[2 * vi], v23 = vis[2 * vi + 1];
                if (flags && flags[vi]) {
                    v01 = make_float4(0.f, 0.f, 0.f, 0.f);
                    v23 = v01;
                }
                s_v01[i] = v01;
                s_v23[i] = v23;
            }
        }
        __syncthreads();
        for (int q = 0; q < nrb; ++q) {
            const float4 A = s_anc[q];
            const float4 S = s_stp[q];
            const int n = s_n[q];
            float2 E[NPX], D[NPX];
            const float bYa = A.y * Y, bYs = S.y * Y;
#pragma unroll
            for (int j = 0; j < NPX; ++j) {
                __sincosf(fmaf(A.x, X[j], fmaf(A.z, NP[j], bYa)), &E[j].y, &E[j].x);
                D[j] = make_float2(1.0f, 0.0f);
                if (n > 1) __sincosf(fmaf(S.x, X[j], fmaf(S.z, NP[j], bYs)), &D[j].y, &D[j].x);
            }
            for (int c = 0; c < n; ++c) {
                const float4 v01 = s_v01[q * R + c];
                const float4 v23 = s_v23[q * R + c];
#pragma unroll
                for (int j = 0; j < NPX; ++j) {
                    const float cs = E[j].x, sn = E[j].y;
                    acc[j][0] = fmaf(v01.x, cs, acc[j][0]); acc[j][0] = fmaf(-v01.y, sn, acc[j][0]);
                    acc[j][1] = fmaf(v01.x, sn, acc[j][1]); acc[j][1] = fmaf(v01.y, cs, acc[j][1]);
                    acc[j][2] = fmaf(v01.z, cs, acc[j][2]); acc[j][2] = fmaf(-v01.w, sn, acc[j][2]);
                    acc[j][3] = fmaf(v01.z, sn, acc[j][3]); acc[j][3] = fmaf(v01.w, cs, acc[j][3]);
                    acc[j][4] = fmaf(v23.x, cs, acc[j][4]); acc[j][4] = fmaf(-v23.y, sn, acc[j][4]);
                    acc[j][5] = fmaf(v23.x, sn, acc[j][5]); acc[j][5] = fmaf(v23.y, cs, acc[j][5]);
                    acc[j][6] = fmaf(v23.z, cs, acc[j][6]); acc[j][6] = fmaf(-v23.w, sn, acc[j][6]);
                    acc[j][7] = fmaf(v23.z, sn, acc[j][7]); acc[j][7] = fmaf(v23.w, cs, acc[j][7]);
                    E[j] = cmul2(E[j], D[j]);
                }
            }
        }
        __syncthreads();
    }

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

// ---------------------------------------------------------------------------
// degridder: every visibility lane owns one run of up to NV consecutive
// channels of one timestep; lanes split the pixels into PG groups when the
// subgrid has few runs, combined with warp shuffles

template <int L, int NV, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
degridder_rec_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ sub,
                     const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                     const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    extern __shared__ float4 smem[];
    float4 *s_p01 = smem;
    float4 *s_p23 = smem + L * L;
    float *s_np = (float *)(smem + 2 * L * L);
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int tid = threadIdx.x;
    degrid_stage_image<L>(g, d, sub + (size_t)blockIdx.x * L * L * 2, aterms, taper, s_p01, s_p23, s_np, tid, NT);
    __syncthreads();

    const int nc = d.nc;
    const int ng = (nc + NV - 1) / NV;
    const int nruns = d.nt * ng;
    const int PG = degrid_pg(nruns, NT, 1);
    const int lane = tid & 31, warp = tid >> 5;
    const int grp = lane % PG;
    const int vlane = warp * (32 / PG) + lane / PG;
    const int per_pass = NT / PG;
    const int ncol = L / PG;

    for (int rb = 0; rb < nruns; rb += per_pass) {
        const int r = rb + vlane;
        const bool valid = r < nruns;
        const int tt = valid ? r / ng : 0;
        const int gg = valid ? r - (r / ng) * ng : 0;
        const int n = valid ? min(NV, nc - gg * NV) : 0;
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), S = A;
        if (valid) run_coefs(g, d, d.t0 + tt, d.c0 + gg * NV, A, S);
        float acc[NV][8];
#pragma unroll
        for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[j][q] = 0.0f;
        for (int y = 0; y < L; ++y) {
            const float Yf = (float)(y - L / 2);
            const float bYa = A.y * Yf, bYs = S.y * Yf;
#pragma unroll 2
            for (int xi = 0; xi < ncol; ++xi) {
                const int x = xi * PG + grp;
                const int pix = y * L + x;
                const float4 p01 = s_p01[pix];
                const float4 p23 = s_p23[pix];
                const float np = s_np[pix];
                const float X = (float)(x - L / 2);
                float2 E, D = make_float2(1.0f, 0.0f);
                __sincosf(fmaf(A.x, X, fmaf(A.z, np, bYa)), &E.y, &E.x);
                if (nc > 1) __sincosf(fmaf(S.x, X, fmaf(S.z, np, bYs)), &D.y, &D.x);
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    const float cs = E.x, sn = E.y;
                    // acc += P * conj(E)
                    acc[j][0] = fmaf(p01.x, cs, acc[j][0]); acc[j][0] = fmaf(p01.y, sn, acc[j][0]);
                    acc[j][1] = fmaf(p01.y, cs, acc[j][1]); acc[j][1] = fmaf(-p01.x, sn, acc[j][1]);
                    acc[j][2] = fmaf(p01.z, cs, acc[j][2]); acc[j][2] = fmaf(p01.w, sn, acc[j][2]);
                    acc[j][3] = fmaf(p01.w, cs, acc[j][3]); acc[j][3] = fmaf(-p01.z, sn, acc[j][3]);
                    acc[j][4] = fmaf(p23.x, cs, acc[j][4]); acc[j][4] = fmaf(p23.y, sn, acc[j][4]);
                    acc[j][5] = fmaf(p23.y, cs, acc[j][5]); acc[j][5] = fmaf(-p23.x, sn, acc[j][5]);
                    acc[j][6] = fmaf(p23.z, cs, acc[j][6]); acc[j][6] = fmaf(p23.w, sn, acc[j][6]);
                    acc[j][7] = fmaf(p23.w, cs, acc[j][7]); acc[j][7] = fmaf(-p23.z, sn, acc[j][7]);
                    E = cmul2(E, D);
                }
            }
        }
        for (int off = 1; off < PG; off <<= 1)
#pragma unroll
            for (int j = 0; j < NV; ++j)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[j][q] += __shfl_xor_sync(0xffffffffu, acc[j][q], off);
        if (grp == 0 && valid) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                if (j < n) {
                    const size_t vi = ((size_t)d.bl * g.n_t + d.t0 + tt) * g.n_chan + d.c0 + gg * NV + j;
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

template <int L, int NPX, int MINB>
idg_status grid_rec(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                    const void *aterms, const float *taper, void *out, cudaStream_t s) {
    gridder_rec_kernel<L, NPX, 8, 32, MINB><<<(unsigned)set.count, L * L / NPX, 0, s>>>(
        g, set.idx, set.first, (const float4 *)vis, flags, (const float4 *)aterms, taper, (float4 *)out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "recurrence gridder launch");
    return IDG_OK;
}

template <int L, int NT, int MINB>
idg_status degrid_rec(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                      const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    const size_t smem = (size_t)L * L * (2 * sizeof(float4) + sizeof(float));
    auto kern = degridder_rec_kernel<L, 8, NT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "recurrence degridder smem attribute");
    kern<<<(unsigned)set.count, NT, smem, s>>>(g, set.idx, set.first, (const float4 *)sub, flags,
                                               (const float4 *)aterms, taper, (float4 *)vis_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "recurrence degridder launch");
    return IDG_OK;
}

}  // namespace

idg_status launch_gridder_rec(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *out, void *stream) {
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    switch (g.L) {
    case 8: return grid_rec<8, 1, 4>(g, set, vis, flags, aterms, taper, out, s);
    case 16: return grid_rec<16, 2, 3>(g, set, vis, flags, aterms, taper, out, s);
    case 24: return grid_rec<24, 3, 3>(g, set, vis, flags, aterms, taper, out, s);
    case 32: return grid_rec<32, 4, 3>(g, set, vis, flags, aterms, taper, out, s);
    case 48: return grid_rec<48, 6, 2>(g, set, vis, flags, aterms, taper, out, s);
    case 64: return grid_rec<64, 8, 1>(g, set, vis, flags, aterms, taper, out, s);
    }
    return fail(IDG_ERR_UNSUPPORTED, "subgrid size not compiled in");
}

idg_status launch_degridder_rec(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                const void *aterms, const float *taper, void *vis_out, void *stream) {
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    switch (g.L) {
    case 8: return degrid_rec<8, 128, 4>(g, set, sub, flags, aterms, taper, vis_out, s);
    case 16: return degrid_rec<16, 128, 4>(g, set, sub, flags, aterms, taper, vis_out, s);
    case 24: return degrid_rec<24, 128, 4>(g, set, sub, flags, aterms, taper, vis_out, s);
    case 32: return degrid_rec<32, 128, 4>(g, set, sub, flags, aterms, taper, vis_out, s);
    case 48: return degrid_rec<48, 128, 2>(g, set, sub, flags, aterms, taper, vis_out, s);
    case 64: return degrid_rec<64, 128, 1>(g, set, sub, flags, aterms, taper, vis_out, s);
    }
    return fail(IDG_ERR_UNSUPPORTED, "subgrid size not compiled in");
}

}  // namespace idg
