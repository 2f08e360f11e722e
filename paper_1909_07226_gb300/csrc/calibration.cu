// Residuals, cost and A-term gradient for calibration (idg_aterm_gradient).
//
// The paper names calibration as an application of image domain gridding
// (Sect. 6): fitting the A-terms themselves against a full-image model needs
// residuals and derivatives, and both come out of the two directions of the
// method.  With the model grid's subgrid images P (split + inverse transform),
// B = taper . P and the degridding phasors e_k(pix) = exp(-2 pi i phi_k):
//   y_k = sum_pix e_k A_p B A_q^H            (Alg. 2 with the Sect. 3.4 A-terms)
//   r_k = yhat_k - y_k  (0 for flagged),     J = sum_k |r_k|^2
//   R(pix) = sum_k conj(e_k(pix)) r_k        (Alg. 1's direct sum, no taper, no A-terms)
//   dJ/dRe A + i dJ/dIm A:   G[a][p] += -2 R A_q B^H,   G[a][q] += -2 R^H A_p B
// per subgrid of baseline (p, q) in A-term slot a and per pixel.
//
// The call composes the library's stage kernels per chunk of subgrids: splitter
// and inverse transform (P into scratch 1), the degridder (y into the residual
// buffer), the residual kernel below (r and J), the gridder with identity
// A-terms and a unit taper (R into scratch 2), and the gradient kernel below,
// which forms both 2 x 2 triple products per pixel and adds them into the
// gradient with vector atomics.
#include <cuda_runtime.h>

#include <algorithm>

#include "idg_internal.h"

namespace idg {
namespace {

constexpr int kResThreads = 256;
constexpr int kGradThreads = 256;

// r = observed - model for the subgrid's visibilities (flagged: 0), and the
// block's share of J = sum |r|^2 added into *cost (FP64).
__global__ void __launch_bounds__(kResThreads) residual_kernel(Geometry g, const int32_t *__restrict__ idx,
                                                               int64_t first, const float4 *__restrict__ obs,
                                                               const uint8_t *__restrict__ flags,
                                                               float4 *__restrict__ res, double *cost) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    // a thread's few terms summed in FP32 (at most 2048 / 256 visibilities of 8
    // components), the block's sums in FP64 (FP64 is slow on this GPU: one use per thread)
    float accf = 0.0f;
    const int n = d.nt * d.nc;
    for (int i = threadIdx.x; i < n; i += kResThreads) {
        const int t = d.t0 + i / d.nc, c = d.c0 + i % d.nc;
        const size_t v = ((size_t)d.bl * g.n_t + t) * g.n_chan + c;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (!(flags && flags[v])) {
            const float4 o0 = obs[2 * v], o1 = obs[2 * v + 1];
            const float4 y0 = res[2 * v], y1 = res[2 * v + 1];
            r0 = make_float4(o0.x - y0.x, o0.y - y0.y, o0.z - y0.z, o0.w - y0.w);
            r1 = make_float4(o1.x - y1.x, o1.y - y1.y, o1.z - y1.z, o1.w - y1.w);
            accf += r0.x * r0.x + r0.y * r0.y + r0.z * r0.z + r0.w * r0.w + r1.x * r1.x + r1.y * r1.y +
                    r1.z * r1.z + r1.w * r1.w;
        }
        res[2 * v] = r0;
        res[2 * v + 1] = r1;
    }
    if (!cost) return;
    double acc = (double)accf;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double s_acc[kResThreads / 32];
    if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kResThreads / 32; ++w) t += s_acc[w];
        atomicAdd(cost, t);
    }
}

// 2 x 2 complex matrices [[m0, m1], [m2, m3]] as (re, im) pairs
struct M2 {
    float2 m[4];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ M2 load_m2(const float4 *p) {
    const float4 a = p[0], b = p[1];
    M2 r;
    r.m[0] = make_float2(a.x, a.y);
    r.m[1] = make_float2(a.z, a.w);
    r.m[2] = make_float2(b.x, b.y);
    r.m[3] = make_float2(b.z, b.w);
    return r;
}

__device__ __forceinline__ M2 mul(const M2 &a, const M2 &b) {
    M2 r;
    r.m[0] = cadd(cmul(a.m[0], b.m[0]), cmul(a.m[1], b.m[2]));
    r.m[1] = cadd(cmul(a.m[0], b.m[1]), cmul(a.m[1], b.m[3]));
    r.m[2] = cadd(cmul(a.m[2], b.m[0]), cmul(a.m[3], b.m[2]));
    r.m[3] = cadd(cmul(a.m[2], b.m[1]), cmul(a.m[3], b.m[3]));
    return r;
}

__device__ __forceinline__ M2 herm(const M2 &a) {
    M2 r;
    r.m[0] = conjf2(a.m[0]);
    r.m[1] = conjf2(a.m[2]);
    r.m[2] = conjf2(a.m[1]);
    r.m[3] = conjf2(a.m[3]);
    return r;
}

__device__ __forceinline__ void add_m2(float4 *dst, const M2 &v, float s) {
    atomicAdd(dst, make_float4(s * v.m[0].x, s * v.m[0].y, s * v.m[1].x, s * v.m[1].y));
    atomicAdd(dst + 1, make_float4(s * v.m[2].x, s * v.m[2].y, s * v.m[3].x, s * v.m[3].y));
}

// Per pixel of subgrid b of the chunk: B = taper P, then G[slot][p] += -2 R A_q B^H
// and G[slot][q] += -2 R^H A_p B.  R and P are the chunk's images at position b.
__global__ void __launch_bounds__(kGradThreads) gradient_kernel(Geometry g, const int32_t *__restrict__ idx,
                                                                int64_t first, const float4 *__restrict__ Rimg,
                                                                const float4 *__restrict__ Pimg,
                                                                const float4 *__restrict__ aterms,
                                                                const float *__restrict__ taper,
                                                                float4 *__restrict__ grad) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int LL = g.L * g.L;
    const size_t img = (size_t)blockIdx.x * LL * 2;
    const size_t ap = ((size_t)d.slot * g.n_stations + d.st_p) * LL * 2;
    const size_t aq = ((size_t)d.slot * g.n_stations + d.st_q) * LL * 2;
    for (int pix = threadIdx.x; pix < LL; pix += kGradThreads) {
        const M2 R = load_m2(Rimg + img + 2 * pix);
        M2 B = load_m2(Pimg + img + 2 * pix);
        const float tw = taper[pix];
#pragma unroll
        for (int i = 0; i < 4; ++i) B.m[i] = make_float2(tw * B.m[i].x, tw * B.m[i].y);
        M2 Ap, Aq;
        if (aterms) {
            Ap = load_m2(aterms + ap + 2 * pix);
            Aq = load_m2(aterms + aq + 2 * pix);
        } else {
            Ap.m[0] = Ap.m[3] = make_float2(1.f, 0.f);
            Ap.m[1] = Ap.m[2] = make_float2(0.f, 0.f);
            Aq = Ap;
        }
        const M2 gp = mul(mul(R, Aq), herm(B));
        const M2 gq = mul(mul(herm(R), Ap), B);
        add_m2(grad + ap + 2 * pix, gp, -2.0f);
        add_m2(grad + aq + 2 * pix, gq, -2.0f);
    }
}

}  // namespace

idg_status launch_calib_residual(const Geometry &g, const SubgridSet &set, const void *obs, const uint8_t *flags,
                                 void *res, double *cost, void *stream) {
    if (set.count <= 0) return IDG_OK;
    residual_kernel<<<(unsigned)set.count, kResThreads, 0, (cudaStream_t)stream>>>(
        g, set.idx, set.first, (const float4 *)obs, flags, (float4 *)res, cost);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "residual kernel launch");
}

idg_status launch_calib_gradient(const Geometry &g, const SubgridSet &set, const void *R, const void *P,
                                 const void *aterms, const float *taper, void *grad, void *stream) {
    if (set.count <= 0) return IDG_OK;
    gradient_kernel<<<(unsigned)set.count, kGradThreads, 0, (cudaStream_t)stream>>>(
        g, set.idx, set.first, (const float4 *)R, (const float4 *)P, (const float4 *)aterms, taper, (float4 *)grad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "gradient kernel launch");
}

}  // namespace idg
