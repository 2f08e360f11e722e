// Device helpers shared by the kernels: visibility phase coefficients, 2x2
// Jones products, compile-time twiddle tables and an in-register FFT.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "idg_internal.h"

namespace idg {
namespace dev {

// ---------------------------------------------------------------------------
// x s - o for float pairs x = xh + xl, s = sh + sl, o = oh + ol, rounded once to FP32.
// The product xh sh is split exactly by an fma (Dekker's two-product, with fma), the
// difference with oh exactly by Knuth's two-sum; the terms left out (xl sl and the
// roundings of the small corrections) are about 2^-48 |x s|.  No FP64 instruction:
// FP64 issues at a small fraction of the FP32 rate on this GPU.
__device__ __forceinline__ float pair_coef(float xh, float xl, float sh, float sl, float oh, float ol) {
    const float p = __fmul_rn(xh, sh);
    float e = __fmaf_rn(xh, sh, -p);
    e = __fmaf_rn(xh, sl, e);
    e = __fmaf_rn(xl, sh, e);
    const float s = __fsub_rn(p, oh);
    const float bb = __fsub_rn(s, p);
    const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(-oh, bb));
    return __fadd_rn(s, __fadd_rn(err, __fsub_rn(e, ol)));
}

// phase coefficients of one visibility relative to its subgrid
//
// The subgrid-image phasor of Eq. (ShiftedDirectImaging) at pixel (y, x) is
//   phi = 2 pi ((u - u0) l + (v - v0) m + (w - w0) n'),  l = X S/L, m = Y S/L,
// with X = x - L/2, Y = y - L/2.  u = u_m * f/c; the coordinates are large and the
// differences small, so a = u_m (f/c) k_uv - u0 k_uv (and b, c alike) is formed from
// float pairs (hi + lo, FP64 accurate) with error-free products and sums and
// rounded once to FP32, as an FP64 evaluation rounded to FP32 would be.
struct PhaseCoef {
    float a, b, c;
};

// the plan's float-pair coordinates of (baseline, timestep) and channel scales
struct PairCoords {
    float4 uv, sc;
    float2 w;
};

__device__ __forceinline__ PairCoords pair_coords(const Geometry &g, const DevSubgrid &d, int t, int c) {
    const float4 *x = (const float4 *)g.uvw_f2 + 2 * ((size_t)d.bl * g.n_t + t);
    PairCoords r;
    r.uv = x[0];
    const float4 w4 = x[1];
    r.w = make_float2(w4.x, w4.y);
    r.sc = ((const float4 *)g.scale_f2)[c];
    return r;
}

__device__ __forceinline__ PhaseCoef pair_phase_coef(const DevSubgrid &d, const PairCoords &x) {
    PhaseCoef r;
    r.a = pair_coef(x.uv.x, x.uv.y, x.sc.x, x.sc.y, d.a0h, d.a0l);
    r.b = pair_coef(x.uv.z, x.uv.w, x.sc.x, x.sc.y, d.b0h, d.b0l);
    r.c = pair_coef(x.w.x, x.w.y, x.sc.z, x.sc.w, d.c0h, d.c0l);
    return r;
}

__device__ __forceinline__ PhaseCoef phase_coef(const Geometry &g, const DevSubgrid &d, int t, int c) {
    return pair_phase_coef(d, pair_coords(g, d, t, c));
}

// *p += v as one 16-byte reduction without a return value (relaxed, GPU scope; each
// component rounded to nearest like atomicAdd)
__device__ __forceinline__ void red_add_f4(float4 *p, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ size_t vis_index(const Geometry &g, const DevSubgrid &d, int k, int &t, int &c) {
    const int tt = k / d.nc;
    t = d.t0 + tt;
    c = d.c0 + (k - tt * d.nc);
    return ((size_t)d.bl * g.n_t + t) * g.n_chan + c;
}

// ---------------------------------------------------------------------------
// 2x2 complex matrices [[0,1],[2,3]] held as 8 floats (re, im interleaved)

struct M22 {
    float2 m[4];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // conj(a) * b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cmul_c(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ M22 load_m22(const float4 *p) {
    const float4 a = p[0], b = p[1];
    M22 r;
    r.m[0] = make_float2(a.x, a.y);
    r.m[1] = make_float2(a.z, a.w);
    r.m[2] = make_float2(b.x, b.y);
    r.m[3] = make_float2(b.z, b.w);
    return r;
}

// A^H P B  (gridding: A_p^H . P . A_q)
__device__ __forceinline__ M22 herm_mul_mul(const M22 &A, const M22 &P, const M22 &B) {
    M22 T, R;
    T.m[0] = cadd(cmulc(A.m[0], P.m[0]), cmulc(A.m[2], P.m[2]));
    T.m[1] = cadd(cmulc(A.m[0], P.m[1]), cmulc(A.m[2], P.m[3]));
    T.m[2] = cadd(cmulc(A.m[1], P.m[0]), cmulc(A.m[3], P.m[2]));
    T.m[3] = cadd(cmulc(A.m[1], P.m[1]), cmulc(A.m[3], P.m[3]));
    R.m[0] = cadd(cmul(T.m[0], B.m[0]), cmul(T.m[1], B.m[2]));
    R.m[1] = cadd(cmul(T.m[0], B.m[1]), cmul(T.m[1], B.m[3]));
    R.m[2] = cadd(cmul(T.m[2], B.m[0]), cmul(T.m[3], B.m[2]));
    R.m[3] = cadd(cmul(T.m[2], B.m[1]), cmul(T.m[3], B.m[3]));
    return R;
}

// A P B^H  (degridding: A_p . P . A_q^H)
__device__ __forceinline__ M22 mul_mul_herm(const M22 &A, const M22 &P, const M22 &B) {
    M22 T, R;
    T.m[0] = cadd(cmul(A.m[0], P.m[0]), cmul(A.m[1], P.m[2]));
    T.m[1] = cadd(cmul(A.m[0], P.m[1]), cmul(A.m[1], P.m[3]));
    T.m[2] = cadd(cmul(A.m[2], P.m[0]), cmul(A.m[3], P.m[2]));
    T.m[3] = cadd(cmul(A.m[2], P.m[1]), cmul(A.m[3], P.m[3]));
    R.m[0] = cadd(cmul_c(T.m[0], B.m[0]), cmul_c(T.m[1], B.m[1]));
    R.m[1] = cadd(cmul_c(T.m[0], B.m[2]), cmul_c(T.m[1], B.m[3]));
    R.m[2] = cadd(cmul_c(T.m[2], B.m[0]), cmul_c(T.m[3], B.m[1]));
    R.m[3] = cadd(cmul_c(T.m[2], B.m[2]), cmul_c(T.m[3], B.m[3]));
    return R;
}

// ---------------------------------------------------------------------------
// packed FP32 pairs (sm_100 family): one instruction performs two IEEE fmas on
// the halves of 64-bit registers; the pair (lo, hi) is (re, im) of a complex
// value or a broadcast (x, x)

typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------------------
// compile-time twiddles exp(-2 pi i e / n) for the subgrid transform sizes.
//
// sin and cos are summed from their Taylor series in FP64 at compile time on
// an argument reduced to [-pi, pi] (30 terms: truncation far below FP64
// rounding), then rounded to FP32.

__host__ __device__ constexpr double taylor_sin_cos(double x, bool want_sin) {
    double x2 = x * x, term = want_sin ? x : 1.0, sum = term;
    for (int k = 1; k < 30; ++k) {
        const double a = want_sin ? 2.0 * k : 2.0 * k - 1.0;
        const double b = want_sin ? 2.0 * k + 1.0 : 2.0 * k;
        term *= -x2 / (a * b);
        sum += term;
    }
    return sum;
}

// Offsets of each transform length in the table.
constexpr int kTwSizes[] = {2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
constexpr int kTwCount = sizeof(kTwSizes) / sizeof(int);
__host__ __device__ constexpr int tw_offset(int n) {
    int off = 0;
    for (int i = 0; i < kTwCount; ++i) {
        if (kTwSizes[i] == n) return off;
        off += kTwSizes[i];
    }
    return -1;
}
constexpr int kTwTotal = tw_offset(64) + 64;

struct TwiddleTable {
    float re[kTwTotal];
    float im[kTwTotal];   // sin(2 pi e / n); exp(sign 2 pi i e/n) = re + i sign im
};

__host__ __device__ constexpr TwiddleTable make_twiddles() {
    TwiddleTable t{};
    for (int i = 0; i < kTwCount; ++i) {
        const int n = kTwSizes[i];
        const int off = tw_offset(n);
        for (int e = 0; e < n; ++e) {
            const int ee = 2 * e > n ? e - n : e;                 // reduce to [-n/2, n/2]
            const double x = 6.283185307179586476925286766559 * (double)ee / (double)n;
            t.re[off + e] = (float)taylor_sin_cos(x, false);
            t.im[off + e] = (float)taylor_sin_cos(x, true);
        }
    }
    return t;
}

}  // namespace dev
}  // namespace idg

// The table lives in constant memory of each translation unit that uses it.
static __constant__ idg::dev::TwiddleTable c_twiddles = idg::dev::make_twiddles();

namespace idg {
namespace dev {

// exp(SIGN * 2 pi i e / N)
template <int N, int SIGN>
__device__ __forceinline__ float2 twiddle(int e) {
    constexpr int off = tw_offset(N);
    static_assert(off >= 0, "transform length without a twiddle table");
    return make_float2(c_twiddles.re[off + e], SIGN * c_twiddles.im[off + e]);
}

// In-register DFT of length N (N = 2^a 3^b), X[k] = sum_n x[n] exp(SIGN 2 pi i n k / N),
// by recursive decimation in time; every index is a compile-time constant after
// unrolling, so the data stays in registers and twiddles are constant operands.
template <int N, int SIGN>
struct RegFFT {
    static constexpr int R = (N % 4 == 0 && N != 8) ? 4 : ((N % 2 == 0) ? 2 : 3);
    static constexpr int M = N / R;
    __device__ __forceinline__ static void run(float2 *x) {
        float2 sub[R][M];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < M; ++m) sub[r][m] = x[m * R + r];
#pragma unroll
        for (int r = 0; r < R; ++r) RegFFT<M, SIGN>::run(sub[r]);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            float2 t[R];
            t[0] = sub[0][k];
#pragma unroll
            for (int r = 1; r < R; ++r) t[r] = cmul(sub[r][k], twiddle<N, SIGN>(r * k));
            RegFFT<R, SIGN>::run(t);
#pragma unroll
            for (int q = 0; q < R; ++q) x[k + M * q] = t[q];
        }
    }
};

template <int SIGN>
struct RegFFT<1, SIGN> {
    __device__ __forceinline__ static void run(float2 *) {}
};

template <int SIGN>
struct RegFFT<2, SIGN> {
    __device__ __forceinline__ static void run(float2 *x) {
        const float2 a = x[0], b = x[1];
        x[0] = make_float2(a.x + b.x, a.y + b.y);
        x[1] = make_float2(a.x - b.x, a.y - b.y);
    }
};

template <int SIGN>
struct RegFFT<3, SIGN> {
    __device__ __forceinline__ static void run(float2 *x) {
        // X1 = x0 + w x1 + w^2 x2, X2 = x0 + w^2 x1 + w x2, w = exp(SIGN 2 pi i / 3)
        const float2 a = x[0], b = x[1], c = x[2];
        const float s = SIGN * 0.866025403784438646763723170753f;   // sin(2 pi / 3)
        const float2 sum = make_float2(b.x + c.x, b.y + c.y);
        const float2 dif = make_float2(b.x - c.x, b.y - c.y);
        const float2 m = make_float2(a.x - 0.5f * sum.x, a.y - 0.5f * sum.y);
        x[0] = make_float2(a.x + sum.x, a.y + sum.y);
        x[1] = make_float2(m.x - s * dif.y, m.y + s * dif.x);
        x[2] = make_float2(m.x + s * dif.y, m.y - s * dif.x);
    }
};

template <int SIGN>
struct RegFFT<4, SIGN> {
    __device__ __forceinline__ static void run(float2 *x) {
        const float2 a = x[0], b = x[1], c = x[2], d = x[3];
        const float2 s02 = make_float2(a.x + c.x, a.y + c.y), d02 = make_float2(a.x - c.x, a.y - c.y);
        const float2 s13 = make_float2(b.x + d.x, b.y + d.y), d13 = make_float2(b.x - d.x, b.y - d.y);
        // (SIGN i) * d13
        const float2 r = make_float2(-SIGN * d13.y, SIGN * d13.x);
        x[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
        x[1] = make_float2(d02.x + r.x, d02.y + r.y);
        x[2] = make_float2(s02.x - s13.x, s02.y - s13.y);
        x[3] = make_float2(d02.x - r.x, d02.y - r.y);
    }
};

}  // namespace dev
}  // namespace idg
