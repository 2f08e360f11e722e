// Image-side steps either side of the gridding path (Alg. 1 last line, Alg. 2 first
// lines; Sect. 3.5 for the W-layers, Sect. 4.2 for the effective window).
//
// Gridding side, for a grid G_k[r][q][pol] of w-layers k (w0_k = (k + k_min) w_step):
//   I(x, y) = sum_k exp(+2 pi i w0_k n'(x, y)) sum_{q,r} G_k[r][q] exp(+2 pi i ((q - N/2)(x - N/2)
//             + (r - N/2)(y - N/2)) / N) / (cbar(x) cbar(y)),
// the un-normalised centred inverse transform of every layer, the phase of the layer's
// w0 that the subgrid phasors left out (they use w - w0), summed, then divided by the
// effective window at zero shift of the 1D window a (taper c[y][x] = a_y a_x):
//   cbar(x) = L^-1 sum_j a_j D(xi_x - xi_j),  xi_x = (x - N/2) / N,  xi_j = (j - L/2) / L,
//   D(t) = sum_{m=-L/2}^{L/2-1} exp(2 pi i m t) = exp(-i pi t) sin(pi L t) / sin(pi t),
// the interpolation that the subgrid transform inside the full transform performs (the
// discrete form of Eq. effective_window; exact for a sample at a subgrid centre).
// Degridding side, its adjoint: G_k = the centred forward transform (sign -) of
// I(x, y) exp(-2 pi i w0_k n'(x, y)) / (conj cbar(x) conj cbar(y)).
// Pixel (x, y) of the image sits at l = (x - N/2) S / N, m = (y - N/2) S / N, and
// n' = sqrt(1 - l^2 - m^2) - 1 = -(l^2 + m^2) / (1 + sqrt(1 - l^2 - m^2)).
//
// For even N the centred transform is the plain one between (-1)^(x+y) and (-1)^(q+r)
// checkerboards.  A 2D transform is three passes over the image, each reading and
// writing it once with long contiguous runs:
//   rows      one CTA per image row (all four polarisations): the N-point transform
//             along x in shared memory, with the input factor applied on the load;
//   columns   the N-point transform along y as N = N1 N2 (four-step):
//     A       one CTA per (y2, block of 16 columns): the N1-point transforms over
//             y1 of the rows y1 N2 + y2, times exp(SIGN 2 pi i y2 k1 / N), written
//             back to the same rows (k1 N2 + y2);
//     B       one CTA per (k1, block of 16 columns): the N2-point transforms over
//             y2 of the contiguous rows k1 N2 + y2, written to rows k1 + N1 k2 with
//             the output factor (and the accumulation over w-layers).
// Every line transform is decimation in frequency with radix-16 steps (radix 8, 4
// or 2 for the last): a thread takes R elements of a line, forms their R-point
// transform in registers and applies the twiddles, so an N-point transform costs
// ceil(log16 N) barriers; the result is in digit-reversed order and is read back
// by index.  Twiddles come from tables of exp(SIGN 2 pi i t / n) built once per CTA
// with sincospif of exact fractions.  N is a power of two, 32 .. 4096.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "idg_internal.h"

namespace idg {
namespace {

constexpr int kRowThreads = 256;
constexpr int kColThreads = 256;
constexpr int kColBlock = 16;             // image columns per CTA of a column pass

// pointwise factor of pixel (x, y): on the way into the row pass, or out of the last column pass
struct PixOp {
    int mode;            // 0: (-1)^(x+y) only (uv side); 1: the image-side factor; 2: none
    int accumulate;      // last pass: add into the output instead of overwriting
    float w0_2pi;        // 2 pi w0 of the layer (image side)
    float sign;          // +1 gridding side (exp(+i ...)), -1 degridding side
    float S;             // image size in direction cosines
    // [N] reciprocal of the effective window at zero shift, 1 / cbar (gridding side) or
    // 1 / conj cbar (degridding side), complex; or null
    const float2 *icbar;
};

// the factor with the window's reciprocal values cx = icbar[x], cy = icbar[y] given
__device__ __forceinline__ float2 pix_factor_w(const PixOp &op, int x, int y, int N, float2 cx, float2 cy);

__device__ __forceinline__ float2 pix_factor(const PixOp &op, int x, int y, int N) {
    if (op.mode == 1 && op.icbar) return pix_factor_w(op, x, y, N, op.icbar[x], op.icbar[y]);
    return pix_factor_w(op, x, y, N, make_float2(1.0f, 0.0f), make_float2(1.0f, 0.0f));
}

__device__ __forceinline__ float2 pix_factor_w(const PixOp &op, int x, int y, int N, float2 cx, float2 cy) {
    if (op.mode == 2) return make_float2(1.0f, 0.0f);
    const float sg = ((x + y) & 1) ? -1.0f : 1.0f;
    if (op.mode == 0) return make_float2(sg, 0.0f);
    float re = sg, im = 0.0f;
    if (op.w0_2pi != 0.0f) {
        const float l = (float)(x - N / 2) * op.S / (float)N, m = (float)(y - N / 2) * op.S / (float)N;
        const float r2 = l * l + m * m;
        const float np = r2 < 1.0f ? -r2 / (1.0f + sqrtf(1.0f - r2)) : -1.0f;
        float s, c;
        sincosf(op.sign * op.w0_2pi * np, &s, &c);
        re = sg * c;
        im = sg * s;
    }
    if (op.icbar) {
        // divide by cbar(x) cbar(y) (gridding side) or by its conjugate (degridding side)
        const float pr = cx.x * cy.x - cx.y * cy.y, pi = cx.x * cy.y + cx.y * cy.x;
        const float nr = re * pr - im * pi, ni = re * pi + im * pr;
        re = nr;
        im = ni;
    }
    return make_float2(re, im);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// cos(pi m / 8), m = 0 .. 8
__device__ __forceinline__ float cos16(int m) {
    switch (m) {
    case 0: return 1.0f;
    case 1: return 0.92387953251128675613f;
    case 2: return 0.70710678118654752440f;
    case 3: return 0.38268343236508977173f;
    case 4: return 0.0f;
    case 5: return -0.38268343236508977173f;
    case 6: return -0.70710678118654752440f;
    case 7: return -0.92387953251128675613f;
    default: return -1.0f;
    }
}

// R-point transform of x in registers (R = 2, 4, 8, 16), X[k] = sum_j x[j] exp(SIGN 2 pi i j k / R),
// in natural order: radix-2 decimation in frequency with constant twiddles, then the
// bit-reversal as a register renaming
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2 (&x)[R]) {
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float2 u = x[b + i], v = x[b + i + h];
                x[b + i] = make_float2(u.x + v.x, u.y + v.y);
                const float2 d = make_float2(u.x - v.x, u.y - v.y);
                const int m = i * (16 / (2 * h));           // angle 2 pi i / (2 h) = pi m / 8
                if (m == 0) {
                    x[b + i + h] = d;
                } else if (m == 4) {                        // exp(SIGN i pi / 2) = SIGN i
                    x[b + i + h] = SIGN > 0 ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
                } else if (m == 2) {                        // (1 + SIGN i) / sqrt 2
                    const float r = 0.70710678118654752440f;
                    x[b + i + h] = SIGN > 0 ? make_float2(r * (d.x - d.y), r * (d.y + d.x))
                                            : make_float2(r * (d.x + d.y), r * (d.y - d.x));
                } else if (m == 6) {                        // (-1 + SIGN i) / sqrt 2
                    const float r = 0.70710678118654752440f;
                    x[b + i + h] = SIGN > 0 ? make_float2(-r * (d.x + d.y), r * (d.x - d.y))
                                            : make_float2(r * (d.y - d.x), -r * (d.y + d.x));
                } else {
                    // exp(SIGN i pi m / 8): cos(pi m / 8) and sin(pi m / 8) = cos(pi |4 - m| / 8)
                    const float c = cos16(m), sn = (float)SIGN * cos16(m < 4 ? 4 - m : m - 4);
                    x[b + i + h] = make_float2(d.x * c - d.y * sn, d.x * sn + d.y * c);
                }
            }
        }
    }
    float2 y[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        int r = 0;
#pragma unroll
        for (int b = 1, q = R >> 1; b < R; b <<= 1, q >>= 1)
            if (k & b) r |= q;
        y[k] = x[r];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = y[k];
}

__host__ __device__ constexpr int radix_of(int len) { return len >= 16 ? 16 : len; }

// Shared-memory layout of a CTA's lines: position-major, the NL lines of a position
// adjacent, so that a thread's polarisations sit together and the threads of a warp
// (lines fastest) touch consecutive words.  With PAD, position p sits at slot
// p + p/16 + p/256, which spreads the strided and the digit-reversed accesses of
// the long row transforms over the banks.
template <bool PAD>
__host__ __device__ __forceinline__ int slot(int p) { return PAD ? p + (p >> 4) + (p >> 8) : p; }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4) + (n >> 8) + 1; }

// Twiddles of every step of an n-point transform, step by step: a step of radix R over
// sub-transforms of length len (h = len / R) holds exp(SIGN 2 pi i i k / len) for
// k = 1 .. R - 1 and i = 0 .. h - 1 at (k - 1) h + i, so that the threads of a warp
// (consecutive i) read consecutive entries.  n - 1 entries in all.
__device__ __forceinline__ void step_twiddles(float2 *tw, int n, int sign, int tid, int nthreads) {
    int off = 0;
    for (int len = n; len > 1;) {
        const int R = radix_of(len), h = len / R;
        for (int t = tid; t < (R - 1) * h; t += nthreads) {
            const int k = t / h + 1, i = t - (k - 1) * h;
            const int e = (i * k * (n / len)) & (n - 1);        // exp(sign 2 pi i e / n), e / n exact
            float s, c;
            sincospif((float)sign * 2.0f * (float)e / (float)n, &s, &c);
            tw[off + t] = make_float2(c, s);
        }
        off += (R - 1) * h;
        len = h;
    }
}

// the step twiddles of an n-point transform into global memory (once per call, read by
// every CTA of the row pass through the cache)
__global__ void __launch_bounds__(256) step_twiddles_kernel(float2 *tw, int n, int sign) {
    step_twiddles(tw, n, sign, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// one radix-R decimation-in-frequency step over the NL lines of length n: sub-transforms
// of length len, h = len / R; tws: this step's twiddles
template <int R, int NL, bool PAD>
__device__ __forceinline__ void dif_step(float2 *buf, int n, int len, const float2 *tws, int sign) {
    const int h = len / R;
    const int gpl = n / R;
    for (int t = threadIdx.x; t < NL * gpl; t += blockDim.x) {
        const int line = t % NL, g = t / NL;
        const int b = g / h, i = g - b * h;
        const int base = b * len + i;
        float2 v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = buf[slot<PAD>(base + j * h) * NL + line];
        if (sign > 0)
            dft_reg<R, 1>(v);
        else
            dft_reg<R, -1>(v);
#pragma unroll
        for (int k = 0; k < R; ++k)      // (tws is shared memory in the column passes, global in the row pass)
            buf[slot<PAD>(base + k * h) * NL + line] = k ? cmulf(v[k], tws[(k - 1) * h + i]) : v[k];
    }
}

// the whole n-point transform of the NL lines (natural order in, digit-reversed out)
template <int NL, bool PAD>
__device__ __forceinline__ void fft_dif_lines(float2 *buf, int n, const float2 *tw, int sign) {
    int off = 0;
    for (int len = n; len > 1;) {
        const int R = radix_of(len);
        switch (R) {
        case 16: dif_step<16, NL, PAD>(buf, n, len, tw + off, sign); break;
        case 8: dif_step<8, NL, PAD>(buf, n, len, tw + off, sign); break;
        case 4: dif_step<4, NL, PAD>(buf, n, len, tw + off, sign); break;
        default: dif_step<2, NL, PAD>(buf, n, len, tw + off, sign); break;
        }
        off += (R - 1) * (len / R);
        len /= R;
        __syncthreads();
    }
}

// The same transform with the length n a compile-time constant (the 4096-point rows
// and 64-point columns of the 4096 x 4096 grid): all index arithmetic folds to shifts,
// and where it holds (no padding, or every step of radix 16: steps h = 1, 16, 256) the
// slots of a butterfly's points are slot(base) + j ps with a constant ps, so a point
// costs one add instead of the slot arithmetic.
template <int N, bool PAD>
__host__ __device__ constexpr bool slots_linear() {
    if (!PAD) return true;
    for (int len = N; len > 1; len /= 16)
        if (radix_of(len) != 16) return false;
    return true;
}

template <int R, int NL, bool PAD, int N, int LEN>
__device__ __forceinline__ void dif_step_ct(float2 *buf, const float2 *tws, int sign) {
    constexpr int H = LEN / R, GPL = N / R;
    constexpr int PS = PAD ? H + H / 16 + H / 256 : H;      // slot stride of a butterfly's points
    for (int t = threadIdx.x; t < NL * GPL; t += blockDim.x) {
        const int line = t % NL, g = t / NL;
        const int b = g / H, i = g % H;
        const int base = b * LEN + i;
        float2 v[R];
        if constexpr (slots_linear<N, PAD>()) {
            const int s0 = slot<PAD>(base) * NL + line;
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = buf[s0 + j * PS * NL];
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = buf[slot<PAD>(base + j * H) * NL + line];
        }
        if (sign > 0)
            dft_reg<R, 1>(v);
        else
            dft_reg<R, -1>(v);
        if constexpr (slots_linear<N, PAD>()) {
            const int s0 = slot<PAD>(base) * NL + line;
#pragma unroll
            for (int k = 0; k < R; ++k)      // (the last step, H = 1, has unit twiddles)
                buf[s0 + k * PS * NL] = (k && H > 1) ? cmulf(v[k], tws[(k - 1) * H + i]) : v[k];
        } else {
#pragma unroll
            for (int k = 0; k < R; ++k)
                buf[slot<PAD>(base + k * H) * NL + line] = (k && H > 1) ? cmulf(v[k], tws[(k - 1) * H + i]) : v[k];
        }
    }
}

template <int NL, bool PAD, int N, int LEN>
__device__ __forceinline__ void dif_steps_ct(float2 *buf, const float2 *tws, int sign) {
    if constexpr (LEN > 1) {
        constexpr int R = LEN >= 16 ? 16 : LEN;
        dif_step_ct<R, NL, PAD, N, LEN>(buf, tws, sign);
        __syncthreads();
        dif_steps_ct<NL, PAD, N, LEN / R>(buf, tws + (R - 1) * (LEN / R), sign);
    }
}

// The compile-time N-point transform (radix 16 only, N = 16^3) with the step twiddles
// formed in registers: T[m] = exp(SIGN 2 pi i m / N) for m < N / 16 (shared memory), a
// butterfly of the step over sub-transforms of length LEN takes w = T[i N / LEN] =
// exp(SIGN 2 pi i i / LEN) and multiplies output k by w^k, the powers by a product tree
// of depth at most 4 (w^2, w^4, w^8 by squaring, the rest as products of two of them):
// 14 complex products instead of 15 table reads, which kept the row pass waiting on L2
// (the full step table, 30 KB at N = 4096, does not stay in the L1 beside three CTAs'
// shared memory).
template <int SIGN, int NL, bool PAD, int N, int LEN>
__device__ __forceinline__ void dif_step_pow(float2 *buf, const float2 *T) {
    constexpr int R = 16, H = LEN / R, GPL = N / R;
    constexpr int PS = PAD ? H + H / 16 + H / 256 : H;
    static_assert(slots_linear<N, PAD>(), "radix 16 throughout");
    for (int t = threadIdx.x; t < NL * GPL; t += blockDim.x) {
        const int line = t % NL, g = t / NL;
        const int b = g / H, i = g % H;
        const int s0 = slot<PAD>(b * LEN + i) * NL + line;
        float2 v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = buf[s0 + j * PS * NL];
        dft_reg<R, SIGN>(v);
        buf[s0] = v[0];
        if constexpr (H > 1) {
            float2 w[R];
            w[1] = T[i * (N / LEN)];
            w[2] = cmulf(w[1], w[1]);
            w[3] = cmulf(w[2], w[1]);
            w[4] = cmulf(w[2], w[2]);
            w[5] = cmulf(w[4], w[1]);
            w[6] = cmulf(w[4], w[2]);
            w[7] = cmulf(w[4], w[3]);
            w[8] = cmulf(w[4], w[4]);
#pragma unroll
            for (int k = 9; k < R; ++k) w[k] = cmulf(w[8], w[k - 8]);
#pragma unroll
            for (int k = 1; k < R; ++k) buf[s0 + k * PS * NL] = cmulf(v[k], w[k]);
        } else {
#pragma unroll
            for (int k = 1; k < R; ++k) buf[s0 + k * PS * NL] = v[k];
        }
    }
}

// The first step (LEN = N) of the same transform with its points read straight from the
// row in global memory: line `line` of position x is polarisation 2 hp + line of pixel x
// of `row` (the image's 32-byte pixels), times the input factor of pixel (x, y).  This
// skips one shared-memory store and load of the whole row.
template <int SIGN, bool PAD, int N>
__device__ __forceinline__ void dif_step_pow_first(float2 *buf, const float2 *T, const float2 *row, int hp, int y,
                                                   const PixOp &pre) {
    constexpr int R = 16, NL = 2, H = N / R, GPL = N / R;
    constexpr int PS = PAD ? H + H / 16 + H / 256 : H;
    for (int t = threadIdx.x; t < NL * GPL; t += blockDim.x) {
        const int line = t % NL, i = t / NL;
        float2 v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int x = i + j * H;
            v[j] = cmulf(row[4 * x + 2 * hp + line], pix_factor(pre, x, y, N));
        }
        dft_reg<R, SIGN>(v);
        const int s0 = slot<PAD>(i) * NL + line;
        buf[s0] = v[0];
        float2 w[R];
        w[1] = T[i];
        w[2] = cmulf(w[1], w[1]);
        w[3] = cmulf(w[2], w[1]);
        w[4] = cmulf(w[2], w[2]);
        w[5] = cmulf(w[4], w[1]);
        w[6] = cmulf(w[4], w[2]);
        w[7] = cmulf(w[4], w[3]);
        w[8] = cmulf(w[4], w[4]);
#pragma unroll
        for (int k = 9; k < R; ++k) w[k] = cmulf(w[8], w[k - 8]);
#pragma unroll
        for (int k = 1; k < R; ++k) buf[s0 + k * PS * NL] = cmulf(v[k], w[k]);
    }
}

// The last step (LEN = 16, unit twiddles) of the 4096-point row transform with its outputs
// written straight to the row in natural order: butterfly b leaves frequency
// f = 256 k + 16 (b % 16) + b / 16 at output k, so the butterflies are taken with b / 16
// fastest across the lanes (16 consecutive pixels per warp and k) and their shared-memory
// reads stay free of bank conflicts (slot stride 273).  orow: polarisation 2 hp + line of
// pixel x at orow[4 x + 2 hp + line].
template <int SIGN>
__device__ __forceinline__ void dif_step_pow_last_store(const float2 *buf, float2 *orow, int hp) {
    constexpr int R = 16, NL = 2, N = 4096;
    for (int t = threadIdx.x; t < NL * (N / R); t += blockDim.x) {
        const int line = t % NL, q = t / NL;
        const int b = (q % 16) * 16 + q / 16;
        const int s0 = slot<true>(16 * b) * NL + line;
        float2 v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = buf[s0 + j * NL];
        dft_reg<R, SIGN>(v);
        const int f0 = 16 * (b % 16) + b / 16;
#pragma unroll
        for (int k = 0; k < R; ++k) orow[4 * (256 * k + f0) + 2 * hp + line] = v[k];
    }
}

template <int SIGN, int NL, bool PAD, int N, int LEN>
__device__ __forceinline__ void dif_steps_pow(float2 *buf, const float2 *T) {
    if constexpr (LEN > 1) {
        dif_step_pow<SIGN, NL, PAD, N, LEN>(buf, T);
        __syncthreads();
        dif_steps_pow<SIGN, NL, PAD, N, LEN / 16>(buf, T);
    }
}

// the n-point transform of the NL lines: compile-time n when NC > 0, else n at run time
template <int NL, bool PAD, int NC>
__device__ __forceinline__ void fft_lines(float2 *buf, int n, const float2 *tw, int sign) {
    if constexpr (NC > 0)
        dif_steps_ct<NL, PAD, NC, NC>(buf, tw, sign);
    else
        fft_dif_lines<NL, PAD>(buf, n, tw, sign);
}

// position of frequency f in the digit-reversed output of fft_dif_lines
__device__ __forceinline__ int dif_pos(int f, int n) {
    int pos = 0;
    for (int len = n; len > 1;) {
        const int R = radix_of(len), h = len / R;
        pos += (f & (R - 1)) * h;
        f >>= (R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1);
        len = h;
    }
    return pos;
}

// row pass: CTA 2 y + hp transforms row y along x for polarisations 2 hp and 2 hp + 1
// (half of each 32-byte pixel; the other CTA of the row reads the other half of the
// same sectors); in -> out, pre on the load.  Two CTAs fit an SM, so one CTA's loads
// and stores overlap the other's transform.
template <int SIGN, int NC>
__global__ void __launch_bounds__(kRowThreads) image_rows_kernel(const float4 *__restrict__ in,
                                                                 float4 *__restrict__ out, int N, PixOp pre,
                                                                 const float2 *__restrict__ tw) {
    extern __shared__ float4 img_smem4[];
    float4 *buf4 = img_smem4;                                     // [slot(N)] x (2 polarisations)
    float2 *buf = (float2 *)img_smem4;
    const int y = blockIdx.x >> 1, hp = blockIdx.x & 1;
    const float4 *row = in + (size_t)y * N * 2 + hp;
    constexpr bool POW = NC == 4096;                 // 16^3: the power-twiddle form
    float2 *T = buf + 2 * padded_len(NC ? NC : 32);  // [N / 16] exp(SIGN 2 pi i m / N)
    if constexpr (POW) {
        for (int m = threadIdx.x; m < NC / 16; m += kRowThreads) {
            float sn, cs;
            sincospif((float)SIGN * 2.0f * (float)m / (float)NC, &sn, &cs);
            T[m] = make_float2(cs, sn);
        }
        // the checkerboard only (the gridding side's uv grid): the first step reads the row
        // itself.  Only instantiated for SIGN > 0: in the image-to-grid kernel a second load
        // path cost its window-factor loads 8 % (measured).
        if (SIGN > 0 && pre.mode == 0) {
            __syncthreads();
            dif_step_pow_first<SIGN, true, 4096>(buf, T, (const float2 *)(in + (size_t)y * N * 2), hp, y, pre);
        } else {                 // (with the window's reciprocal: once per pixel, on the load)
            for (int x = threadIdx.x; x < N; x += kRowThreads) {
                const float4 a = row[2 * x];
                const float2 f = pix_factor(pre, x, y, N);
                const float2 p0 = cmulf(make_float2(a.x, a.y), f), p1 = cmulf(make_float2(a.z, a.w), f);
                buf4[slot<true>(x)] = make_float4(p0.x, p0.y, p1.x, p1.y);
            }
            __syncthreads();
            dif_step_pow<SIGN, 2, true, 4096, 4096>(buf, T);
        }
        __syncthreads();
        dif_step_pow<SIGN, 2, true, 4096, 256>(buf, T);
        __syncthreads();
        dif_step_pow_last_store<SIGN>(buf, (float2 *)(out + (size_t)y * N * 2), hp);
        return;
    } else {
        for (int x = threadIdx.x; x < N; x += kRowThreads) {
            const float4 a = row[2 * x];
            const float2 f = pix_factor(pre, x, y, N);
            const float2 p0 = cmulf(make_float2(a.x, a.y), f), p1 = cmulf(make_float2(a.z, a.w), f);
            buf4[slot<true>(x)] = make_float4(p0.x, p0.y, p1.x, p1.y);
        }
        __syncthreads();
        fft_lines<2, true, NC>(buf, N, tw, SIGN);
    }
    float4 *orow = out + (size_t)y * N * 2 + hp;
    for (int x = threadIdx.x; x < N; x += kRowThreads) orow[2 * x] = buf4[slot<true>(dif_pos(x, NC ? NC : N))];
}

// N1 of split_n at compile time (N = N1 N2, N1 >= N2, both powers of two)
__host__ __device__ constexpr int split_n_ct(int N) {
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    return 1 << ((logN + 1) / 2);
}
static_assert(split_n_ct(4096) == 64, "4096 = 64 x 64");

// The 64-point transforms of the column passes at N = 4096 (N1 = N2 = 64) straight from
// global memory to global memory: line l of a CTA is polarisation l % 4 of column
// c0 + l / 4, so the 32 lines of a warp are 256 contiguous bytes of an image row.  The
// first step (radix 16, H = 4) reads its 16 points (positions i + 4 j) from the rows
// src_row(i + 4 j), the second (radix 4, H = 1) leaves frequency f = b + 16 k at
// position 4 b + k and hands it to out(f, line, value): one shared-memory exchange
// between the steps instead of a load, two steps and a store through shared memory.
// tw: the step twiddles of the 64-point transform (step_twiddles).
template <int SIGN, typename SrcRow, typename Out>
__device__ __forceinline__ void cols64(float2 *buf, const float2 *tw, SrcRow src_row, Out out) {
    constexpr int NL = 4 * kColBlock, H = 4;
    static_assert(NL * H == kColThreads, "one first-step butterfly per thread");
    {
        const int line = threadIdx.x % NL, i = threadIdx.x / NL;
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = src_row(i + H * j)[line];
        dft_reg<16, SIGN>(v);
        buf[i * NL + line] = v[0];
#pragma unroll
        for (int k = 1; k < 16; ++k) buf[(i + H * k) * NL + line] = cmulf(v[k], tw[(k - 1) * H + i]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NL * 16; t += kColThreads) {
        const int line = t % NL, b = t / NL;
        float2 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = buf[(4 * b + k) * NL + line];
        dft_reg<4, SIGN>(v);
#pragma unroll
        for (int k = 0; k < 4; ++k) out(b + 16 * k, line, v[k]);
    }
}

// column pass A (four-step, N = N1 N2): CTA (y2, column block) transforms over y1 the
// rows y1 N2 + y2 of kColBlock columns (4 kColBlock lines of N1 points), multiplies
// output k1 by exp(SIGN 2 pi i y2 k1 / N) and writes it to row k1 N2 + y2 (in place)
template <int SIGN, int NC>
__global__ void __launch_bounds__(kColThreads) image_cols_a_kernel(float4 *__restrict__ img, int N, int N1, int N2) {
    extern __shared__ float4 img_smem4[];
    constexpr int NL = 4 * kColBlock;
    float4 *buf4 = img_smem4;                       // [N1][NL]: position-major, 16 pixels of 4 polarisations
    float2 *buf = (float2 *)img_smem4;
    float2 *tw = buf + NL * N1;
    const int nb = N / kColBlock;
    const int y2 = blockIdx.x / nb, c0 = (blockIdx.x % nb) * kColBlock;
    float2 *w4 = tw + N1;                           // exp(SIGN 2 pi i y2 k1 / N), k1 < N1
    step_twiddles(tw, N1, SIGN, threadIdx.x, blockDim.x);
    for (int k1 = threadIdx.x; k1 < N1; k1 += blockDim.x) {
        float s, co;
        sincospif((float)SIGN * 2.0f * (float)((y2 * k1) & (N - 1)) / (float)N, &s, &co);
        w4[k1] = make_float2(co, s);
    }
    if constexpr (NC == 4096) {
        __syncthreads();                            // the twiddles
        float2 *img2 = (float2 *)img;
        cols64<SIGN>(buf, tw,
                     [&](int y1) { return img2 + ((size_t)(y1 * 64 + y2) * 4096 + c0) * 4; },
                     [&](int k1, int line, float2 v) {
                         img2[((size_t)(k1 * 64 + y2) * 4096 + c0) * 4 + line] = cmulf(v, w4[k1]);
                     });
        return;
    }
    for (int t = threadIdx.x; t < N1 * kColBlock; t += kColThreads) {
        const int y1 = t / kColBlock, c = t % kColBlock;
        const float4 *p = img + ((size_t)(y1 * N2 + y2) * N + c0 + c) * 2;
        buf4[(y1 * NL + 4 * c) / 2] = p[0];
        buf4[(y1 * NL + 4 * c) / 2 + 1] = p[1];
    }
    __syncthreads();
    constexpr int NS = NC ? split_n_ct(NC) : 0;       // N1 = N2 at the compile-time sizes
    fft_lines<NL, false, NS>(buf, N1, tw, SIGN);
    for (int t = threadIdx.x; t < N1 * kColBlock; t += kColThreads) {
        const int k1 = t / kColBlock, c = t % kColBlock;
        const int q = (dif_pos(k1, NS ? NS : N1) * NL + 4 * c) / 2;
        const float2 w = w4[k1];
        const float4 a = buf4[q], b = buf4[q + 1];
        const float2 p0 = cmulf(make_float2(a.x, a.y), w), p1 = cmulf(make_float2(a.z, a.w), w);
        const float2 p2 = cmulf(make_float2(b.x, b.y), w), p3 = cmulf(make_float2(b.z, b.w), w);
        float4 *o = img + ((size_t)(k1 * N2 + y2) * N + c0 + c) * 2;
        o[0] = make_float4(p0.x, p0.y, p1.x, p1.y);
        o[1] = make_float4(p2.x, p2.y, p3.x, p3.y);
    }
}

// column pass B: CTA (k1, column block) transforms over y2 the contiguous rows k1 N2 + y2
// and writes frequency k = k1 + N1 k2 to row k of out, times post(x, k) (added with
// accumulate)
template <int SIGN, int NC>
__global__ void __launch_bounds__(kColThreads) image_cols_b_kernel(const float4 *__restrict__ img,
                                                                   float4 *__restrict__ out, int N, int N1, int N2,
                                                                   PixOp post) {
    extern __shared__ float4 img_smem4[];
    constexpr int NL = 4 * kColBlock;
    float4 *buf4 = img_smem4;
    float2 *buf = (float2 *)img_smem4;
    float2 *tw = buf + NL * N2;
    const int nb = N / kColBlock;
    const int k1 = blockIdx.x / nb, c0 = (blockIdx.x % nb) * kColBlock;
    // the window's reciprocal at this CTA's columns and output rows (k1 + N1 k2)
    float2 *icx = tw + N2, *icy = icx + kColBlock;
    const bool win = post.mode == 1 && post.icbar;
    if (win) {
        for (int t = threadIdx.x; t < kColBlock + N2; t += kColThreads)
            icx[t] = t < kColBlock ? post.icbar[c0 + t] : post.icbar[k1 + N1 * (t - kColBlock)];
    }
    step_twiddles(tw, N2, SIGN, threadIdx.x, blockDim.x);
    if constexpr (NC == 4096) {
        __syncthreads();                            // the twiddles and window values
        const float2 *img2 = (const float2 *)img;
        float2 *out2 = (float2 *)out;
        cols64<SIGN>(buf, tw,
                     [&](int y2) { return img2 + ((size_t)(k1 * 64 + y2) * 4096 + c0) * 4; },
                     [&](int k2, int line, float2 v) {
                         const int y = k1 + 64 * k2, c = line >> 2, x = c0 + c;
                         const float2 f = win ? pix_factor_w(post, x, y, 4096, icx[c], icy[k2])
                                              : pix_factor(post, x, y, 4096);
                         float2 r = cmulf(v, f);
                         float2 *o = out2 + ((size_t)y * 4096 + c0) * 4 + line;
                         if (post.accumulate) {
                             const float2 u = *o;
                             r = make_float2(r.x + u.x, r.y + u.y);
                         }
                         *o = r;
                     });
        return;
    }
    for (int t = threadIdx.x; t < N2 * kColBlock; t += kColThreads) {
        const int y2 = t / kColBlock, c = t % kColBlock;
        const float4 *p = img + ((size_t)(k1 * N2 + y2) * N + c0 + c) * 2;
        buf4[(y2 * NL + 4 * c) / 2] = p[0];
        buf4[(y2 * NL + 4 * c) / 2 + 1] = p[1];
    }
    __syncthreads();
    constexpr int NS = NC ? split_n_ct(NC) : 0;
    fft_lines<NL, false, NS>(buf, N2, tw, SIGN);
    for (int t = threadIdx.x; t < N2 * kColBlock; t += kColThreads) {
        const int k2 = t / kColBlock, c = t % kColBlock;
        const int q = (dif_pos(k2, NS ? NS : N2) * NL + 4 * c) / 2;
        const int y = k1 + N1 * k2, x = c0 + c;
        const float2 f = win ? pix_factor_w(post, x, y, N, icx[c], icy[k2]) : pix_factor(post, x, y, N);
        const float4 a = buf4[q], b = buf4[q + 1];
        const float2 q0 = cmulf(make_float2(a.x, a.y), f), q1 = cmulf(make_float2(a.z, a.w), f);
        const float2 q2 = cmulf(make_float2(b.x, b.y), f), q3 = cmulf(make_float2(b.z, b.w), f);
        float4 *o = out + ((size_t)y * N + x) * 2;
        float4 v0 = make_float4(q0.x, q0.y, q1.x, q1.y), v1 = make_float4(q2.x, q2.y, q3.x, q3.y);
        if (post.accumulate) {
            const float4 u0 = o[0], u1 = o[1];
            v0 = make_float4(v0.x + u0.x, v0.y + u0.y, v0.z + u0.z, v0.w + u0.w);
            v1 = make_float4(v1.x + u1.x, v1.y + u1.y, v1.z + u1.z, v1.w + u1.w);
        }
        o[0] = v0;
        o[1] = v1;
    }
}

template <int NC>
cudaError_t set_image_smem(int rs, int ca, int cb) {
    cudaError_t e = cudaFuncSetAttribute(image_rows_kernel<+1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_rows_kernel<-1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_cols_a_kernel<+1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, ca);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_cols_a_kernel<-1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, ca);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_cols_b_kernel<+1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, cb);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_cols_b_kernel<-1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, cb);
    return e;
}

void split_n(int N, int &N1, int &N2) {
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    N1 = 1 << ((logN + 1) / 2);
    N2 = N / N1;
}

size_t rows_smem(int N) { return (size_t)(2 * padded_len(N) + N / 16) * sizeof(float2); }
size_t cols_smem(int n) { return (size_t)(4 * kColBlock * n + 3 * n + kColBlock) * sizeof(float2); }

// in -> out: pre on the way in, the 2D transform of sign SIGN, post on the way out
template <int SIGN>
cudaError_t transform2d(const float4 *in, float4 *out, float4 *s1, float2 *tw, int N, const PixOp &pre,
                        const PixOp &post, cudaStream_t s) {
    int N1, N2;
    split_n(N, N1, N2);
    const int nb = N / kColBlock;
    if (N == 4096) {           // the compile-time form of the LOFAR-sized grid (its own twiddles)
        image_rows_kernel<SIGN, 4096><<<2 * N, kRowThreads, rows_smem(N), s>>>(in, s1, N, pre, tw);          // along x
        image_cols_a_kernel<SIGN, 4096><<<N2 * nb, kColThreads, cols_smem(N1), s>>>(s1, N, N1, N2);          // y1
        image_cols_b_kernel<SIGN, 4096><<<N1 * nb, kColThreads, cols_smem(N2), s>>>(s1, out, N, N1, N2, post);  // y2
    } else {
        step_twiddles_kernel<<<(N + 255) / 256, 256, 0, s>>>(tw, N, SIGN);
        image_rows_kernel<SIGN, 0><<<2 * N, kRowThreads, rows_smem(N), s>>>(in, s1, N, pre, tw);
        image_cols_a_kernel<SIGN, 0><<<N2 * nb, kColThreads, cols_smem(N1), s>>>(s1, N, N1, N2);
        image_cols_b_kernel<SIGN, 0><<<N1 * nb, kColThreads, cols_smem(N2), s>>>(s1, out, N, N1, N2, post);
    }
    return cudaGetLastError();
}

// effective window at zero shift on the image pixels (host, FP64), as (re, im) pairs.
// With t = xi_x - xi_j, e^{i pi t} = e^{i pi xi_x} e^{-i pi xi_j} and sin(pi L t) =
// (-1)^(j - L/2) sin(pi L xi_x), so only N + L exponentials are evaluated.  |t| < 2, so t
// is an integer only for N L t = -N L, 0 or N L (checked in integers); there the limit
// D = L (-1)^(t (L - 1)) e^{-i pi t} is taken.
std::vector<float> effective_window_eval(const double *a, int L, int N) {
    std::vector<float> cb(2 * (size_t)N);
    const double pi = 3.14159265358979323846;
    std::vector<double> fr(L), fi(L);
    for (int j = 0; j < L; ++j) {                 // e^{-i pi xi_j}
        const double ph = -pi * (double)(j - L / 2) / (double)L;
        fr[j] = std::cos(ph);
        fi[j] = std::sin(ph);
    }
    const long long NL = (long long)N * L;
    for (int x = 0; x < N; ++x) {
        const double xi = (double)(x - N / 2) / (double)N;
        const double er = std::cos(pi * xi), ei = std::sin(pi * xi);
        const double sl = std::sin(pi * L * xi);
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < L; ++j) {
            const double cr = er * fr[j] - ei * fi[j], ci = er * fi[j] + ei * fr[j];     // e^{i pi t}
            const long long num = (long long)(x - N / 2) * L - (long long)(j - L / 2) * N;   // t = num / (N L)
            double d;                                                                   // sin(pi L t) / sin(pi t)
            if (num == 0 || num == NL || num == -NL) {
                const long long k = num / NL;
                d = (double)L * (((k * (L - 1)) & 1) ? -1.0 : 1.0);
            } else {
                d = (((j - L / 2) & 1) ? -sl : sl) / ci;
            }
            sr += a[j] * d * cr;                     // D = e^{-i pi t} d
            si -= a[j] * d * ci;
        }
        cb[2 * x] = (float)(sr / L);
        cb[2 * x + 1] = (float)(si / L);
    }
    return cb;
}

// the last few windows (keyed by L, N and the coefficients), so that repeated calls with
// the same taper skip the host evaluation
std::vector<float> effective_window(const double *a, int L, int N) {
    struct Entry {
        int L, N;
        std::vector<double> a;
        std::vector<float> cb;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry &e : cache)
            if (e.L == L && e.N == N && std::equal(e.a.begin(), e.a.end(), a)) return e.cb;
    }
    std::vector<float> cb = effective_window_eval(a, L, N);
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() >= 8) cache.erase(cache.begin());
    cache.push_back(Entry{L, N, std::vector<double>(a, a + L), cb});
    return cb;
}

struct ImageBufs {
    cudaStream_t s;
    void *s1 = nullptr, *cbar = nullptr, *tw = nullptr;     // cbar: the reciprocal window
    explicit ImageBufs(cudaStream_t st) : s(st) {}
    ~ImageBufs() {
        if (s1) cudaFreeAsync(s1, s);
        if (cbar) cudaFreeAsync(cbar, s);
        if (tw) cudaFreeAsync(tw, s);
    }
};

idg_status image_setup(const idg_plan *p, const void *a_ptr, const void *b_ptr, const double *h_window, int sign,
                       cudaStream_t s, ImageBufs &bufs, int &logN) {
    if (!p || !a_ptr || !b_ptr) return fail(IDG_ERR_INVALID_ARG, "plan, input and output are required");
    const int N = p->N;
    if (N < 32 || N > 4096 || (N & (N - 1))) return fail(IDG_ERR_UNSUPPORTED, "the image transform needs N a power of two, 32 .. 4096");
    logN = 0;
    while ((1 << logN) < N) ++logN;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(IDG_ERR_INVALID_ARG, "the plan was created on another device");
    {
        int N1, N2;
        split_n(N, N1, N2);
        const int rs = (int)rows_smem(N), ca = (int)cols_smem(N1), cb = (int)cols_smem(N2);
        e = set_image_smem<0>(rs, ca, cb);
        if (e == cudaSuccess && N == 4096) e = set_image_smem<4096>(rs, ca, cb);
        if (e != cudaSuccess) return cuda_fail(e, "image transform shared-memory attribute");
    }
    if (h_window) {
        for (int j = 0; j < p->L; ++j)
            if (!std::isfinite(h_window[j])) return fail(IDG_ERR_INVALID_ARG, "the window must be finite");
    }
    idg_status st = scratch_alloc(dev, (size_t)N * N * 32, s, &bufs.s1);
    if (st == IDG_OK) st = scratch_alloc(dev, sizeof(float2) * N, s, &bufs.tw);
    if (st != IDG_OK) return st;
    if (h_window) {
        const std::vector<float> cb = effective_window(h_window, p->L, N);
        for (int x = 0; x < N; ++x)
            if (!(std::hypot(cb[2 * x], cb[2 * x + 1]) > 1e-30))
                return fail(IDG_ERR_INVALID_ARG, "the effective window vanishes on the image");
        // the kernels multiply by 1 / cbar (gridding side) or 1 / conj cbar (degridding side),
        // formed here in FP64 and rounded once
        std::vector<float> icb(2 * (size_t)N);
        for (int x = 0; x < N; ++x) {
            const double re = cb[2 * x], im = sign > 0 ? cb[2 * x + 1] : -(double)cb[2 * x + 1];
            const double d = re * re + im * im;
            icb[2 * x] = (float)(re / d);
            icb[2 * x + 1] = (float)(-im / d);
        }
        st = scratch_alloc(dev, sizeof(float) * 2 * N, s, &bufs.cbar);
        if (st != IDG_OK) return st;
        // (a copy from pageable memory returns once the source has been staged)
        e = cudaMemcpyAsync(bufs.cbar, icb.data(), sizeof(float) * 2 * N, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "effective window upload");
    }
    return IDG_OK;
}

}  // namespace
}  // namespace idg

using namespace idg;

extern "C" {

idg_status idg_image_from_grid(const idg_plan *p, const void *d_grid, const double *h_window, void *d_image,
                               idg_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    ImageBufs bufs(s);
    int logN = 0;
    idg_status st = image_setup(p, d_grid, d_image, h_window, +1, s, bufs, logN);
    if (st != IDG_OK) return st;
    const int N = p->N;
    for (int k = 0; k < p->stats.n_w_layers; ++k) {
        const double w0 = p->w_step > 0.0 ? (double)(k + p->stats.w_layer_min) * p->w_step : 0.0;
        const PixOp pre = {0, 0, 0.0f, 1.0f, (float)p->S, nullptr};
        const PixOp post = {1, k > 0, (float)(6.283185307179586 * w0), 1.0f, (float)p->S, (const float2 *)bufs.cbar};
        const float4 *g = (const float4 *)d_grid + (size_t)k * N * N * 2;
        cudaError_t e = transform2d<+1>(g, (float4 *)d_image, (float4 *)bufs.s1, (float2 *)bufs.tw, N, pre, post, s);
        if (e != cudaSuccess) return cuda_fail(e, "image transform launch");
    }
    return IDG_OK;
}

idg_status idg_grid_from_image(const idg_plan *p, const void *d_image, const double *h_window, void *d_grid,
                               idg_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    ImageBufs bufs(s);
    int logN = 0;
    idg_status st = image_setup(p, d_image, d_grid, h_window, -1, s, bufs, logN);
    if (st != IDG_OK) return st;
    const int N = p->N;
    for (int k = 0; k < p->stats.n_w_layers; ++k) {
        const double w0 = p->w_step > 0.0 ? (double)(k + p->stats.w_layer_min) * p->w_step : 0.0;
        const PixOp pre = {1, 0, (float)(6.283185307179586 * w0), -1.0f, (float)p->S, (const float2 *)bufs.cbar};
        const PixOp post = {0, 0, 0.0f, -1.0f, (float)p->S, nullptr};
        float4 *g = (float4 *)d_grid + (size_t)k * N * N * 2;
        cudaError_t e = transform2d<-1>((const float4 *)d_image, g, (float4 *)bufs.s1, (float2 *)bufs.tw, N, pre,
                                        post, s);
        if (e != cudaSuccess) return cuda_fail(e, "image transform launch");
    }
    return IDG_OK;
}

}  // extern "C"
