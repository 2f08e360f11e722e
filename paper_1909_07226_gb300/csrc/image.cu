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
// checkerboards.  Both 2D transforms run as a row pass and a column pass, one CTA per
// line holding the line's four polarisations in shared memory (4 N complex values and
// a table of N / 2 twiddles): bit-reversed loads, then log2 N radix-2 stages.  The
// pointwise factors are applied on the way in (row pass) and on the way out (column
// pass).  N is a power of two, 16 .. 4096.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "idg_internal.h"

namespace idg {
namespace {

constexpr int kImgThreads = 512;

// pointwise factor of pixel (x, y) before (row pass) or after (column pass) a transform
struct PixOp {
    int mode;            // 0: (-1)^(x+y) only (uv side); 1: the image-side factor
    int accumulate;      // column pass: add into the output instead of overwriting
    float w0_2pi;        // 2 pi w0 of the layer (image side)
    float sign;          // +1 gridding side (exp(+i ...)), -1 degridding side
    float S;             // image size in direction cosines
    const float2 *cbar;  // [N] effective window at zero shift (complex), or null; conjugated if sign < 0
};

__device__ __forceinline__ float2 pix_factor(const PixOp &op, int x, int y, int N) {
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
    if (op.cbar) {
        // divide by cbar(x) cbar(y) (gridding side) or by its conjugate (degridding side)
        const float2 cx = op.cbar[x], cy = op.cbar[y];
        float pr = cx.x * cy.x - cx.y * cy.y, pi = cx.x * cy.y + cx.y * cy.x;
        if (op.sign < 0.0f) pi = -pi;
        const float inv = 1.0f / (pr * pr + pi * pi);
        const float nr = (re * pr + im * pi) * inv, ni = (im * pr - re * pi) * inv;
        re = nr;
        im = ni;
    }
    return make_float2(re, im);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 transform of the four lines buf[pol][N] (bit-reversed on entry),
// X[j] = sum_n x[n] exp(SIGN 2 pi i n j / N); tw[t] = exp(SIGN 2 pi i t / N), t < N / 2.
template <int SIGN>
__device__ __forceinline__ void fft_lines4(float2 *buf, const float2 *tw, int N) {
    const int half_n = N >> 1;
    for (int half = 1; half < N; half <<= 1) {
        const int stride = half_n / half;            // twiddle index step for groups of 2 half
        for (int t = threadIdx.x; t < 4 * half_n; t += blockDim.x) {
            const int pol = t / half_n, b = t - pol * half_n;
            const int j = b & (half - 1);
            const int i0 = ((b - j) << 1) + j, i1 = i0 + half;
            float2 *line = buf + pol * N;
            const float2 u = line[i0], v = cmulf(line[i1], tw[j * stride]);
            line[i0] = make_float2(u.x + v.x, u.y + v.y);
            line[i1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

template <int SIGN>
__device__ __forceinline__ void twiddles(float2 *tw, int N) {
    for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
        float s, c;
        sincospif(SIGN * 2.0f * (float)t / (float)N, &s, &c);    // t / N exact for N a power of two
        tw[t] = make_float2(c, s);
    }
}

// one CTA per row y: out[y][x][:] = transform over x of (in[y][x][:] * pre(x, y))
template <int SIGN>
__global__ void __launch_bounds__(kImgThreads)
image_rows_kernel(const float4 *__restrict__ in, float4 *__restrict__ out, int N, int logN, PixOp pre) {
    extern __shared__ float2 img_smem[];
    float2 *buf = img_smem, *tw = img_smem + 4 * N;
    const int y = blockIdx.x;
    twiddles<SIGN>(tw, N);
    const float4 *row = in + (size_t)y * N * 2;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        const float2 f = pix_factor(pre, x, y, N);
        const float4 a = row[2 * x], b = row[2 * x + 1];
        const int rx = (int)(__brev((unsigned)x) >> (32 - logN));
        buf[0 * N + rx] = cmulf(make_float2(a.x, a.y), f);
        buf[1 * N + rx] = cmulf(make_float2(a.z, a.w), f);
        buf[2 * N + rx] = cmulf(make_float2(b.x, b.y), f);
        buf[3 * N + rx] = cmulf(make_float2(b.z, b.w), f);
    }
    __syncthreads();
    fft_lines4<SIGN>(buf, tw, N);
    float4 *orow = out + (size_t)y * N * 2;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        orow[2 * x] = make_float4(buf[x].x, buf[x].y, buf[N + x].x, buf[N + x].y);
        orow[2 * x + 1] = make_float4(buf[2 * N + x].x, buf[2 * N + x].y, buf[3 * N + x].x, buf[3 * N + x].y);
    }
}

// one CTA per column x: out[y][x][:] (+)= post(x, y) * transform over y of in[.][x][:]
template <int SIGN>
__global__ void __launch_bounds__(kImgThreads)
image_cols_kernel(const float4 *__restrict__ in, float4 *__restrict__ out, int N, int logN, PixOp post) {
    extern __shared__ float2 img_smem[];
    float2 *buf = img_smem, *tw = img_smem + 4 * N;
    const int x = blockIdx.x;
    twiddles<SIGN>(tw, N);
    for (int y = threadIdx.x; y < N; y += blockDim.x) {
        const float4 a = in[((size_t)y * N + x) * 2], b = in[((size_t)y * N + x) * 2 + 1];
        const int ry = (int)(__brev((unsigned)y) >> (32 - logN));
        buf[0 * N + ry] = make_float2(a.x, a.y);
        buf[1 * N + ry] = make_float2(a.z, a.w);
        buf[2 * N + ry] = make_float2(b.x, b.y);
        buf[3 * N + ry] = make_float2(b.z, b.w);
    }
    __syncthreads();
    fft_lines4<SIGN>(buf, tw, N);
    for (int y = threadIdx.x; y < N; y += blockDim.x) {
        const float2 f = pix_factor(post, x, y, N);
        const float2 p0 = cmulf(buf[y], f), p1 = cmulf(buf[N + y], f);
        const float2 p2 = cmulf(buf[2 * N + y], f), p3 = cmulf(buf[3 * N + y], f);
        float4 *o = out + ((size_t)y * N + x) * 2;
        float4 v0 = make_float4(p0.x, p0.y, p1.x, p1.y), v1 = make_float4(p2.x, p2.y, p3.x, p3.y);
        if (post.accumulate) {
            const float4 q0 = o[0], q1 = o[1];
            v0 = make_float4(v0.x + q0.x, v0.y + q0.y, v0.z + q0.z, v0.w + q0.w);
            v1 = make_float4(v1.x + q1.x, v1.y + q1.y, v1.z + q1.z, v1.w + q1.w);
        }
        o[0] = v0;
        o[1] = v1;
    }
}

// effective window at zero shift on the image pixels (host, FP64), as (re, im) pairs
std::vector<float> effective_window(const double *a, int L, int N) {
    std::vector<float> cb(2 * (size_t)N);
    const double pi = 3.14159265358979323846;
    for (int x = 0; x < N; ++x) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < L; ++j) {
            const double t = (double)(x - N / 2) / (double)N - (double)(j - L / 2) / (double)L;
            const double k = std::nearbyint(t);
            double d;                                      // sin(pi L t) / sin(pi t)
            if (std::fabs(t - k) < 1e-12) d = (double)L * ((((long long)k * (L - 1)) & 1) ? -1.0 : 1.0);
            else d = std::sin(pi * L * t) / std::sin(pi * t);
            sr += a[j] * d * std::cos(pi * t);
            si -= a[j] * d * std::sin(pi * t);
        }
        cb[2 * x] = (float)(sr / L);
        cb[2 * x + 1] = (float)(si / L);
    }
    return cb;
}

struct ImageBufs {
    cudaStream_t s;
    void *scratch = nullptr, *cbar = nullptr;
    explicit ImageBufs(cudaStream_t st) : s(st) {}
    ~ImageBufs() {
        if (scratch) cudaFreeAsync(scratch, s);
        if (cbar) cudaFreeAsync(cbar, s);
    }
};

idg_status image_setup(const idg_plan *p, const void *a_ptr, const void *b_ptr, const double *h_window,
                       cudaStream_t s, ImageBufs &bufs, int &logN) {
    if (!p || !a_ptr || !b_ptr) return fail(IDG_ERR_INVALID_ARG, "plan, input and output are required");
    const int N = p->N;
    if (N < 16 || N > 4096 || (N & (N - 1))) return fail(IDG_ERR_UNSUPPORTED, "the image transform needs N a power of two, 16 .. 4096");
    logN = 0;
    while ((1 << logN) < N) ++logN;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(IDG_ERR_INVALID_ARG, "the plan was created on another device");
    const size_t smem = (size_t)(4 * N + N / 2) * sizeof(float2);
    e = cudaFuncSetAttribute(image_rows_kernel<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_rows_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_cols_kernel<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_cols_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "image transform shared-memory attribute");
    e = cudaMallocAsync(&bufs.scratch, (size_t)N * N * 32, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(image scratch)");
    if (h_window) {
        for (int j = 0; j < p->L; ++j)
            if (!std::isfinite(h_window[j])) return fail(IDG_ERR_INVALID_ARG, "the window must be finite");
        const std::vector<float> cb = effective_window(h_window, p->L, N);
        for (int x = 0; x < N; ++x)
            if (!(std::hypot(cb[2 * x], cb[2 * x + 1]) > 1e-30))
                return fail(IDG_ERR_INVALID_ARG, "the effective window vanishes on the image");
        e = cudaMallocAsync(&bufs.cbar, sizeof(float) * 2 * N, s);
        // (a copy from pageable memory returns once the source has been staged)
        if (e == cudaSuccess) e = cudaMemcpyAsync(bufs.cbar, cb.data(), sizeof(float) * 2 * N, cudaMemcpyHostToDevice, s);
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
    idg_status st = image_setup(p, d_grid, d_image, h_window, s, bufs, logN);
    if (st != IDG_OK) return st;
    const int N = p->N;
    const size_t smem = (size_t)(4 * N + N / 2) * sizeof(float2);
    const int n_w = p->stats.n_w_layers;
    for (int k = 0; k < n_w; ++k) {
        const double w0 = p->w_step > 0.0 ? (double)(k + p->stats.w_layer_min) * p->w_step : 0.0;
        const PixOp pre = {0, 0, 0.0f, 1.0f, (float)p->S, nullptr};
        const PixOp post = {1, k > 0, (float)(6.283185307179586 * w0), 1.0f, (float)p->S, (const float2 *)bufs.cbar};
        const float4 *g = (const float4 *)d_grid + (size_t)k * N * N * 2;
        image_rows_kernel<+1><<<N, kImgThreads, smem, s>>>(g, (float4 *)bufs.scratch, N, logN, pre);
        image_cols_kernel<+1><<<N, kImgThreads, smem, s>>>((const float4 *)bufs.scratch, (float4 *)d_image, N, logN, post);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "image transform launch");
    return IDG_OK;
}

idg_status idg_grid_from_image(const idg_plan *p, const void *d_image, const double *h_window, void *d_grid,
                               idg_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    ImageBufs bufs(s);
    int logN = 0;
    idg_status st = image_setup(p, d_image, d_grid, h_window, s, bufs, logN);
    if (st != IDG_OK) return st;
    const int N = p->N;
    const size_t smem = (size_t)(4 * N + N / 2) * sizeof(float2);
    const int n_w = p->stats.n_w_layers;
    for (int k = 0; k < n_w; ++k) {
        const double w0 = p->w_step > 0.0 ? (double)(k + p->stats.w_layer_min) * p->w_step : 0.0;
        const PixOp pre = {1, 0, (float)(6.283185307179586 * w0), -1.0f, (float)p->S, (const float2 *)bufs.cbar};
        const PixOp post = {0, 0, 0.0f, -1.0f, (float)p->S, nullptr};
        float4 *g = (float4 *)d_grid + (size_t)k * N * N * 2;
        image_rows_kernel<-1><<<N, kImgThreads, smem, s>>>((const float4 *)d_image, (float4 *)bufs.scratch, N, logN, pre);
        image_cols_kernel<-1><<<N, kImgThreads, smem, s>>>((const float4 *)bufs.scratch, g, N, logN, post);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "image transform launch");
    return IDG_OK;
}

}  // extern "C"
