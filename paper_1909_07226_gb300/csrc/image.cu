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
// checkerboards.  A 2D transform is four passes whose global accesses are all long
// contiguous runs: a row transform, a tiled transpose (32 x 32 pixels through shared
// memory), a second row transform (now along the other axis, in place) and a tiled
// transpose back, which applies the output factor and the accumulation over layers.  A row
// transform takes two CTAs per line, each holding two of the line's polarisations in
// shared memory (2 N complex values and N / 2 twiddles, about 80 KB at N = 4096, two CTAs
// per SM): bit-reversed loads into a padded layout (one slot per 128, free of bank
// conflicts), then log2 N radix-2 stages.  The input factor is applied on the first
// row pass.  N is a power of two, 32 .. 4096.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "idg_internal.h"

namespace idg {
namespace {

constexpr int kImgThreads = 512;
constexpr int kLines = 2;                 // polarisations per CTA of a row transform
constexpr int kTile = 32;                 // transpose tile (pixels)
constexpr int kPer = 4096 / kImgThreads;  // line elements per thread at the largest N

// pointwise factor of pixel (x, y): on the way into the first row pass, or in the final transpose
struct PixOp {
    int mode;            // 0: (-1)^(x+y) only (uv side); 1: the image-side factor; 2: none
    int accumulate;      // column pass: add into the output instead of overwriting
    float w0_2pi;        // 2 pi w0 of the layer (image side)
    float sign;          // +1 gridding side (exp(+i ...)), -1 degridding side
    float S;             // image size in direction cosines
    const float2 *cbar;  // [N] effective window at zero shift (complex), or null; conjugated if sign < 0
};

__device__ __forceinline__ float2 pix_factor(const PixOp &op, int x, int y, int N) {
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

// padded shared-memory slot of element i of a line (one spare slot per 128)
__device__ __forceinline__ int pad(int i) { return i + (i >> 7); }

// In-place radix-2 transform of the kLines lines buf[line][pad(N)] (bit-reversed on entry),
// X[j] = sum_n x[n] exp(SIGN 2 pi i n j / N); tw[t] = exp(SIGN 2 pi i t / N), t < N / 2.
template <int SIGN>
__device__ __forceinline__ void fft_lines(float2 *buf, const float2 *tw, int N, int logN, int stride_line) {
    const int half_n = N >> 1;
    for (int lh = 0; lh < logN; ++lh) {
        const int half = 1 << lh;
        const int stride = half_n >> lh;             // twiddle index step for groups of 2 half
        for (int t = threadIdx.x; t < kLines * half_n; t += blockDim.x) {
            const int pol = t >> (logN - 1), b = t & (half_n - 1);
            const int j = b & (half - 1);
            const int i0 = ((b - j) << 1) + j, i1 = i0 + half;
            float2 *line = buf + pol * stride_line;
            const float2 u = line[pad(i0)], v = cmulf(line[pad(i1)], tw[j * stride]);
            line[pad(i0)] = make_float2(u.x + v.x, u.y + v.y);
            line[pad(i1)] = make_float2(u.x - v.x, u.y - v.y);
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

// CTA 2 y + h (line y, polarisations 2 h, 2 h + 1): out[y][x][2h..] = transform over x of
// (in[y][x][2h..] * pre(x, y)); in place when in == out (the line is read whole first)
template <int SIGN>
__global__ void __launch_bounds__(kImgThreads)
image_rows_kernel(const float4 *in, float4 *out, int N, int logN, PixOp pre) {
    extern __shared__ float2 img_smem[];
    const int stride_line = pad(N - 1) + 1;
    float2 *buf = img_smem, *tw = img_smem + kLines * stride_line;
    const int y = blockIdx.x >> 1, h = blockIdx.x & 1;
    twiddles<SIGN>(tw, N);
    const float4 *row = in + (size_t)y * N * 2 + h;
    // all of the thread's loads first (up to kPer in flight), then the stores
    float4 v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int x = threadIdx.x + i * kImgThreads;
        if (x < N) v[i] = row[2 * x];
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int x = threadIdx.x + i * kImgThreads;
        if (x < N) {
            const float2 f = pix_factor(pre, x, y, N);
            const int rx = pad((int)(__brev((unsigned)x) >> (32 - logN)));
            buf[rx] = cmulf(make_float2(v[i].x, v[i].y), f);
            buf[stride_line + rx] = cmulf(make_float2(v[i].z, v[i].w), f);
        }
    }
    __syncthreads();
    fft_lines<SIGN>(buf, tw, N, logN, stride_line);
    float4 *orow = out + (size_t)y * N * 2 + h;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        const float2 p0 = buf[pad(x)], p1 = buf[stride_line + pad(x)];
        orow[2 * x] = make_float4(p0.x, p0.y, p1.x, p1.y);
    }
}

// out[r][c] (+)= post(x = c, y = r) * in[c][r] for 32-byte pixels, one 32 x 32 tile per CTA
// (32 x 8 threads), staged through shared memory so that reads and writes are contiguous
__global__ void __launch_bounds__(kTile * 8)
image_transpose_kernel(const float4 *__restrict__ in, float4 *__restrict__ out, int N, PixOp post) {
    __shared__ float4 tile[kTile][kTile + 1][2];
    const int tx = threadIdx.x & (kTile - 1), ty = threadIdx.x >> 5;
    const int c0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;      // output tile origin
    float4 ld[kTile / 8][2];
#pragma unroll
    for (int i = 0; i < kTile / 8; ++i) {        // input rows c0 + ty + 8 i, columns r0 + tx
        const float4 *p = in + ((size_t)(c0 + ty + 8 * i) * N + (r0 + tx)) * 2;
        ld[i][0] = p[0];
        ld[i][1] = p[1];
    }
#pragma unroll
    for (int i = 0; i < kTile / 8; ++i) {
        tile[ty + 8 * i][tx][0] = ld[i][0];
        tile[ty + 8 * i][tx][1] = ld[i][1];
    }
    __syncthreads();
#pragma unroll
    for (int k = ty; k < kTile; k += 8) {        // output row r0 + k, column c0 + tx
        const int r = r0 + k, c = c0 + tx;
        const float2 f = pix_factor(post, c, r, N);
        const float4 a = tile[tx][k][0], b = tile[tx][k][1];
        const float2 q0 = cmulf(make_float2(a.x, a.y), f), q1 = cmulf(make_float2(a.z, a.w), f);
        const float2 q2 = cmulf(make_float2(b.x, b.y), f), q3 = cmulf(make_float2(b.z, b.w), f);
        float4 *o = out + ((size_t)r * N + c) * 2;
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

// in -> out: pre on the way in, the 2D transform of sign SIGN, post on the way out
template <int SIGN>
cudaError_t transform2d(const float4 *in, float4 *out, float4 *s1, float4 *s2, int N, int logN, const PixOp &pre,
                        const PixOp &post, cudaStream_t s) {
    const int stride_line = (N - 1) + ((N - 1) >> 7) + 1;
    const size_t smem = (size_t)(kLines * stride_line + N / 2) * sizeof(float2);
    const PixOp none = {2, 0, 0.0f, 1.0f, 0.0f, nullptr};
    const dim3 tiles(N / kTile, N / kTile);
    PixOp mid = none;
    image_rows_kernel<SIGN><<<2 * N, kImgThreads, smem, s>>>(in, s1, N, logN, pre);          // along x
    image_transpose_kernel<<<tiles, kTile * 8, 0, s>>>(s1, s2, N, mid);                      // s2[x][y]
    image_rows_kernel<SIGN><<<2 * N, kImgThreads, smem, s>>>(s2, s2, N, logN, none);         // along y
    image_transpose_kernel<<<tiles, kTile * 8, 0, s>>>(s2, out, N, post);                    // out[y][x]
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
    void *s1 = nullptr, *s2 = nullptr, *cbar = nullptr;
    explicit ImageBufs(cudaStream_t st) : s(st) {}
    ~ImageBufs() {
        if (s1) cudaFreeAsync(s1, s);
        if (s2) cudaFreeAsync(s2, s);
        if (cbar) cudaFreeAsync(cbar, s);
    }
};

idg_status image_setup(const idg_plan *p, const void *a_ptr, const void *b_ptr, const double *h_window,
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
    const int stride_line = (N - 1) + ((N - 1) >> 7) + 1;
    const size_t smem = (size_t)(kLines * stride_line + N / 2) * sizeof(float2);
    e = cudaFuncSetAttribute(image_rows_kernel<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(image_rows_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "image transform shared-memory attribute");
    if (h_window) {
        for (int j = 0; j < p->L; ++j)
            if (!std::isfinite(h_window[j])) return fail(IDG_ERR_INVALID_ARG, "the window must be finite");
    }
    idg_status st = scratch_alloc(dev, (size_t)N * N * 32, s, &bufs.s1);
    if (st == IDG_OK) st = scratch_alloc(dev, (size_t)N * N * 32, s, &bufs.s2);
    if (st != IDG_OK) return st;
    if (h_window) {
        const std::vector<float> cb = effective_window(h_window, p->L, N);
        for (int x = 0; x < N; ++x)
            if (!(std::hypot(cb[2 * x], cb[2 * x + 1]) > 1e-30))
                return fail(IDG_ERR_INVALID_ARG, "the effective window vanishes on the image");
        st = scratch_alloc(dev, sizeof(float) * 2 * N, s, &bufs.cbar);
        if (st != IDG_OK) return st;
        // (a copy from pageable memory returns once the source has been staged)
        e = cudaMemcpyAsync(bufs.cbar, cb.data(), sizeof(float) * 2 * N, cudaMemcpyHostToDevice, s);
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
    for (int k = 0; k < p->stats.n_w_layers; ++k) {
        const double w0 = p->w_step > 0.0 ? (double)(k + p->stats.w_layer_min) * p->w_step : 0.0;
        const PixOp pre = {0, 0, 0.0f, 1.0f, (float)p->S, nullptr};
        const PixOp post = {1, k > 0, (float)(6.283185307179586 * w0), 1.0f, (float)p->S, (const float2 *)bufs.cbar};
        const float4 *g = (const float4 *)d_grid + (size_t)k * N * N * 2;
        cudaError_t e = transform2d<+1>(g, (float4 *)d_image, (float4 *)bufs.s1, (float4 *)bufs.s2, N, logN, pre, post, s);
        if (e != cudaSuccess) return cuda_fail(e, "image transform launch");
    }
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
    for (int k = 0; k < p->stats.n_w_layers; ++k) {
        const double w0 = p->w_step > 0.0 ? (double)(k + p->stats.w_layer_min) * p->w_step : 0.0;
        const PixOp pre = {1, 0, (float)(6.283185307179586 * w0), -1.0f, (float)p->S, (const float2 *)bufs.cbar};
        const PixOp post = {0, 0, 0.0f, -1.0f, (float)p->S, nullptr};
        float4 *g = (float4 *)d_grid + (size_t)k * N * N * 2;
        cudaError_t e = transform2d<-1>((const float4 *)d_image, g, (float4 *)bufs.s1, (float4 *)bufs.s2, N, logN, pre, post, s);
        if (e != cudaSuccess) return cuda_fail(e, "image transform launch");
    }
    return IDG_OK;
}

}  // extern "C"
