// Classical gridding with oversampled A/W-projection kernels (idg_classical_grid).
//
// This is the gridding the paper sets image domain gridding against (Sect. 2:
// a convolution kernel per visibility, precomputed on an oversampled grid as the
// Fourier transform of its zero-padded image-domain window; W-projection and
// A-projection put the w-term and the station beams into that window).  It runs
// on the same plan, visibilities and grid layout as the library's gridder:
//
//   window of subgrid p (baseline (p, q), A-term slot a) and W-projection plane j,
//   on the M x M lattice l_x = (x - M/2) S / M, as a 4 x 4 operator on the
//   polarisations (vec X = XX, XY, YX, YY) of X -> b e^{2 pi i w_j n'} A_p^H X A_q:
//       c[(i, j), (a, b)] = b e^{2 pi i w_j n'} conj(A_p[a][i]) A_q[b][j],  w_j = j dw
//   kernel  C(dv, du) = M^-2 sum_{y,x} c[y][x] e^{-2 pi i (du (x - M/2) + dv (y - M/2)) / M}
//   tabulated at du, dv = d - M/2 + 1 - o/O (support index d, phase o < O);
//   visibility k: pu = (u f/c) S + N/2, support floor(pu) - M/2 + 1 .. floor(pu) + M/2,
//   phase o = floor(frac(pu) O + 1/2) (o = O moves the support one pixel on),
//   plane j = floor((w f/c - w0) / dw + 1/2) (0 without W-projection);
//   grid[layer][r][q] += C . y_k, support pixels outside the grid dropped.
//
// Kernels are rebuilt per subgrid -- so per A-term slot, every slot -- which is
// the cost the paper's method removes.  Two kernels per chunk of subgrids:
//   classical_kernels_kernel  one CTA per (subgrid, plane): the window in shared
//       memory, then the zero-padded transform as two small DFT stages (along x
//       into a scratch tile, along y into the table) with exact integer argument
//       reduction of the twiddles (indices advanced by additions); table
//       [O][O][M][M][16] complex64 in HBM, each (phase, pixel) a contiguous row.
//   classical_grid_kernel     one CTA per subgrid: its visibilities' kernel blocks
//       (M^2 x 16 complex, contiguous per phase) applied into a shared-memory tile
//       that covers the subgrid box plus the support margin, flushed to the grid
//       with vector atomics.
// Coordinates, phases and planes are formed in FP64 with explicitly rounded
// operations (no contraction), so the phase and plane choice is the one a host
// computes with the same formulas.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "idg_internal.h"

namespace idg {

// device error word of the classical gridder (0 = ok; 2 = a visibility's support
// fell outside its subgrid's tile, which a valid plan rules out; it was skipped)
__device__ int g_classical_error = 0;

namespace {

constexpr int kKThreads = 256;
constexpr size_t kClassicalSetMax = size_t(256) << 20;        // bytes of one kernel (subgrid, plane)
constexpr size_t kClassicalTableBudget = size_t(2) << 30;    // bytes of kernels per chunk
constexpr int kGThreads = 256;
constexpr int kVisBatch = 64;

struct ClassicalArgs {
    int M, O;
    double dw;              // W-projection plane spacing (0: no w-term)
    const float *taper;     // [M][M]
    const float4 *aterms;   // [n_slots][n_st][M][M][2 float4] or null (identity)
    const double *nprime;   // [M][M] n' of the kernel lattice
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// twiddle index (n (v - M/2)) mod MO of v = 0, advanced by n mod MO per step of v
__device__ __forceinline__ int tw_start(int n, int M, int MO) {
    int k = (n * (-M / 2)) % MO;
    return k < 0 ? k + MO : k;
}
__device__ __forceinline__ int tw_step(int n, int MO) {
    int k = n % MO;
    return k < 0 ? k + MO : k;
}

// One CTA per (subgrid, plane): sets[k] = (plan index, plane j).  Output table k at
// tables + k * O^2 M^2 16.  The Mueller entries go EG at a time (all 16 for M <= 16),
// so that each output (phase, support pixel) leaves as EG contiguous complex values.
template <int EG>
__global__ void __launch_bounds__(kKThreads) classical_kernels_kernel(Geometry g, ClassicalArgs a,
                                                                      const int2 *__restrict__ sets,
                                                                      float2 *__restrict__ tables) {
    extern __shared__ float2 sm[];
    const int M = a.M, O = a.O, MM = M * M, MO = M * O;
    float2 *win = sm;               // [EG][M][M]  current group of Mueller entries
    float2 *tx = win + EG * MM;     // [EG][M][M]  x-transformed rows for one phase ox
    float2 *tw = tx + EG * MM;      // [MO]        e^{-2 pi i k / (M O)}
    const int2 sj = sets[blockIdx.x];
    const DevSubgrid d = g.sub[sj.x];
    const double wj = (double)sj.y * a.dw;
    for (int k = threadIdx.x; k < MO; k += kKThreads) {
        float s, c;
        sincospif(-2.0f * (float)k / (float)MO, &s, &c);
        tw[k] = make_float2(c, s);
    }
    float2 *out = tables + (size_t)blockIdx.x * O * O * MM * 16;
    const float norm = 1.0f / (float)MM;
    for (int e0 = 0; e0 < 16; e0 += EG) {
        __syncthreads();
        // window entries e = e0 .. e0 + EG - 1: output polarisation i j = e / 4, input a b = e % 4
        for (int t = threadIdx.x; t < EG * MM; t += kKThreads) {
            const int e = e0 + t / MM, pix = t % MM;
            const int pi = e >> 3, pj = (e >> 2) & 1, qa = (e >> 1) & 1, qb = e & 1;
            float2 ap = make_float2(qa == pi ? 1.f : 0.f, 0.f), aq = make_float2(qb == pj ? 1.f : 0.f, 0.f);
            if (a.aterms) {
                const float2 *P = (const float2 *)(a.aterms + (((size_t)d.slot * g.n_stations + d.st_p) * MM + pix) * 2);
                const float2 *Q = (const float2 *)(a.aterms + (((size_t)d.slot * g.n_stations + d.st_q) * MM + pix) * 2);
                ap = P[2 * qa + pi];
                aq = Q[2 * qb + pj];
            }
            float2 ph = make_float2(1.f, 0.f);
            if (a.dw > 0.0) {
                double turns = wj * a.nprime[pix];
                turns -= rint(turns);
                float s, c;
                sincospif(2.0f * (float)turns, &s, &c);
                ph = make_float2(c, s);
            }
            const float2 v = cmulf(cmulf(ph, make_float2(ap.x, -ap.y)), aq);
            const float tb = a.taper[pix];
            win[t] = make_float2(tb * v.x, tb * v.y);
        }
        for (int ox = 0; ox < O; ++ox) {
            __syncthreads();
            // along x: tx[e][y][dx] = sum_x win[e][y][x] e^{-2 pi i n (x - M/2) / (M O)},
            // n = O (dx - M/2 + 1) - ox
            for (int t = threadIdx.x; t < EG * MM; t += kKThreads) {
                const int e = t / MM, y = (t / M) % M, dx = t % M;
                const int n = O * (dx - M / 2 + 1) - ox;
                int k = tw_start(n, M, MO);
                const int dk = tw_step(n, MO);
                float2 acc = make_float2(0.f, 0.f);
                const float2 *wr = win + (e * M + y) * M;
                for (int x = 0; x < M; ++x) {
                    const float2 c = wr[x], w = tw[k];
                    acc.x += c.x * w.x - c.y * w.y;
                    acc.y += c.x * w.y + c.y * w.x;
                    k += dk;
                    k -= k >= MO ? MO : 0;
                }
                tx[t] = acc;
            }
            __syncthreads();
            // along y, every phase oy: table[oy][ox][dy][dx][e0 ..].  A thread takes 4 phases x
            // 4 entries of one support pixel, so each window value and twiddle it loads from
            // shared memory serves 4 multiply-adds (the loop is then bound by the FMA pipe)
            const int n_o4 = (O + 3) / 4;              // phase quads (the last one partial when 4 does not divide O)
            for (int t = threadIdx.x; t < n_o4 * MM * (EG / 4); t += kKThreads) {
                const int e4 = t % (EG / 4), pix = (t / (EG / 4)) % MM, o4 = t / ((EG / 4) * MM);
                const int dy = pix / M, dx = pix % M;
                int k[4], dk[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int n = O * (dy - M / 2 + 1) - (4 * o4 + a);
                    k[a] = tw_start(n, M, MO);
                    dk[a] = tw_step(n, MO);
                }
                float2 acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[a][e] = make_float2(0.f, 0.f);
                for (int y = 0; y < M; ++y) {
                    float2 c[4], w[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) c[e] = tx[((4 * e4 + e) * M + y) * M + dx];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        w[a] = tw[k[a]];
                        k[a] += dk[a];
                        k[a] -= k[a] >= MO ? MO : 0;
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            acc[a][e].x += c[e].x * w[a].x - c[e].y * w[a].y;
                            acc[a][e].y += c[e].x * w[a].y + c[e].y * w[a].x;
                        }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int oy = 4 * o4 + a;
                    if (oy >= O) break;
                    float4 *dst = (float4 *)(out + ((((size_t)oy * O + ox) * MM + pix) * 16 + e0 + 4 * e4));
                    dst[0] = make_float4(norm * acc[a][0].x, norm * acc[a][0].y, norm * acc[a][1].x, norm * acc[a][1].y);
                    dst[1] = make_float4(norm * acc[a][2].x, norm * acc[a][2].y, norm * acc[a][3].x, norm * acc[a][3].y);
                }
            }
        }
    }
}

// support start and oversampled phase of one coordinate (FP64, each operation rounded)
__device__ __forceinline__ void position(double um, double s, double S, int N, int O, int &iq, int &o) {
    const double pu = __dadd_rn(__dmul_rn(__dmul_rn(um, s), S), 0.5 * (double)N);
    const double fl = floor(pu);
    int oo = (int)floor(__dadd_rn(__dmul_rn(__dsub_rn(pu, fl), (double)O), 0.5));
    int i = (int)fl;
    if (oo == O) {
        ++i;
        oo = 0;
    }
    iq = i;
    o = oo;
}

__device__ __forceinline__ int plane_of(double wm, double s, double w0, double dw) {
    if (!(dw > 0.0)) return 0;
    return (int)floor(__dadd_rn(__ddiv_rn(__dsub_rn(__dmul_rn(wm, s), w0), dw), 0.5));
}

// per subgrid: smallest and largest W-projection plane of its visibilities
__global__ void __launch_bounds__(256) classical_planes_kernel(Geometry g, double dw, int2 *__restrict__ range) {
    const DevSubgrid d = g.sub[blockIdx.x];
    int lo = 0x7FFFFFFF, hi = -0x7FFFFFFF;
    for (int i = threadIdx.x; i < d.nt * d.nc; i += 256) {
        const int t = d.t0 + i / d.nc, c = d.c0 + i % d.nc;
        const int j = plane_of(g.uvw[((size_t)d.bl * g.n_t + t) * 3 + 2], g.scale[c], d.w0, dw);
        lo = min(lo, j);
        hi = max(hi, j);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ int s_lo[8], s_hi[8];
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
        }
        range[blockIdx.x] = make_int2(d.nt * d.nc > 0 ? lo : 0, d.nt * d.nc > 0 ? hi : 0);
    }
}

// One CTA per subgrid of the chunk: work[b] = (plan index, first table of its
// planes - chunk's first table), jmin[b] its lowest plane.
__global__ void __launch_bounds__(kGThreads) classical_grid_kernel(Geometry g, ClassicalArgs a,
                                                                   const int2 *__restrict__ work,
                                                                   const int *__restrict__ jmin,
                                                                   const float2 *__restrict__ tables,
                                                                   const float4 *__restrict__ vis,
                                                                   const uint8_t *__restrict__ flags,
                                                                   float4 *__restrict__ grid) {
    extern __shared__ float sm_f[];
    const int M = a.M, O = a.O, MM = M * M;
    const int T = g.L + M + 3;                      // tile side: subgrid box, support margin, one spare pixel
    float *tile = sm_f;                             // [T][T][8] (4 polarisations, re/im)
    float2 *yv = (float2 *)(tile + (size_t)T * T * 8);   // [kVisBatch][4]
    int4 *info = (int4 *)(yv + 4 * kVisBatch);            // [kVisBatch]: tile row, tile col, block offset / 16, valid
    const int2 wk = work[blockIdx.x];
    const DevSubgrid d = g.sub[wk.x];
    for (int i = threadIdx.x; i < T * T * 8; i += kGThreads) tile[i] = 0.f;
    const int row0 = d.r0 - M / 2 - 1, col0 = d.q0 - M / 2 - 1;  // grid position of tile (0, 0)
    const size_t set_elems = (size_t)O * O * MM * 16;
    const int n = d.nt * d.nc;
    for (int b0 = 0; b0 < n; b0 += kVisBatch) {
        __syncthreads();
        if (threadIdx.x < kVisBatch) {
            const int i = b0 + threadIdx.x;
            int4 inf = make_int4(0, 0, 0, 0);
            if (i < n) {
                const int t = d.t0 + i / d.nc, c = d.c0 + i % d.nc;
                const size_t v = ((size_t)d.bl * g.n_t + t) * g.n_chan + c;
                if (!(flags && flags[v])) {
                    const double *uvw = g.uvw + ((size_t)d.bl * g.n_t + t) * 3;
                    const double s = g.scale[c];
                    int iq, ox, ir, oy;
                    position(uvw[0], s, g.S, g.N, O, iq, ox);
                    position(uvw[1], s, g.S, g.N, O, ir, oy);
                    const int j = plane_of(uvw[2], s, d.w0, a.dw);
                    const size_t off = (size_t)(wk.y + j - jmin[blockIdx.x]) * set_elems +
                                       ((size_t)oy * O + ox) * MM * 16;
                    inf = make_int4(ir - M / 2 + 1 - row0, iq - M / 2 + 1 - col0, (int)(off >> 4), 1);
                    // the plan keeps every sample within (L - beta + 1)/2 of the centre, so the
                    // support lies inside the tile; anything else is skipped and reported
                    if (inf.x < 0 || inf.x > T - M || inf.y < 0 || inf.y > T - M) {
                        inf.w = 0;
                        atomicOr(&g_classical_error, 2);
                    }
                    const float4 v0 = vis[2 * v], v1 = vis[2 * v + 1];
                    yv[4 * threadIdx.x + 0] = make_float2(v0.x, v0.y);
                    yv[4 * threadIdx.x + 1] = make_float2(v0.z, v0.w);
                    yv[4 * threadIdx.x + 2] = make_float2(v1.x, v1.y);
                    yv[4 * threadIdx.x + 3] = make_float2(v1.z, v1.w);
                }
            }
            info[threadIdx.x] = inf;
        }
        __syncthreads();
        const int nb = min(kVisBatch, n - b0);
        for (int k = 0; k < nb; ++k) {
            const int4 inf = info[k];
            if (!inf.w) continue;
            const float4 *blk = (const float4 *)(tables + ((size_t)inf.z << 4));
            const float2 y0 = yv[4 * k], y1 = yv[4 * k + 1], y2 = yv[4 * k + 2], y3 = yv[4 * k + 3];
            for (int item = threadIdx.x; item < MM * 4; item += kGThreads) {
                // item = (dy M + dx) 4 + output polarisation: its 4 kernel entries are contiguous
                const float4 k01 = blk[2 * item], k23 = blk[2 * item + 1];
                float re = k01.x * y0.x - k01.y * y0.y + k01.z * y1.x - k01.w * y1.y + k23.x * y2.x - k23.y * y2.y +
                           k23.z * y3.x - k23.w * y3.y;
                float im = k01.x * y0.y + k01.y * y0.x + k01.z * y1.y + k01.w * y1.x + k23.x * y2.y + k23.y * y2.x +
                           k23.z * y3.y + k23.w * y3.x;
                const int pix = item >> 2, pol = item & 3;
                const int tr = inf.x + pix / M, tc = inf.y + pix % M;
                float *dst = tile + ((size_t)tr * T + tc) * 8 + 2 * pol;
                atomicAdd(dst, re);
                atomicAdd(dst + 1, im);
            }
        }
    }
    __syncthreads();
    float4 *gl = grid + (size_t)d.layer * g.N * g.N * 2;
    for (int i = threadIdx.x; i < T * T * 2; i += kGThreads) {
        const int px = i >> 1, half = i & 1;
        const int r = row0 + px / T, q = col0 + px % T;
        if (r < 0 || r >= g.N || q < 0 || q >= g.N) continue;
        const float *s = tile + (size_t)px * 8 + 4 * half;
        if (s[0] == 0.f && s[1] == 0.f && s[2] == 0.f && s[3] == 0.f) continue;
        atomicAdd(gl + ((size_t)r * g.N + q) * 2 + half, make_float4(s[0], s[1], s[2], s[3]));
    }
}

}  // namespace

// Mueller entries per pass of the kernel builder: all 16 while the window and the
// x-transformed tile fit comfortably, else 4
int classical_entry_group(int M) { return M <= 16 ? 16 : 4; }
size_t classical_kernels_smem(int M, int O) {
    return (size_t)(2 * classical_entry_group(M) * M * M + M * O) * sizeof(float2);
}
size_t classical_grid_smem(int L, int M) {
    const size_t T = (size_t)(L + M + 3);
    return T * T * 8 * sizeof(float) + 4 * kVisBatch * sizeof(float2) + kVisBatch * sizeof(int4);
}

idg_status launch_classical_planes(const Geometry &g, int64_t n_sub, double dw, int2 *range, void *stream) {
    if (n_sub <= 0) return IDG_OK;
    classical_planes_kernel<<<(unsigned)n_sub, 256, 0, (cudaStream_t)stream>>>(g, dw, range);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "classical plane-range launch");
}

idg_status read_classical_error(int *code) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(code, g_classical_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_classical_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the classical gridder's error word");
    return IDG_OK;
}

idg_status launch_classical_kernels(const Geometry &g, int M, int O, double dw, const float *taper,
                                    const void *aterms, const double *nprime, const int2 *sets, int64_t n_sets,
                                    void *tables, void *stream) {
    if (n_sets <= 0) return IDG_OK;
    const ClassicalArgs a{M, O, dw, taper, (const float4 *)aterms, nprime};
    const size_t smem = classical_kernels_smem(M, O);
    const bool all16 = classical_entry_group(M) == 16;
    cudaError_t e = all16 ? cudaFuncSetAttribute(classical_kernels_kernel<16>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaFuncSetAttribute(classical_kernels_kernel<4>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "classical kernels: shared memory attribute");
    if (all16)
        classical_kernels_kernel<16><<<(unsigned)n_sets, kKThreads, smem, (cudaStream_t)stream>>>(g, a, sets,
                                                                                              (float2 *)tables);
    else
        classical_kernels_kernel<4><<<(unsigned)n_sets, kKThreads, smem, (cudaStream_t)stream>>>(g, a, sets,
                                                                                             (float2 *)tables);
    e = cudaGetLastError();
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "classical kernels launch");
}

idg_status launch_classical_grid(const Geometry &g, int M, int O, double dw, const int2 *work, const int *jmin,
                                 int64_t count, const void *tables, const void *vis, const uint8_t *flags,
                                 void *grid, void *stream) {
    if (count <= 0) return IDG_OK;
    const ClassicalArgs a{M, O, dw, nullptr, nullptr, nullptr};
    const size_t smem = classical_grid_smem(g.L, M);
    cudaError_t e = cudaFuncSetAttribute(classical_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "classical gridder: shared memory attribute");
    classical_grid_kernel<<<(unsigned)count, kGThreads, smem, (cudaStream_t)stream>>>(
        g, a, work, jmin, (const float2 *)tables, (const float4 *)vis, flags, (float4 *)grid);
    e = cudaGetLastError();
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "classical gridder launch");
}

}  // namespace idg

using namespace idg;

extern "C" idg_status idg_classical_grid(const idg_plan *p, int M, int O, double dw, const void *vis,
                                         const uint8_t *flags, const void *aterms, const float *taper, void *grid,
                                         idg_stream stream) {
    if (!p) return fail(IDG_ERR_INVALID_ARG, "plan is NULL");
    if (!vis) return fail(IDG_ERR_INVALID_ARG, "d_vis is NULL");
    if (!grid) return fail(IDG_ERR_INVALID_ARG, "d_grid is NULL");
    if (M < 2 || M > 32 || M % 2) return fail(IDG_ERR_INVALID_ARG, "support must be even, 2 .. 32");
    if (O < 1 || O > 128) return fail(IDG_ERR_INVALID_ARG, "oversample must be 1 .. 128");
    if (!(dw >= 0.0) || !std::isfinite(dw)) return fail(IDG_ERR_INVALID_ARG, "w_plane_step must be >= 0");
    const size_t set_elems = (size_t)O * O * M * M * 16;
    if (set_elems * 8 > kClassicalSetMax)
        return fail(IDG_ERR_INVALID_ARG, "oversample^2 * support^2 * 128 bytes (one kernel) exceeds 256 MiB");
    if (classical_grid_smem(p->L, M) > 200 * 1024)
        return fail(IDG_ERR_UNSUPPORTED, "subgrid size + support too large for the shared-memory tile");
    if (p->device < 0) return fail(IDG_ERR_INVALID_ARG, "the plan was created without a CUDA device");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(IDG_ERR_INVALID_ARG, "the plan belongs to another device");
    const int64_t n = p->stats.n_subgrids;
    if (n == 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const Geometry g = p->geometry();
    // the window b on the kernel lattice (default: the PSWF of width M) and n' there
    std::vector<float> tap_h;
    if (!taper) {
        std::vector<double> a1((size_t)M);
        idg_status st = idg_taper_window(M, (double)M, IDG_TAPER_PSWF, a1.data(), nullptr);
        if (st != IDG_OK) return st;
        tap_h.resize((size_t)M * M);
        for (int y = 0; y < M; ++y)
            for (int x = 0; x < M; ++x) tap_h[(size_t)y * M + x] = (float)(a1[y] * a1[x]);
    }
    std::vector<double> n1((size_t)M * M);
    for (int y = 0; y < M; ++y)
        for (int x = 0; x < M; ++x) {
            const double l = ((double)x - 0.5 * M) * p->S / M, m = ((double)y - 0.5 * M) * p->S / M;
            n1[(size_t)y * M + x] = std::sqrt(1.0 - l * l - m * m) - 1.0;
        }
    // W-projection planes of every subgrid (one small launch and a copy back)
    std::vector<int2> range((size_t)n, make_int2(0, 0));
    void *small = nullptr;
    const size_t small_bytes = (size_t)M * M * (sizeof(double) + sizeof(float)) + (size_t)n * sizeof(int2);
    idg_status st = scratch_alloc(p->device, small_bytes, s, &small);
    if (st != IDG_OK) return st;
    double *d_n1 = (double *)small;
    float *d_tap = (float *)(d_n1 + (size_t)M * M);
    int2 *d_range = (int2 *)(d_tap + (size_t)M * M);
    e = cudaMemcpyAsync(d_n1, n1.data(), n1.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !taper)
        e = cudaMemcpyAsync(d_tap, tap_h.data(), tap_h.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "classical gridder set-up copies");
    if (st == IDG_OK && dw > 0.0) {
        st = launch_classical_planes(g, n, dw, d_range, s);
        if (st == IDG_OK) {
            e = cudaMemcpyAsync(range.data(), d_range, (size_t)n * sizeof(int2), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "classical gridder: plane ranges");
        }
    }
    const float *tap = taper ? taper : d_tap;
    // chunks of subgrids (work order) whose kernels fit the table budget
    int64_t max_sets = 0;
    for (int64_t i = 0; i < n; ++i) max_sets = std::max<int64_t>(max_sets, range[i].y - range[i].x + 1);
    if (st == IDG_OK && (size_t)max_sets * set_elems * 8 > 8 * kClassicalTableBudget)
        st = fail(IDG_ERR_INVALID_ARG, "a subgrid spans " + std::to_string(max_sets) +
                                           " W-projection planes, whose kernels exceed 16 GiB: raise w_plane_step");
    const int64_t budget_sets = std::max<int64_t>(max_sets, (int64_t)(kClassicalTableBudget / (set_elems * 8)));
    void *tables = nullptr, *meta = nullptr;
    if (st == IDG_OK) st = scratch_alloc(p->device, (size_t)budget_sets * set_elems * 8, s, &tables);
    const int64_t max_chunk = std::min<int64_t>(n, budget_sets);
    if (st == IDG_OK)
        st = scratch_alloc(p->device, (size_t)budget_sets * sizeof(int2) + (size_t)max_chunk * (sizeof(int2) + sizeof(int)),
                           s, &meta);
    std::vector<int2> sets, work;
    std::vector<int> jmin;
    for (int64_t f = 0; f < n && st == IDG_OK;) {
        sets.clear();
        work.clear();
        jmin.clear();
        int64_t i = f;
        while (i < n) {
            const int sid = p->order[i];
            const int cnt = range[sid].y - range[sid].x + 1;
            if ((int64_t)sets.size() + cnt > budget_sets) break;
            work.push_back(make_int2(sid, (int)sets.size()));
            jmin.push_back(range[sid].x);
            for (int j = range[sid].x; j <= range[sid].y; ++j) sets.push_back(make_int2(sid, j));
            ++i;
        }
        int2 *d_sets = (int2 *)meta;
        int2 *d_work = d_sets + budget_sets;
        int *d_jmin = (int *)(d_work + max_chunk);
        e = cudaMemcpyAsync(d_sets, sets.data(), sets.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_jmin, jmin.data(), jmin.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "classical gridder: chunk tables");
            break;
        }
        {
            ProfileScope ps(IDG_KERNEL_CLASSICAL_KERNELS, s, (double)sets.size() * set_elems * 8);
            st = launch_classical_kernels(g, M, O, dw, tap, aterms, d_n1, d_sets, (int64_t)sets.size(), tables, s);
        }
        if (st == IDG_OK) {
            double nv = 0.0;
            for (int64_t k = f; k < i; ++k) nv += (double)p->kp_order[k];
            ProfileScope ps(IDG_KERNEL_CLASSICAL_GRID, s, nv * M * M);
            st = launch_classical_grid(g, M, O, dw, d_work, d_jmin, (int64_t)work.size(), tables, vis, flags, grid, s);
        }
        f = i;
    }
    if (meta) cudaFreeAsync(meta, s);
    if (tables) cudaFreeAsync(tables, s);
    cudaFreeAsync(small, s);
    return st;
}
