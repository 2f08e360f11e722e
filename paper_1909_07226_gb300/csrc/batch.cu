// Batched form: many independent jobs (one plan each) processed together.
//
// All subgrids of all jobs that share a subgrid size L form one work list,
// ordered by cost (K_p, largest first).  One persistent launch per L (a few
// CTAs per SM) pulls work items from a device counter; each item is a whole
// subgrid pipeline inside one CTA, the subgrid never leaving shared memory:
//   gridding    direct sum -> taper and A-terms -> FFT -> atomic add to the grid
//   degridding  split from the grid -> IFFT -> taper and A-terms -> degrid sum
// (Algorithms 1 and 2 per block p).  No subgrid scratch in device memory.
// The launch sequence (counter resets, the persistent launches, zeroing of
// dropped visibilities) can be captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "degridder_impl.cuh"
#include "batch_jobs.cuh"
#include "fft_impl.cuh"
#include "gridder_impl.cuh"

namespace idg {

namespace {

using namespace dev;

// ---------------------------------------------------------------------------
// gridding: direct sum (packed f32x2 form) + epilogue + FFT + adder in one CTA

template <int L, int NPX, int VB, int MINB>
__global__ void __launch_bounds__(L * L / NPX, MINB)
batch_grid_kernel(const JobDev *__restrict__ jobs, const int2 *__restrict__ items, int n_items,
                  int *__restrict__ counter) {
    constexpr int NT = L * L / NPX;
    constexpr int TPR = L / NPX;
    constexpr int P = L + 1;
    __shared__ float4 s_coef[VB];
    __shared__ float4 s_v01[VB];
    __shared__ float4 s_v23[VB];
    __shared__ float4 s_iv01[VB];
    __shared__ float4 s_iv23[VB];
    __shared__ int s_item;
    extern __shared__ float2 s_fft[];   // [4][L][L + 1]

    const int tid = threadIdx.x;
    const int y = tid / TPR;
    const int x0 = (tid % TPR) * NPX;
    const float Y = (float)(y - L / 2);
    const float inv = 1.0f / (float)(L * L);
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 w = items[it];
        const JobDev *J = jobs + w.x;
        const Geometry g = J->g;
        const DevSubgrid d = g.sub[w.y];
        const float4 *vis = J->vis;
        const uint8_t *flags = J->flags;
        float X[NPX], NP[NPX];
#pragma unroll
        for (int j = 0; j < NPX; ++j) {
            X[j] = (float)(x0 + j - L / 2);
            NP[j] = g.nprime[y * L + x0 + j];
        }
        f2_t acc[NPX][4];
#pragma unroll
        for (int j = 0; j < NPX; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = f2_pack(0.0f, 0.0f);
        for (int k0 = 0; k0 < d.kp; k0 += VB) {
            const int nb = min(VB, d.kp - k0);
            for (int i = tid; i < nb; i += NT) {
                RawVis r;
                fetch_raw(g, d, k0 + i, vis, flags, r);
                store_raw(g, d, r, s_coef, s_v01, s_v23, i);
                const float4 a = s_v01[i], b = s_v23[i];
                s_iv01[i] = make_float4(-a.y, a.x, -a.w, a.z);
                s_iv23[i] = make_float4(-b.y, b.x, -b.w, b.z);
            }
            __syncthreads();
            sum_batch_f2<NPX>(s_coef, s_v01, s_v23, s_iv01, s_iv23, nb, Y, X, NP, acc);
            __syncthreads();
        }
        // taper * A_p^H . I . A_q, with the (-1)^(x+y) centring factor, into the FFT planes
#pragma unroll
        for (int j = 0; j < NPX; ++j) {
            const int x = x0 + j;
            const int pix = y * L + x;
            M22 Pm;
            f2_unpack(acc[j][0], Pm.m[0].x, Pm.m[0].y);
            f2_unpack(acc[j][1], Pm.m[1].x, Pm.m[1].y);
            f2_unpack(acc[j][2], Pm.m[2].x, Pm.m[2].y);
            f2_unpack(acc[j][3], Pm.m[3].x, Pm.m[3].y);
            if (J->aterms) {
                const size_t base = ((size_t)d.slot * g.n_stations) * L * L;
                const M22 Ap = load_m22(J->aterms + 2 * (base + (size_t)d.st_p * L * L + pix));
                const M22 Aq = load_m22(J->aterms + 2 * (base + (size_t)d.st_q * L * L + pix));
                Pm = herm_mul_mul(Ap, Pm, Aq);
            }
            const float tw = ((x + y) & 1) ? -J->taper[pix] : J->taper[pix];
#pragma unroll
            for (int q = 0; q < 4; ++q) s_fft[(q * L + y) * P + x] = make_float2(tw * Pm.m[q].x, tw * Pm.m[q].y);
        }
        __syncthreads();
        fft2_planar<L, -1>(s_fft, tid, NT);
        // adder with the (-1)^(i+j) factor and 1/L^2
        float4 *dst = J->grid + (size_t)d.layer * g.N * g.N * 2;
        for (int pix = tid; pix < L * L; pix += NT) {
            const int i = pix / L, j = pix - (pix / L) * L;
            const float sg = ((i + j) & 1) ? -inv : inv;
            const float2 p0 = s_fft[(0 * L + i) * P + j], p1 = s_fft[(1 * L + i) * P + j];
            const float2 p2 = s_fft[(2 * L + i) * P + j], p3 = s_fft[(3 * L + i) * P + j];
            const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
            red_add_f4(dst + 2 * gp, make_float4(sg * p0.x, sg * p0.y, sg * p1.x, sg * p1.y));
            red_add_f4(dst + 2 * gp + 1, make_float4(sg * p2.x, sg * p2.y, sg * p3.x, sg * p3.y));
        }
        __syncthreads();
    }
}

// degrid sum of one subgrid from the packed shared-memory image, PGS pixel
// groups per warp (fixed), NV visibilities per lane
template <int L, int NV, int PGS, int NT>
__device__ __forceinline__ void degrid_sum_f2(const Geometry &g, const DevSubgrid &d, const JobDev *J,
                                              const float4 *s_p01, const float4 *s_p23, const float4 *s_q01,
                                              const float4 *s_q23, const float *s_np, int tid) {
    const int lane = tid & 31, warp = tid >> 5;
    const int grp = lane % PGS;
    const int vlane = warp * (32 / PGS) + lane / PGS;
    constexpr int per_pass = (NT / PGS) * NV;
    for (int kb = 0; kb < d.kp; kb += per_pass) {
        float ca[NV], cb[NV], cc[NV];
        degrid_coefs<NV>(g, d, kb + vlane * NV, ca, cb, cc);
        f2_t acc[NV][4];
#pragma unroll
        for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = f2_pack(0.0f, 0.0f);
        for (int yy = 0; yy < L; ++yy) {
            const float Yf = (float)(yy - L / 2);
            float bY[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) bY[j] = cb[j] * Yf;
            const int row = yy * L + grp;
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
        if (grp == 0) degrid_write<NV>(g, d, kb + vlane * NV, J->flags, facc, J->vis_out);
    }
}

// ---------------------------------------------------------------------------
// degridding: splitter + IFFT + image-domain kernel + degrid sum in one CTA

template <int L, int NV, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
batch_degrid_kernel(const JobDev *__restrict__ jobs, const int2 *__restrict__ items, int n_items,
                    int *__restrict__ counter) {
    constexpr int P = L + 1;
    extern __shared__ float4 smem[];
    float2 *s_fft = (float2 *)smem;                                  // [4][L][L + 1]
    float4 *s_p01 = smem + (4 * L * P) / 2;                          // [L*L]
    float4 *s_p23 = s_p01 + L * L;
    float4 *s_q01 = s_p23 + L * L;
    float4 *s_q23 = s_q01 + L * L;
    float *s_np = (float *)(s_q23 + L * L);
    __shared__ int s_item;

    const int tid = threadIdx.x;
    const float inv = 1.0f / (float)(L * L);
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 w = items[it];
        const JobDev *J = jobs + w.x;
        const Geometry g = J->g;
        const DevSubgrid d = g.sub[w.y];
        // splitter with the (-1)^(i+j) pre-factor
        const float4 *src = J->grid + (size_t)d.layer * g.N * g.N * 2;
        for (int pix = tid; pix < L * L; pix += NT) {
            const int i = pix / L, j = pix - (pix / L) * L;
            const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
            const float sg = ((i + j) & 1) ? -1.0f : 1.0f;
            const float4 a = src[2 * gp], b = src[2 * gp + 1];
            s_fft[(0 * L + i) * P + j] = make_float2(sg * a.x, sg * a.y);
            s_fft[(1 * L + i) * P + j] = make_float2(sg * a.z, sg * a.w);
            s_fft[(2 * L + i) * P + j] = make_float2(sg * b.x, sg * b.y);
            s_fft[(3 * L + i) * P + j] = make_float2(sg * b.z, sg * b.w);
        }
        __syncthreads();
        fft2_planar<L, +1>(s_fft, tid, NT);
        // (-1)^(x+y) / L^2, taper * A_p . I . A_q^H, packed layout for the sum
        for (int pix = tid; pix < L * L; pix += NT) {
            const int y = pix / L, x = pix - (pix / L) * L;
            const float sg = ((x + y) & 1) ? -inv : inv;
            M22 Pm;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = s_fft[(q * L + y) * P + x];
                Pm.m[q] = make_float2(sg * v.x, sg * v.y);
            }
            if (J->aterms) {
                const size_t base = ((size_t)d.slot * g.n_stations) * L * L;
                const M22 Ap = load_m22(J->aterms + 2 * (base + (size_t)d.st_p * L * L + pix));
                const M22 Aq = load_m22(J->aterms + 2 * (base + (size_t)d.st_q * L * L + pix));
                Pm = mul_mul_herm(Ap, Pm, Aq);
            }
            const float tw = J->taper[pix];
            s_p01[pix] = make_float4(tw * Pm.m[0].x, tw * Pm.m[0].y, tw * Pm.m[1].x, tw * Pm.m[1].y);
            s_p23[pix] = make_float4(tw * Pm.m[2].x, tw * Pm.m[2].y, tw * Pm.m[3].x, tw * Pm.m[3].y);
            s_q01[pix] = make_float4(tw * Pm.m[0].y, -tw * Pm.m[0].x, tw * Pm.m[1].y, -tw * Pm.m[1].x);
            s_q23[pix] = make_float4(tw * Pm.m[2].y, -tw * Pm.m[2].x, tw * Pm.m[3].y, -tw * Pm.m[3].x);
            s_np[pix] = g.nprime[pix];
        }
        __syncthreads();
        // degrid sum (packed form); the pixel groups per warp follow from K_p and
        // select a copy of the sum with the column loop unrolled for that split
        switch (degrid_pg(d.kp, NT, NV)) {
        case 1: degrid_sum_f2<L, NV, 1, NT>(g, d, J, s_p01, s_p23, s_q01, s_q23, s_np, tid); break;
        case 2: degrid_sum_f2<L, NV, 2, NT>(g, d, J, s_p01, s_p23, s_q01, s_q23, s_np, tid); break;
        case 4: degrid_sum_f2<L, NV, 4, NT>(g, d, J, s_p01, s_p23, s_q01, s_q23, s_np, tid); break;
        default: degrid_sum_f2<L, NV, 8, NT>(g, d, J, s_p01, s_p23, s_q01, s_q23, s_np, tid); break;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// per-L dispatch

template <int L>
size_t grid_smem() { return sizeof(float2) * 4 * L * (L + 1); }

template <int L>
size_t degrid_smem() {
    return sizeof(float2) * 4 * L * (L + 1) + (size_t)L * L * (4 * sizeof(float4) + sizeof(float));
}

struct KernelShape {
    const char *name;
    const void *fn;      // persistent fused kernel, or null for the tensor-core path
    int threads;
    size_t smem;
    bool tc = false;     // tensor-core path: one CTA per work item instead of a persistent grid
};

// L = 32 on the tensor cores: the fused tensor-core gridder (degridder), one
// CTA per work item, with the transform in shared memory and the adder
// (splitter) in the same CTA
const KernelShape kTcShape = {"tcgen05_fused", nullptr, 288, 0, true};

template <int L, int NPX, int MINB>
KernelShape gshape(const char *name) {
    return {name, (const void *)batch_grid_kernel<L, NPX, 128, MINB>, L * L / NPX, grid_smem<L>()};
}

template <int L, int NV, int NT, int MINB>
KernelShape dshape(const char *name) {
    return {name, (const void *)batch_degrid_kernel<L, NV, NT, MINB>, NT, degrid_smem<L>()};
}

// compiled shapes per L (first = default)
std::vector<KernelShape> grid_shapes(int L) {
    switch (L) {
    case 8: return {gshape<8, 1, 4>("npx1_minb4"), gshape<8, 2, 6>("npx2_minb6")};
    case 16: return {gshape<16, 2, 2>("npx2_minb2"), gshape<16, 2, 4>("npx2_minb4"), gshape<16, 4, 4>("npx4_minb4")};
    case 24: return {gshape<24, 3, 2>("npx3_minb2"), gshape<24, 3, 3>("npx3_minb3"), gshape<24, 6, 4>("npx6_minb4")};
    case 32: return {kTcShape, gshape<32, 8, 4>("npx8_minb4"), gshape<32, 4, 3>("npx4_minb3"),
                     gshape<32, 4, 2>("npx4_minb2"), gshape<32, 2, 2>("npx2_minb2")};
    }
    return {};
}

std::vector<KernelShape> degrid_shapes(int L) {
    switch (L) {
    case 8: return {dshape<8, 4, 256, 2>("nv4_nt256_minb2"), dshape<8, 4, 128, 3>("nv4_nt128_minb3")};
    case 16: return {dshape<16, 4, 128, 3>("nv4_nt128_minb3"), dshape<16, 4, 256, 2>("nv4_nt256_minb2"),
                     dshape<16, 2, 256, 3>("nv2_nt256_minb3")};
    case 24: return {dshape<24, 4, 128, 3>("nv4_nt128_minb3"), dshape<24, 4, 256, 2>("nv4_nt256_minb2"),
                     dshape<24, 2, 256, 3>("nv2_nt256_minb3")};
    case 32: return {kTcShape, dshape<32, 4, 128, 2>("nv4_nt128_minb2"), dshape<32, 4, 128, 3>("nv4_nt128_minb3"),
                     dshape<32, 4, 256, 2>("nv4_nt256_minb2"), dshape<32, 2, 256, 3>("nv2_nt256_minb3")};
    }
    return {};
}

bool shapes_for(int L, KernelShape *g, KernelShape *dg) {
    auto gs = grid_shapes(L), ds = degrid_shapes(L);
    if (gs.empty() || ds.empty()) return false;
    int vg = get_variant(IDG_KERNEL_BATCH_GRID, L), vd = get_variant(IDG_KERNEL_BATCH_DEGRID, L);
    *g = gs[(vg >= 0 && vg < (int)gs.size()) ? vg : 0];
    *dg = ds[(vd >= 0 && vd < (int)ds.size()) ? vd : 0];
    return true;
}

}  // namespace
}  // namespace idg

using namespace idg;

struct idg_batch {
    struct Class {
        int L;
        bool sep = false;              // subgrids within the remainder bound (L = 32, 24, 16): the separable kernels
        int64_t n_items;
        double vispix;                 // sum of K_p L^2 of its items
        int2 *d_items = nullptr;
        // the tensor-core kernels: one launch per job over its entries d_idx[run_first[r] ..
        // run_first[r + 1]) (job run_job[r]), most visibilities first within the job
        int32_t *d_idx = nullptr;
        std::vector<int64_t> run_first;
        std::vector<int> run_job;
        KernelShape grid, degrid;
        int grid_blocks = 0, degrid_blocks = 0;
    };
    int device = -1;
    int n_jobs = 0;
    int flags = 0;
    int64_t n_vis = 0;                 // visibilities of all jobs (planned)
    JobDev *d_jobs = nullptr;
    std::vector<JobDev> host_jobs;     // the same on the host: the tensor-core launches' arguments
    int *d_counters = nullptr;         // one per class
    std::vector<Class> classes;
    std::vector<std::pair<void *, size_t>> zero_on_degrid;   // vis_out of jobs with dropped samples
    cudaGraphExec_t graph_grid = nullptr, graph_degrid = nullptr;
    cudaStream_t capture_stream = nullptr;   // private stream the graphs are recorded on
};

static idg_status batch_enqueue(idg_batch *b, bool degrid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->classes.size(), s);
    if (e != cudaSuccess) return cuda_fail(e, "batch counter reset");
    if (degrid)
        for (auto &z : b->zero_on_degrid) {
            e = cudaMemsetAsync(z.first, 0, z.second, s);
            if (e != cudaSuccess) return cuda_fail(e, "batch zeroing of dropped visibilities");
        }
    for (size_t c = 0; c < b->classes.size(); ++c) {
        auto &cl = b->classes[c];
        if (cl.n_items == 0) continue;
        const KernelShape &ks = degrid ? cl.degrid : cl.grid;
        if (ks.tc) {
            // one launch per job, its geometry as kernel arguments; every launch after the
            // first may begin while the one before finishes (the jobs' outputs are disjoint
            // or summed by atomic adds)
            ProfileScope ps(degrid ? IDG_KERNEL_BATCH_DEGRID : IDG_KERNEL_BATCH_GRID, s, cl.vispix);
            for (size_t r = 0; r + 1 < cl.run_first.size(); ++r) {
                const JobDev &J = b->host_jobs[cl.run_job[r]];
                const SubgridSet set{cl.d_idx + cl.run_first[r], 0, cl.run_first[r + 1] - cl.run_first[r], nullptr};
                const bool pdl = r > 0;
                const idg_status st =
                    cl.sep ? (degrid ? launch_degridder_sep_job(J.g, set, J.grid, J.flags, J.aterms, J.taper,
                                                                J.vis_out, s, pdl)
                                     : launch_gridder_sep_job(J.g, set, J.vis, J.flags, J.aterms, J.taper, J.grid, s,
                                                              pdl))
                           : (degrid ? launch_degridder_tcw_job(J.g, set, J.grid, J.flags, J.aterms, J.taper,
                                                                J.vis_out, s, pdl)
                                     : launch_gridder_tcw_job(J.g, set, J.vis, J.flags, J.aterms, J.taper, J.grid, s,
                                                              pdl));
                if (st != IDG_OK) return st;
            }
            continue;
        }
        const int blocks = degrid ? cl.degrid_blocks : cl.grid_blocks;
        const JobDev *jobs = b->d_jobs;
        const int2 *items = cl.d_items;
        int n_items = (int)cl.n_items;
        int *counter = b->d_counters + c;
        void *args[] = {(void *)&jobs, (void *)&items, (void *)&n_items, (void *)&counter};
        ProfileScope ps(degrid ? IDG_KERNEL_BATCH_DEGRID : IDG_KERNEL_BATCH_GRID, s, cl.vispix);
        e = cudaLaunchKernel(ks.fn, dim3(blocks), dim3(ks.threads), args, ks.smem, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch persistent launch");
    }
    return IDG_OK;
}

static idg_status batch_run(idg_batch *b, bool degrid, idg_stream stream) {
    if (!b) return fail(IDG_ERR_INVALID_ARG, "batch is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != b->device) return fail(IDG_ERR_INVALID_ARG, "the batch belongs to another device");
    cudaStream_t s = (cudaStream_t)stream;
    if (!(b->flags & IDG_BATCH_GRAPH)) return batch_enqueue(b, degrid, s);
    cudaGraphExec_t &exec = degrid ? b->graph_degrid : b->graph_grid;
    if (!exec) {
        // Record on the batch's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); nothing executes while
        // recording, and the graph is launched on the caller's stream below.
        if (!b->capture_stream) {
            e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        cudaStream_t cs = b->capture_stream;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        idg_status st = batch_enqueue(b, degrid, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (st != IDG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return IDG_OK;
}

namespace idg {
int batch_variant_count(int kernel, int L) {
    return (int)(kernel == IDG_KERNEL_BATCH_GRID ? grid_shapes(L).size() : degrid_shapes(L).size());
}
const char *batch_variant_name(int kernel, int L, int v) {
    auto s = kernel == IDG_KERNEL_BATCH_GRID ? grid_shapes(L) : degrid_shapes(L);
    return (v >= 0 && v < (int)s.size()) ? s[v].name : nullptr;
}
}  // namespace idg

extern "C" {

void idg_batch_destroy(idg_batch *b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (b->device >= 0) cudaSetDevice(b->device);
    if (b->graph_grid) cudaGraphExecDestroy(b->graph_grid);
    if (b->graph_degrid) cudaGraphExecDestroy(b->graph_degrid);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (auto &c : b->classes) {
        cudaFree(c.d_items);
        cudaFree(c.d_idx);
    }
    cudaFree(b->d_jobs);
    cudaFree(b->d_counters);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

idg_status idg_batch_create(const idg_plan *const *plans, const idg_job_buffers *bufs, int n_jobs, int flags,
                            idg_batch **out) {
    if (!out) return fail(IDG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || !bufs || n_jobs < 1) return fail(IDG_ERR_INVALID_ARG, "plans, buffers and n_jobs >= 1 are required");
    if (flags & ~IDG_BATCH_GRAPH) return fail(IDG_ERR_INVALID_ARG, "unknown batch flag");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    for (int j = 0; j < n_jobs; ++j) {
        const idg_plan *p = plans[j];
        if (!p) return fail(IDG_ERR_INVALID_ARG, "plan " + std::to_string(j) + " is NULL");
        if (p->device != dev) return fail(IDG_ERR_INVALID_ARG, "plan " + std::to_string(j) + " is not on the current device");
        if (p->opts.precision_mode != IDG_PHASOR_SINCOS)
            return fail(IDG_ERR_UNSUPPORTED, "batches run the direct (sin/cos) phasor form only");
        if (p->opts.fft_mode != IDG_FFT_FP32)
            return fail(IDG_ERR_UNSUPPORTED, "batches run the FP32 subgrid transform only");
        KernelShape a, c;
        if (!shapes_for(p->L, &a, &c))
            return fail(IDG_ERR_UNSUPPORTED, "batches support subgrid sizes 8, 16, 24 and 32 (job " + std::to_string(j) + ")");
        if (!p->taper_or_default(bufs[j].taper))
            return fail(IDG_ERR_INVALID_ARG, "job " + std::to_string(j) + " has no taper and its plan no default");
    }
    idg_batch *b = new idg_batch();
    b->device = dev;
    b->n_jobs = n_jobs;
    b->flags = flags;
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    std::vector<JobDev> hj(n_jobs);
    std::vector<std::vector<int2>> per_class;
    for (int j = 0; j < n_jobs; ++j) {
        const idg_plan *p = plans[j];
        JobDev &J = hj[j];
        J.g = p->geometry();
        J.vis = (const float4 *)bufs[j].vis;
        J.vis_out = (float4 *)bufs[j].vis_out;
        J.flags = bufs[j].flags;
        J.aterms = (const float4 *)bufs[j].aterms;
        J.taper = p->taper_or_default(bufs[j].taper);
        J.grid = (float4 *)bufs[j].grid;
        b->n_vis += p->stats.n_vis_planned;
        if (p->any_dropped && bufs[j].vis_out)
            b->zero_on_degrid.push_back({bufs[j].vis_out, (size_t)p->n_bl * p->n_t * p->n_chan * 32});
        // one class per (L, separable): a plan's subgrids within the remainder bound and the
        // pieces of the subgrids it splits go to the separable kernels, the others to the
        // direct ones (entries s index the plan's device table: pieces at n_subgrids ..)
        const int64_t n_sub = p->stats.n_subgrids, n_ent = n_sub + (int64_t)p->pieces.size();
        for (int64_t s = 0; s < n_ent; ++s) {
            if (s < n_sub && p->split_sub[s]) continue;
            const bool sep = separable_size(p->L) && (s >= n_sub || p->sep_sub[s]);
            size_t c = 0;
            while (c < b->classes.size() && (b->classes[c].L != p->L || b->classes[c].sep != sep)) ++c;
            if (c == b->classes.size()) {
                idg_batch::Class cl;
                cl.L = p->L;
                cl.sep = sep;
                cl.n_items = 0;
                cl.vispix = 0.0;
                shapes_for(p->L, &cl.grid, &cl.degrid);
                // L = 24 and 16 have tensor-core kernels only in the separable form
                if (sep && p->L != 32) cl.grid = cl.degrid = kTcShape;
                b->classes.push_back(cl);
                per_class.emplace_back();
            }
            per_class[c].push_back(make_int2(j, (int)s));
            b->classes[c].vispix += (double)p->kp_all[s] * p->L * p->L;
        }
    }
    idg_status st = IDG_OK;
    bool need_tc = false;                         // some class runs the tensor-core kernels
    for (size_t c = 0; c < b->classes.size() && st == IDG_OK; ++c) {
        auto &items = per_class[c];
        // cost order: most visibilities first, ties by job and subgrid
        std::stable_sort(items.begin(), items.end(), [&](const int2 &x, const int2 &y) {
            return plans[x.x]->kp_all[x.y] > plans[y.x]->kp_all[y.y];
        });
        auto &cl = b->classes[c];
        cl.n_items = (int64_t)items.size();
        if (cl.n_items > 2147483647) st = fail(IDG_ERR_INVALID_ARG, "too many subgrids in one batch class");
        // the tensor-core path pays a fixed cost per subgrid: classes whose visibilities
        // sit mostly in subgrids of fewer than kTcwFusedKpMin (direct) or kSepFusedKpMin
        // (separable) visibilities take the persistent kernels
        const int64_t kmin = cl.sep ? kSepFusedKpMin : kTcwFusedKpMin;
        int64_t small = 0, all = 0;
        for (const int2 &it : items) {
            const int64_t kp = plans[it.x]->kp_all[it.y];
            all += kp;
            if (kp < kmin) small += kp;
        }
        for (int k = 0; k < 2; ++k) {
            KernelShape &ks = k ? cl.degrid : cl.grid;
            if (ks.tc && 2 * small > all) {
                auto alt = k ? degrid_shapes(cl.L) : grid_shapes(cl.L);
                for (const KernelShape &x : alt)
                    if (!x.tc) {
                        ks = x;
                        break;
                    }
            }
            if (ks.tc) need_tc = true;
        }
        if (st == IDG_OK && cl.n_items > 0) {
            e = cudaMalloc(&cl.d_items, sizeof(int2) * items.size());
            if (e == cudaSuccess) e = cudaMemcpy(cl.d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_fail(e, "batch work list");
        }
        // the tensor-core launches: the items grouped by job, most visibilities first in each
        if (st == IDG_OK && cl.n_items > 0 && (cl.grid.tc || cl.degrid.tc)) {
            std::vector<int2> by_job(items);
            std::stable_sort(by_job.begin(), by_job.end(), [](const int2 &x, const int2 &y) { return x.x < y.x; });
            std::vector<int32_t> idx(by_job.size());
            for (size_t i = 0; i < by_job.size(); ++i) {
                idx[i] = by_job[i].y;
                if (i == 0 || by_job[i].x != by_job[i - 1].x) {
                    cl.run_first.push_back((int64_t)i);
                    cl.run_job.push_back(by_job[i].x);
                }
            }
            cl.run_first.push_back((int64_t)idx.size());
            e = cudaMalloc(&cl.d_idx, sizeof(int32_t) * idx.size());
            if (e == cudaSuccess) e = cudaMemcpy(cl.d_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_fail(e, "batch tensor-core work list");
        }
        // persistent grid: resident CTAs per SM x SMs, never more than the items
        for (int k = 0; k < 2 && st == IDG_OK; ++k) {
            KernelShape &ks = k ? cl.degrid : cl.grid;
            if (ks.tc) continue;
            e = cudaFuncSetAttribute(ks.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks.smem);
            int per_sm = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.fn, ks.threads, ks.smem);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "batch kernel occupancy");
                break;
            }
            const int64_t blocks = std::min<int64_t>(std::max(1, per_sm) * (int64_t)n_sm, std::max<int64_t>(1, cl.n_items));
            (k ? cl.degrid_blocks : cl.grid_blocks) = (int)blocks;
        }
    }
    if (st == IDG_OK && need_tc) {
        e = prepare_tcw_batch_kernels();      // outside any graph capture
        if (e != cudaSuccess) st = cuda_fail(e, "batch tensor-core kernel attributes");
    }
    if (st == IDG_OK) {
        b->host_jobs = hj;
        e = cudaMalloc(&b->d_jobs, sizeof(JobDev) * hj.size());
        if (e == cudaSuccess) e = cudaMemcpy(b->d_jobs, hj.data(), sizeof(JobDev) * hj.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(int) * std::max<size_t>(1, b->classes.size()));
        if (e != cudaSuccess) st = cuda_fail(e, "batch job table");
    }
    if (st != IDG_OK) {
        idg_batch_destroy(b);
        return st;
    }
    *out = b;
    return IDG_OK;
}

// resident CTAs per SM x SMs for a persistent shape, never more than the items
static idg_status persistent_blocks(const KernelShape &ks, int n_sm, int64_t n_items, int *blocks) {
    cudaError_t e = cudaFuncSetAttribute(ks.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ks.smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.fn, ks.threads, ks.smem);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel occupancy");
    *blocks = (int)std::min<int64_t>(std::max(1, per_sm) * (int64_t)n_sm, std::max<int64_t>(1, n_items));
    return IDG_OK;
}

idg_status idg_batch_autotune(idg_batch *b, double *ms, int cap, idg_stream stream) {
    if (!b) return fail(IDG_ERR_INVALID_ARG, "batch is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != b->device) return fail(IDG_ERR_INVALID_ARG, "the batch belongs to another device");
    cudaStream_t s = (cudaStream_t)stream;
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return cuda_fail(e, "batch autotune events");
    idg_status st = IDG_OK;
    int slot = 0;
    for (size_t c = 0; c < b->classes.size() && st == IDG_OK; ++c) {
        auto &cl = b->classes[c];
        for (int dir = 0; dir < 2 && st == IDG_OK; ++dir) {
            KernelShape &cur = dir ? cl.degrid : cl.grid;
            int &cur_blocks = dir ? cl.degrid_blocks : cl.grid_blocks;
            if (cl.n_items == 0 || cur.tc) continue;     // the tensor-core classes have one shape
            const auto shapes = dir ? degrid_shapes(cl.L) : grid_shapes(cl.L);
            double best_ms = 1e300;
            for (const KernelShape &x : shapes) {
                if (x.tc) continue;
                int blocks = 0;
                if ((st = persistent_blocks(x, n_sm, cl.n_items, &blocks)) != IDG_OK) break;
                const JobDev *jobs = b->d_jobs;
                const int2 *items = cl.d_items;
                int n_items = (int)cl.n_items;
                int *counter = b->d_counters + c;
                void *args[] = {(void *)&jobs, (void *)&items, (void *)&n_items, (void *)&counter};
                float t = 0.f;
                for (int rep = 0; rep < 2 && st == IDG_OK; ++rep) {      // one warm-up, one timed launch
                    e = cudaMemsetAsync(counter, 0, sizeof(int), s);
                    if (e == cudaSuccess && rep) e = cudaEventRecord(e0, s);
                    if (e == cudaSuccess) e = cudaLaunchKernel(x.fn, dim3(blocks), dim3(x.threads), args, x.smem, s);
                    if (e == cudaSuccess && rep) e = cudaEventRecord(e1, s);
                    if (e == cudaSuccess && rep) e = cudaEventSynchronize(e1);
                    if (e == cudaSuccess && rep) e = cudaEventElapsedTime(&t, e0, e1);
                    if (e != cudaSuccess) st = cuda_fail(e, "batch autotune trial");
                }
                if (st != IDG_OK) break;
                if (ms && slot < cap) ms[slot] = t;
                ++slot;
                if (t < best_ms) {
                    best_ms = t;
                    cur = x;
                    cur_blocks = blocks;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // recorded graphs hold the previous shapes
    if (b->graph_grid) cudaGraphExecDestroy(b->graph_grid);
    if (b->graph_degrid) cudaGraphExecDestroy(b->graph_degrid);
    b->graph_grid = b->graph_degrid = nullptr;
    return st;
}

idg_status idg_batch_grid(idg_batch *b, idg_stream stream) { return batch_run(b, false, stream); }

idg_status idg_batch_degrid(idg_batch *b, idg_stream stream) { return batch_run(b, true, stream); }

idg_status idg_batch_info(const idg_batch *b, int64_t *n_vis, int64_t *n_items, int *n_launches) {
    if (!b) return fail(IDG_ERR_INVALID_ARG, "batch is NULL");
    int64_t items = 0;
    int launches = 0;
    for (auto &c : b->classes) {
        items += c.n_items;
        if (c.n_items == 0) continue;
        launches += 1;      // work classes: one persistent launch, or one tensor-core launch per job
    }
    if (n_vis) *n_vis = b->n_vis;
    if (n_items) *n_items = items;
    if (n_launches) *n_launches = launches;
    return IDG_OK;
}

}  // extern "C"
