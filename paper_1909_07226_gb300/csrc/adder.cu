// Adder and splitter: move subgrids to and from the master uv grid
// (Algorithm 1 "Add subgrid to master grid", Algorithm 2 "initialize subgrid
// from master grid").  A pixel of a grid or subgrid is 32 contiguous bytes (4
// complex64 polarisations); consecutive threads move consecutive pixels of a
// subgrid row, so every warp touches a contiguous 32*L-byte run of a grid row.
// The adder uses 16-byte vector reductions because subgrids overlap.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"

namespace cg = cooperative_groups;

namespace idg {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
adder_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ sub,
             float4 *__restrict__ grid) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int L = g.L;
    const float4 *src = sub + (size_t)blockIdx.x * L * L * 2;
    float4 *dst = grid + (size_t)d.layer * g.N * g.N * 2;
    for (int pix = threadIdx.x; pix < L * L; pix += kThreads) {
        const int i = pix / L, j = pix - (pix / L) * L;
        const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
        dev::red_add_f4(dst + 2 * gp, src[2 * pix]);
        dev::red_add_f4(dst + 2 * gp + 1, src[2 * pix + 1]);
    }
}

// Compensated form: every vector atomic returns the value it replaced, so the
// rounding error of old + x can be recovered exactly (Knuth's TwoSum, valid in
// round-to-nearest for any magnitudes) and accumulated into a compensation
// grid, which is folded into the grid once at the end.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
    const float bb = s - a;
    return (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void add_compensated(float4 *dst, float4 *comp, float4 v) {
    const float4 old = atomicAdd(dst, v);
    const float4 e = make_float4(two_sum_err(old.x, v.x, old.x + v.x), two_sum_err(old.y, v.y, old.y + v.y),
                                 two_sum_err(old.z, v.z, old.z + v.z), two_sum_err(old.w, v.w, old.w + v.w));
    atomicAdd(comp, e);
}

__global__ void __launch_bounds__(kThreads)
adder_comp_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ sub,
                  float4 *__restrict__ grid, float4 *__restrict__ comp) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int L = g.L;
    const float4 *src = sub + (size_t)blockIdx.x * L * L * 2;
    const size_t off = (size_t)d.layer * g.N * g.N * 2;
    for (int pix = threadIdx.x; pix < L * L; pix += kThreads) {
        const int i = pix / L, j = pix - (pix / L) * L;
        const size_t gp = off + 2 * ((size_t)(d.r0 + i) * g.N + (d.q0 + j));
        add_compensated(grid + gp, comp + gp, src[2 * pix]);
        add_compensated(grid + gp + 1, comp + gp + 1, src[2 * pix + 1]);
    }
}

__global__ void fold_compensation_kernel(float4 *__restrict__ grid, const float4 *__restrict__ comp, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 a = grid[i], c = comp[i];
        grid[i] = make_float4(a.x + c.x, a.y + c.y, a.z + c.z, a.w + c.w);
    }
}

__global__ void __launch_bounds__(kThreads)
splitter_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ grid,
                float4 *__restrict__ sub) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    const DevSubgrid d = g.sub[sid];
    const int L = g.L;
    float4 *out = sub + (size_t)blockIdx.x * L * L * 2;
    const float4 *src = grid + (size_t)d.layer * g.N * g.N * 2;
    for (int pix = threadIdx.x; pix < L * L; pix += kThreads) {
        const int i = pix / L, j = pix - (pix / L) * L;
        const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
        out[2 * pix] = src[2 * gp];
        out[2 * pix + 1] = src[2 * gp + 1];
    }
}

}  // namespace

idg_status launch_adder(const Geometry &g, const SubgridSet &set, const void *sub, void *grid, void *stream) {
    if (set.count <= 0) return IDG_OK;
    adder_kernel<<<(unsigned)set.count, kThreads, 0, (cudaStream_t)stream>>>(g, set.idx, set.first,
                                                                              (const float4 *)sub, (float4 *)grid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adder launch");
    return IDG_OK;
}

idg_status launch_splitter(const Geometry &g, const SubgridSet &set, const void *grid, void *sub, void *stream) {
    if (set.count <= 0) return IDG_OK;
    splitter_kernel<<<(unsigned)set.count, kThreads, 0, (cudaStream_t)stream>>>(g, set.idx, set.first,
                                                                                 (const float4 *)grid, (float4 *)sub);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "splitter launch");
    return IDG_OK;
}

}  // namespace idg

namespace idg {

idg_status launch_adder_compensated(const Geometry &g, const SubgridSet &set, const void *sub, void *grid, void *comp,
                                    void *stream) {
    if (set.count <= 0) return IDG_OK;
    adder_comp_kernel<<<(unsigned)set.count, kThreads, 0, (cudaStream_t)stream>>>(
        g, set.idx, set.first, (const float4 *)sub, (float4 *)grid, (float4 *)comp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "compensated adder launch");
    return IDG_OK;
}

idg_status launch_fold_compensation(void *grid, const void *comp, size_t n_float4, void *stream) {
    if (n_float4 == 0) return IDG_OK;
    const unsigned blocks = (unsigned)std::min<size_t>((n_float4 + 255) / 256, 152 * 16);
    fold_compensation_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((float4 *)grid, (const float4 *)comp, n_float4);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "compensation fold launch");
    return IDG_OK;
}

}  // namespace idg

// Sorted (deterministic) adder, IDG_ADDER_SORTED.  The grid is cut into tiles of kTile x
// kTile pixels per layer; the plan lists, for every tile that a subgrid overlaps, those
// subgrids by plan index (ascending).  The subgrids come in chunks of consecutive plan
// indices [first, first + count) (scratch slot = plan index - first).  A tile's CTA finds
// the chunk's part of the tile's list by binary search and sums the parts of those subgrid
// images that fall on the tile in that order.  A tile whose whole list is longer than
// kHeavyEntries (the uv centre of a long observation: a few tiles hold most subgrids) takes
// a cluster of kHeavyCluster CTAs instead: rank r sums the r-th of kHeavyCluster equal
// contiguous segments of the chunk's part, and the ranks' partial sums are added in rank
// order through distributed shared memory.  The sum goes to the tile with plain loads and
// stores.  No two CTAs write a pixel and every summation order is fixed by the plan and
// the chunk, so the grid is the same bit for bit from run to run.
namespace idg {
namespace {

constexpr int kTileThreads = 256;
constexpr int kTilePix = kTile * kTile / kTileThreads;     // pixels per thread

// [lo, hi): the entries of list row `row` with first <= plan index < first + count
__device__ __forceinline__ void chunk_entries(const int32_t *__restrict__ tile_first,
                                              const int32_t *__restrict__ tile_sub, int row, int first, int count,
                                              int &lo, int &hi) {
    int a = tile_first[row], b = tile_first[row + 1];
    hi = b;
    while (a < b) {
        const int m = (a + b) >> 1;
        if (tile_sub[m] < first) a = m + 1;
        else b = m;
    }
    lo = a;
    b = hi;
    while (a < b) {
        const int m = (a + b) >> 1;
        if (tile_sub[m] < first + count) a = m + 1;
        else b = m;
    }
    hi = a;
}

// acc += the tile's part of the images of entries [e0, e1), in entry order; this thread's
// pixels are threadIdx.x + m kTileThreads (row-major in the tile)
__device__ __forceinline__ void sum_entries(const Geometry &g, const int32_t *__restrict__ tile_sub, int e0, int e1,
                                            int first, const float4 *__restrict__ sub, int y0, int x0,
                                            float4 (&acc)[kTilePix][2]) {
    const int L = g.L;
    for (int e = e0; e < e1; ++e) {
        const int s = tile_sub[e];
        const int r0 = g.sub[s].r0, q0 = g.sub[s].q0;
        const float4 *src = sub + (size_t)(s - first) * L * L * 2;
#pragma unroll
        for (int m = 0; m < kTilePix; ++m) {
            const int p = threadIdx.x + m * kTileThreads;
            const int i = y0 + p / kTile - r0, j = x0 + p % kTile - q0;
            if (i >= 0 && i < L && j >= 0 && j < L) {
                const float4 u = src[2 * (i * L + j)], v = src[2 * (i * L + j) + 1];
                acc[m][0] = make_float4(acc[m][0].x + u.x, acc[m][0].y + u.y, acc[m][0].z + u.z, acc[m][0].w + u.w);
                acc[m][1] = make_float4(acc[m][1].x + v.x, acc[m][1].y + v.y, acc[m][1].z + v.z, acc[m][1].w + v.w);
            }
        }
    }
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// rows [0, gridDim.x) of the tile lists: one CTA each
__global__ void __launch_bounds__(kTileThreads)
tile_adder_kernel(Geometry g, const int32_t *__restrict__ tile_ids, const int32_t *__restrict__ tile_first,
                  const int32_t *__restrict__ tile_sub, int first, int count, const float4 *__restrict__ sub,
                  float4 *__restrict__ grid) {
    const int N = g.N, ntx = (N + kTile - 1) / kTile;
    int lo, hi;
    chunk_entries(tile_first, tile_sub, blockIdx.x, first, count, lo, hi);
    if (lo == hi) return;                 // (the same for every thread of the CTA)
    const int tile = tile_ids[blockIdx.x];
    const int layer = tile / (ntx * ntx), rem = tile - layer * ntx * ntx;
    const int y0 = (rem / ntx) * kTile, x0 = (rem % ntx) * kTile;
    float4 a[kTilePix][2];
#pragma unroll
    for (int m = 0; m < kTilePix; ++m) a[m][0] = a[m][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    sum_entries(g, tile_sub, lo, hi, first, sub, y0, x0, a);
    float4 *dst = grid + (size_t)layer * N * N * 2;
#pragma unroll
    for (int m = 0; m < kTilePix; ++m) {
        const int p = threadIdx.x + m * kTileThreads;
        const int y = y0 + p / kTile, x = x0 + p % kTile;
        if (y >= N || x >= N) continue;
        float4 *o = dst + 2 * ((size_t)y * N + x);
        o[0] = add4(o[0], a[m][0]);
        o[1] = add4(o[1], a[m][1]);
    }
}

// rows [row0, row0 + gridDim.x / kHeavyCluster): one cluster of kHeavyCluster CTAs each
__global__ void __cluster_dims__(kHeavyCluster, 1, 1) __launch_bounds__(kTileThreads)
tile_adder_cluster_kernel(Geometry g, const int32_t *__restrict__ tile_ids, const int32_t *__restrict__ tile_first,
                          const int32_t *__restrict__ tile_sub, int row0, int first, int count,
                          const float4 *__restrict__ sub, float4 *__restrict__ grid) {
    constexpr int kParts = kTile * kTile * 2;                // float4 values of a tile
    constexpr int kPerRank = kParts / kHeavyCluster;         // of those, each rank's to finish
    static_assert(kPerRank % kTileThreads == 0, "each rank finishes whole passes of its threads");
    __shared__ float4 part[kParts];
    const cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int row = row0 + (int)(blockIdx.x / kHeavyCluster);
    const int N = g.N, ntx = (N + kTile - 1) / kTile;
    int lo, hi;
    chunk_entries(tile_first, tile_sub, row, first, count, lo, hi);
    if (lo == hi) return;                 // (the same for every CTA of the cluster)
    const int tile = tile_ids[row];
    const int layer = tile / (ntx * ntx), rem = tile - layer * ntx * ntx;
    const int y0 = (rem / ntx) * kTile, x0 = (rem % ntx) * kTile;
    const int seg = (hi - lo + kHeavyCluster - 1) / kHeavyCluster;
    const int e0 = min(hi, lo + rank * seg), e1 = min(hi, e0 + seg);
    float4 a[kTilePix][2];
#pragma unroll
    for (int m = 0; m < kTilePix; ++m) a[m][0] = a[m][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    sum_entries(g, tile_sub, e0, e1, first, sub, y0, x0, a);
#pragma unroll
    for (int m = 0; m < kTilePix; ++m) {
        const int p = threadIdx.x + m * kTileThreads;
        part[2 * p] = a[m][0];
        part[2 * p + 1] = a[m][1];
    }
    cluster.sync();                       // every rank's partial sums are in its shared memory
    float4 *dst = grid + (size_t)layer * N * N * 2;
#pragma unroll
    for (int k = 0; k < kPerRank / kTileThreads; ++k) {
        const int q = rank * kPerRank + k * kTileThreads + (int)threadIdx.x;
        float4 t = *cluster.map_shared_rank(&part[q], 0);
#pragma unroll
        for (int r = 1; r < kHeavyCluster; ++r) t = add4(t, *cluster.map_shared_rank(&part[q], r));
        const int p = q >> 1, y = y0 + p / kTile, x = x0 + p % kTile;
        if (y < N && x < N) {
            float4 *o = dst + 2 * ((size_t)y * N + x) + (q & 1);
            *o = add4(*o, t);
        }
    }
    cluster.sync();                       // no rank leaves while another reads its partial sums
}

}  // namespace

idg_status launch_adder_sorted(const Geometry &g, const SubgridSet &set, const void *sub, void *grid,
                               const SortedTiles &t, void *stream) {
    if (set.count <= 0 || t.n_tiles == 0) return IDG_OK;
    if (set.idx) return fail(IDG_ERR_INVALID_ARG, "the sorted adder takes consecutive plan indices");
    const int64_t n_light = t.n_tiles - t.n_heavy;
    if (n_light > 0)
        tile_adder_kernel<<<(unsigned)n_light, kTileThreads, 0, (cudaStream_t)stream>>>(
            g, t.tile_ids, t.tile_first, t.tile_sub, (int)set.first, (int)set.count, (const float4 *)sub,
            (float4 *)grid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sorted adder launch");
    if (t.n_heavy > 0)
        tile_adder_cluster_kernel<<<(unsigned)(t.n_heavy * kHeavyCluster), kTileThreads, 0, (cudaStream_t)stream>>>(
            g, t.tile_ids, t.tile_first, t.tile_sub, (int)n_light, (int)set.first, (int)set.count,
            (const float4 *)sub, (float4 *)grid);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sorted adder (cluster) launch");
    return IDG_OK;
}

}  // namespace idg
