// Adder and splitter: move subgrids to and from the master uv grid
// (Algorithm 1 "Add subgrid to master grid", Algorithm 2 "initialize subgrid
// from master grid").  A pixel of a grid or subgrid is 32 contiguous bytes (4
// complex64 polarisations); consecutive threads move consecutive pixels of a
// subgrid row, so every warp touches a contiguous 32*L-byte run of a grid row.
// The adder uses 16-byte vector reductions because subgrids overlap.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"

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
