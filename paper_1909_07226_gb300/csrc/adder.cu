// Adder and splitter: move subgrids to and from the master uv grid
// (Algorithm 1 "Add subgrid to master grid", Algorithm 2 "initialize subgrid
// from master grid").  A pixel of a grid or subgrid is 32 contiguous bytes (4
// complex64 polarisations); consecutive threads move consecutive pixels of a
// subgrid row, so every warp touches a contiguous 32*L-byte run of a grid row.
// The adder uses 16-byte vector atomics because subgrids overlap.
#include <cuda_runtime.h>

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
        atomicAdd(dst + 2 * gp, src[2 * pix]);
        atomicAdd(dst + 2 * gp + 1, src[2 * pix + 1]);
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
