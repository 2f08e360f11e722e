// Batched subgrid transform ("FFT"/"IFFT" of Algorithms 1 and 2).
//
//   out[i][j] = L^-2 sum_{y,x} in[y][x] exp(SIGN 2 pi i ((j-L/2)(x-L/2) + (i-L/2)(y-L/2)) / L)
//
// For even L the centred 2D transform equals (-1)^(i+j) DFT2((-1)^(x+y) in):
// the two factors (-1)^(L/2) of the 1D centring cancel in 2D.  One CTA
// transforms one subgrid (all four polarisations) in shared memory: one
// thread per row for the row pass, one per column for the column pass, each
// a length-L FFT held in registers.  Rows are padded by one element so both
// passes are free of bank conflicts.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace idg {
namespace {

using namespace dev;

template <int L, int SIGN>
__global__ void __launch_bounds__(4 * L) fft_kernel(float4 *__restrict__ data) {
    constexpr int P = L + 1;   // padded row pitch (float2)
    extern __shared__ float2 s[];   // [4][L][P]
    float4 *g = data + (size_t)blockIdx.x * L * L * 2;
    const int tid = threadIdx.x;
    const float scale = 1.0f / (float)(L * L);

    // load [y][x][pol] -> s[pol][y][x] with the (-1)^(x+y) pre-factor
    for (int pix = tid; pix < L * L; pix += 4 * L) {
        const int y = pix / L, x = pix % L;
        const float sg = ((x + y) & 1) ? -1.0f : 1.0f;
        const float4 a = g[2 * pix], b = g[2 * pix + 1];
        s[(0 * L + y) * P + x] = make_float2(sg * a.x, sg * a.y);
        s[(1 * L + y) * P + x] = make_float2(sg * a.z, sg * a.w);
        s[(2 * L + y) * P + x] = make_float2(sg * b.x, sg * b.y);
        s[(3 * L + y) * P + x] = make_float2(sg * b.z, sg * b.w);
    }
    __syncthreads();
    {   // rows: thread (pol, y)
        float2 v[L];
        float2 *row = s + tid * P;
#pragma unroll
        for (int x = 0; x < L; ++x) v[x] = row[x];
        RegFFT<L, SIGN>::run(v);
#pragma unroll
        for (int x = 0; x < L; ++x) row[x] = v[x];
    }
    __syncthreads();
    {   // columns: thread (pol, x)
        const int pol = tid / L, x = tid % L;
        float2 v[L];
        float2 *col = s + pol * L * P + x;
#pragma unroll
        for (int y = 0; y < L; ++y) v[y] = col[y * P];
        RegFFT<L, SIGN>::run(v);
#pragma unroll
        for (int y = 0; y < L; ++y) col[y * P] = v[y];
    }
    __syncthreads();
    for (int pix = tid; pix < L * L; pix += 4 * L) {
        const int i = pix / L, j = pix % L;
        const float sg = ((i + j) & 1) ? -scale : scale;
        const float2 p0 = s[(0 * L + i) * P + j], p1 = s[(1 * L + i) * P + j];
        const float2 p2 = s[(2 * L + i) * P + j], p3 = s[(3 * L + i) * P + j];
        g[2 * pix] = make_float4(sg * p0.x, sg * p0.y, sg * p1.x, sg * p1.y);
        g[2 * pix + 1] = make_float4(sg * p2.x, sg * p2.y, sg * p3.x, sg * p3.y);
    }
}

template <int L>
idg_status launch(int64_t count, int direction, void *data, cudaStream_t s) {
    const size_t smem = sizeof(float2) * 4 * L * (L + 1);
    auto kern = direction < 0 ? fft_kernel<L, -1> : fft_kernel<L, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "fft smem attribute");
    kern<<<(unsigned)count, 4 * L, smem, s>>>((float4 *)data);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fft launch");
    return IDG_OK;
}

}  // namespace

idg_status launch_fft(int L, int64_t count, int direction, void *data, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    switch (L) {
    case 8: return launch<8>(count, direction, data, s);
    case 16: return launch<16>(count, direction, data, s);
    case 24: return launch<24>(count, direction, data, s);
    case 32: return launch<32>(count, direction, data, s);
    case 48: return launch<48>(count, direction, data, s);
    case 64: return launch<64>(count, direction, data, s);
    }
    return fail(IDG_ERR_UNSUPPORTED, "subgrid size not compiled in");
}

}  // namespace idg
