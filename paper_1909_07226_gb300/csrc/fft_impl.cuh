// Centred 2D transform of the four polarisation planes of one subgrid held in
// shared memory as s[pol][y][x] (row pitch L + 1, which keeps both passes free
// of bank conflicts).  Rows, then columns, each a length-L FFT in registers,
// spread over the nt threads of the CTA.  The caller applies the (-1)^(x+y)
// centring factors and the 1/L^2 scale.  Ends with a barrier.
#pragma once

#include "device_common.cuh"

namespace idg {
namespace dev {

template <int L, int SIGN>
__device__ __forceinline__ void fft2_planar(float2 *s, int tid, int nt) {
    constexpr int P = L + 1;
    for (int line = tid; line < 4 * L; line += nt) {
        float2 v[L];
        float2 *row = s + line * P;
#pragma unroll
        for (int x = 0; x < L; ++x) v[x] = row[x];
        RegFFT<L, SIGN>::run(v);
#pragma unroll
        for (int x = 0; x < L; ++x) row[x] = v[x];
    }
    __syncthreads();
    for (int line = tid; line < 4 * L; line += nt) {
        const int pol = line / L, x = line - (line / L) * L;
        float2 v[L];
        float2 *col = s + pol * L * P + x;
#pragma unroll
        for (int y = 0; y < L; ++y) v[y] = col[y * P];
        RegFFT<L, SIGN>::run(v);
#pragma unroll
        for (int y = 0; y < L; ++y) col[y * P] = v[y];
    }
    __syncthreads();
}

}  // namespace dev
}  // namespace idg
