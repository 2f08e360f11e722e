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

// The same transform for L = 32 with two threads per line, for the fused kernels
// whose CTAs have at least 256 threads: thread t of a pair transforms the samples
// 2 m + t (16 points in registers), and the last radix-2 step combines the halves,
// X[k] = E[k] + w^k O[k] and X[k + 16] = E[k] - w^k O[k] (w = exp(SIGN 2 pi i / 32)),
// through a shuffle: the odd thread premultiplies its O[k] by w^k, the pair swaps
// values and each thread writes its half of the line.  The pair is lanes l and
// l + 16 of a warp, so every half-warp touches 16 consecutive lines (rows) or 16
// consecutive x (columns): with the row pitch of 33 both passes are free of bank
// conflicts.  Threads from 256 on only take part in the barriers.  Ends with a barrier.
template <int SIGN>
__device__ __forceinline__ void fft2_planar_pairs32(float2 *s, int tid) {
    constexpr int L = 32, P = L + 1;
    const int t = (tid >> 4) & 1;                    // even (0) or odd (1) samples
    const int line = 16 * (tid >> 5) + (tid & 15);   // 0 .. 127 for tid < 256
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        if (tid < 8 * L) {
            // rows: line = pol L + y, samples along x; columns: line = pol L + x, samples along y
            const int pol = line >> 5, i = line & (L - 1);
            float2 *base = pass == 0 ? s + line * P : s + pol * L * P + i;
            const int stride = pass == 0 ? 1 : P;
            float2 v[L / 2];
#pragma unroll
            for (int m = 0; m < L / 2; ++m) v[m] = base[(2 * m + t) * stride];
            RegFFT<L / 2, SIGN>::run(v);
            const float sg = t ? -1.0f : 1.0f;
#pragma unroll
            for (int k = 0; k < L / 2; ++k) {
                const float2 p = t ? cmul(v[k], twiddle<L, SIGN>(k)) : v[k];
                const float qx = __shfl_xor_sync(0xffffffffu, p.x, 16);
                const float qy = __shfl_xor_sync(0xffffffffu, p.y, 16);
                v[k] = make_float2(fmaf(sg, p.x, qx), fmaf(sg, p.y, qy));
            }
#pragma unroll
            for (int k = 0; k < L / 2; ++k) base[(L / 2 * t + k) * stride] = v[k];
        }
        __syncthreads();
    }
}

}  // namespace dev
}  // namespace idg
