// Degridder on the 5th-generation tensor cores (tcgen05), L = 32.
//
// The degridding sum of Algorithm 2, y_k[q] = sum_pix P[pix][q] exp(-i phi_k(pix))
// with P = taper * A_p . I_p . A_q^H (Sect. 3.4), is a complex contraction over
// the pixels.  As a real GEMM with M = visibilities, K = 2 per pixel and N = 16:
//   A[k][2 pix] = cos phi,  A[k][2 pix + 1] = -sin phi          (the phasor exp(-i phi))
//   B[2q][2 pix] = Re P_q,  B[2q][2 pix + 1] = -Im P_q,
//   B[2q+1][2 pix] = Im P_q, B[2q+1][2 pix + 1] = Re P_q        (rows 0..7: P_hi, 8..15: P_lo)
// so D[k][2q + r] + D[k][8 + 2q + r] is (Re, Im)[r] of y_k[q].  P is scaled by a
// power of two per subgrid (largest component in [2^9, 2^10)) and split into FP16
// hi/lo parts, as are the phasors; the two MMAs per tile and K step are
// A_hi [P_hi | P_lo] and A_lo [P_hi | P_lo].
//
// One CTA per subgrid: 8 producer warps and one MMA warp.  Visibilities are
// taken in blocks of 256 (two M tiles of 128); producer warp w owns tile w / 4,
// tensor-memory lanes 32 (w % 4) .. + 31, one visibility per thread.  A step
// covers 16 pixels (two K = 16 chunks): each producer writes the phasor rows of
// its visibility (hi, lo) into one of three A stages in tensor memory and
// arrives on full[s]; the MMA warp issues 8 MMAs and commits to empty[s].
// Tensor memory (256 columns, two CTAs per SM):
//   columns  0..63   two accumulator regions r (32 r, tile t at + 16 t)
//   columns 64..255  three A stages s (64 + 64 s, tile t at + 32 t, chunk at + 16 kc; 8 hi, 8 lo)
// The tensor cores' FP32 accumulation truncates, so the sum over 1024 pixels
// is cut into periods of 16 steps that alternate between the two regions: the
// MMA warp commits a period to foldbar[r]; one step into the next period each
// producer adds its own row of region r into FP32 registers and arrives on
// folded[r], which the MMA warp waits for before it reuses the region.  The
// last period of a block is folded one step into the next block, and the
// block's visibilities are written then.  Waits are bounded;
// after a failed wait a thread skips every later wait, the error word is set
// and no output is written.
#include "batch_jobs.cuh"
#include "degridder_impl.cuh"
#include "fft_impl.cuh"
#include "tc_common.cuh"

namespace idg {

// device error word of the tensor-core degridder (0 = ok)
__device__ int g_tcd_error = 0;

namespace {

using namespace dev;
using namespace tc;

constexpr int DL = 32;
constexpr int DPIX = DL * DL;
constexpr int DNP = 256;                          // producer threads
constexpr int DNT = DNP + 32;                     // + the MMA warp
constexpr int DBLK = 256;                         // visibilities per block
constexpr int DSTEPS = DPIX / 16;                 // 64 steps of 16 pixels per block
constexpr int DFOLD = 16;                         // steps per accumulation period
constexpr int DSTAGES = 3;
constexpr int DCOLS = 256;
constexpr int D_B_BYTES = (2 * DPIX / 16) * kTile16;   // 128 K chunks of 8 pixels = 64 KB
constexpr int D_SMEM = D_B_BYTES + DPIX * 4;            // + n'
constexpr int FFT_P = DL + 1;                            // padded row pitch of the transform planes (float2)
static_assert(4 * DL * FFT_P * 8 <= D_B_BYTES, "transform planes fit in the P operand buffer");

// Visibilities of subgrid d of geometry g from its image src[L][L][4], or with
// FUSED from the grid src[layer][N][N][4]: split and transformed in shared memory
// first (Algorithm 2: split from the master grid, "IFFT", image-domain kernel, sum).
template <bool FUSED>
__device__ __forceinline__ void degridder_tcw_body(const Geometry &g, const DevSubgrid d,
                                                   const float4 *__restrict__ src, const uint8_t *__restrict__ flags,
                                                   const float4 *__restrict__ aterms, const float *__restrict__ taper,
                                                   float4 *__restrict__ vis_out) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;                               // P operand, chunk c (pixels 8c .. 8c + 7) at c * 512
    float *s_np = (float *)(smem + D_B_BYTES);        // n' per pixel
    float2 *s_fft = (float2 *)smem;                   // FUSED prologue: [4][L][L + 1], before the P operand is built
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[DSTAGES], s_empty[DSTAGES], s_foldbar[2], s_folded[2], s_drain;
    __shared__ float s_red[8];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == 8;
    const int nblk = (d.kp + DBLK - 1) / DBLK;
    const int total_steps = nblk * DSTEPS;

    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "n"(DCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < DSTAGES; ++s) {
            mbar_init(smem_u32(&s_full[s]), 8);
            mbar_init(smem_u32(&s_empty[s]), 1);
        }
        for (int r = 0; r < 2; ++r) {
            mbar_init(smem_u32(&s_foldbar[r]), 1);
            mbar_init(smem_u32(&s_folded[r]), 8);
        }
        mbar_init(smem_u32(&s_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    if (FUSED) {
        // every thread: split from the grid with the (-1)^(i+j) factor, then the inverse transform
        const float4 *gsrc = src + (size_t)d.layer * g.N * g.N * 2;
        for (int pix = tid; pix < DPIX; pix += DNT) {
            const int i = pix / DL, j = pix % DL;
            const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
            const float sg = ((i + j) & 1) ? -1.0f : 1.0f;
            const float4 a = gsrc[2 * gp], b = gsrc[2 * gp + 1];
            s_fft[(0 * DL + i) * FFT_P + j] = make_float2(sg * a.x, sg * a.y);
            s_fft[(1 * DL + i) * FFT_P + j] = make_float2(sg * a.z, sg * a.w);
            s_fft[(2 * DL + i) * FFT_P + j] = make_float2(sg * b.x, sg * b.y);
            s_fft[(3 * DL + i) * FFT_P + j] = make_float2(sg * b.z, sg * b.w);
        }
        __syncthreads();
        fft2_planar<DL, +1>(s_fft, tid, DNT);
    }
    // image-domain kernel: P = taper * A_p . I . A_q^H, four pixels per producer thread
    float pv[4][8];
    float m = 0.0f;
    if (!mma_warp) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int pix = tid + DNP * i;
            M22 P;
            if (FUSED) {      // (-1)^(x+y) / L^2 of the transform
                const int y = pix / DL, x = pix % DL;
                const float sg = ((x + y) & 1) ? -1.0f / DPIX : 1.0f / DPIX;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 v = s_fft[(q * DL + y) * FFT_P + x];
                    P.m[q] = make_float2(sg * v.x, sg * v.y);
                }
            } else {
                P = load_m22(src + 2 * pix);
            }
            if (aterms) {
                const size_t base = ((size_t)d.slot * g.n_stations) * DPIX;
                const M22 Ap = load_m22(aterms + 2 * (base + (size_t)d.st_p * DPIX + pix));
                const M22 Aq = load_m22(aterms + 2 * (base + (size_t)d.st_q * DPIX + pix));
                P = mul_mul_herm(Ap, P, Aq);
            }
            const float tw = taper[pix];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                pv[i][2 * q] = tw * P.m[q].x;
                pv[i][2 * q + 1] = tw * P.m[q].y;
                m = fmaxf(m, fmaxf(fabsf(pv[i][2 * q]), fabsf(pv[i][2 * q + 1])));
            }
            s_np[pix] = g.nprime[pix];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && !mma_warp) s_red[warp] = m;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    float inv_scale = 1.0f;
    if (!mma_warp) {
        m = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) m = fmaxf(m, s_red[w]);
        int e2 = 0;
        if (m > 0.0f) frexpf(m, &e2);
        const float scale = ldexpf(1.0f, 10 - e2);
        inv_scale = ldexpf(1.0f, e2 - 10);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int pix = tid + DNP * i;
            uint8_t *Bc = sB + (pix >> 3) * kTile16;
            const int kl = 2 * (pix & 7);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float re = pv[i][2 * q] * scale, im = pv[i][2 * q + 1] * scale;
                uint32_t h0, l0, h1, l1;
                split_e(re, -im, h0, l0);     // row 2q:     (Re P, -Im P) at k = 2 pix, 2 pix + 1
                split_e(im, re, h1, l1);      // row 2q + 1: (Im P,  Re P)
                *(uint32_t *)(Bc + kmaj_off(2 * q, kl)) = h0;
                *(uint32_t *)(Bc + kmaj_off(8 + 2 * q, kl)) = l0;
                *(uint32_t *)(Bc + kmaj_off(2 * q + 1, kl)) = h1;
                *(uint32_t *)(Bc + kmaj_off(9 + 2 * q, kl)) = l1;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (mma_warp) {
        if (lane == 0) {
            bool failed = false;
            int st = 0;
            uint32_t full_par = 0;                 // parity of the current use of stage st
            for (int S = 0; S < total_steps; ++S) {
                const int s = S % DSTEPS, P = S / DFOLD, r = P & 1;
                const int nt = (S / DSTEPS) * DBLK + 128 < d.kp ? 2 : 1;   // the block's second tile may be empty
                if (S % DFOLD == 0 && P >= 2)      // the producers have folded period P - 2 out of region r
                    wait_or_fail(smem_u32(&s_folded[r]), (uint32_t)(((P - 2) >> 1) & 1), failed);
                wait_or_fail(smem_u32(&s_full[st]), full_par, failed);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int t = 0; t < 2; ++t)
#pragma unroll
                    for (int kc = 0; kc < 2; ++kc) {
                        if (t >= nt) continue;
                        const uint32_t dt = tmem + (uint32_t)(32 * r + 16 * t);
                        const uint32_t at = tmem + (uint32_t)(64 + 64 * st + 32 * t + 16 * kc);
                        const uint64_t db = smem_desc(smem_u32(sB + (2 * s + kc) * kTile16));
                        const uint32_t acc = (S % DFOLD == 0 && kc == 0) ? 0u : 1u;
                        mma_ta(dt, at, db, acc);
                        mma_ta(dt, at + 8, db, 1u);
                    }
                commit(smem_u32(&s_empty[st]));
                if (S % DFOLD == DFOLD - 1) commit(smem_u32(&s_foldbar[r]));
                if (++st == DSTAGES) {
                    st = 0;
                    full_par ^= 1u;
                }
            }
            commit(smem_u32(&s_drain));
            bool drained = false;
            wait_or_fail(smem_u32(&s_drain), 0u, drained);   // bounded: own MMAs finish before the free
            if (failed) atomicExch(&g_tcd_error, 1);
        }
    } else {
        const int t = warp >> 2, q4 = warp & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16);
        bool failed = false;
        float acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = 0.0f;

        // add region r of period P into acc, then release the region to the MMA warp
        auto fold = [&](int P) {
            const int r = P & 1;
            wait_or_fail(smem_u32(&s_foldbar[r]), (uint32_t)((P >> 1) & 1), failed);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[16];
            tmem_ld16(lane_base + (uint32_t)(32 * r + 16 * t), v);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] += __uint_as_float(v[c]) + __uint_as_float(v[8 + c]);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_folded[r]));
        };
        // write the finished visibility of a block and clear the sums
        auto flush = [&](bool valid, size_t vi) {
            if (valid && !failed) {
                float4 o01 = make_float4(acc[0] * inv_scale, acc[1] * inv_scale, acc[2] * inv_scale, acc[3] * inv_scale);
                float4 o23 = make_float4(acc[4] * inv_scale, acc[5] * inv_scale, acc[6] * inv_scale, acc[7] * inv_scale);
                if (flags && flags[vi]) {           // flagged visibilities are output as 0
                    o01 = make_float4(0.f, 0.f, 0.f, 0.f);
                    o23 = o01;
                }
                vis_out[2 * vi] = o01;
                vis_out[2 * vi + 1] = o23;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
        };

        int S = 0;
        int st = 0;                  // A stage of step S (S mod 3)
        uint32_t empty_par = 0;      // parity of the MMAs that last read stage st (from step S - 3)
        bool prev_valid = false;
        size_t prev_vi = 0;
        for (int blk = 0; blk < nblk; ++blk) {
            const int k = blk * DBLK + t * 128 + 32 * q4 + lane;      // this thread's visibility
            const bool live = blk * DBLK + t * 128 < d.kp;            // the tile holds a visibility
            float na = 0.0f, nb = 0.0f, nc = 0.0f;                    // -a, -b, -c: sin/cos give exp(-i phi)
            size_t vi = 0;
            if (k < d.kp) {
                int tt, cc;
                vi = vis_index(g, d, k, tt, cc);
                const PhaseCoef pc = phase_coef(g, d, tt, cc);
                na = -pc.a;
                nb = -pc.b;
                nc = -pc.c;
            }
#pragma unroll 2      // a row of 32 pixels per iteration: the column offset of each half is constant
            for (int s = 0; s < DSTEPS; ++s, ++S) {
                if (S >= DSTAGES) wait_or_fail(smem_u32(&s_empty[st]), empty_par, failed);
                const int y = s >> 1, x0 = 16 * (s & 1);
                if (live) {
                    const float base = fmaf(na, (float)(x0 - DL / 2), nb * (float)(y - DL / 2));
                    const float4 *np4 = (const float4 *)(s_np + 16 * s);
#pragma unroll
                    for (int kc = 0; kc < 2; ++kc) {
                        const float4 n0 = np4[2 * kc], n1 = np4[2 * kc + 1];
                        const float np[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
                        uint32_t e[16];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float phase = fmaf(na, (float)(8 * kc + j), fmaf(nc, np[j], base));
                            float sn, cs;
                            __sincosf(phase, &sn, &cs);
                            split_e(cs, sn, e[j], e[8 + j]);
                        }
                        tmem_st16(lane_base + (uint32_t)(64 + 64 * st + 32 * t + 16 * kc), e);
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&s_full[st]));
                // fold the previous period one step late; at the second step of a block that
                // period is the previous block's last, after which that block's result is final
                if (s % DFOLD == 1 && S > DFOLD) {
                    fold(S / DFOLD - 1);
                    if (s == 1) flush(prev_valid, prev_vi);
                }
                if (++st == DSTAGES) {
                    st = 0;
                    if (S >= DSTAGES) empty_par ^= 1u;   // the wait at step S + 1 is for step S - 2
                }
            }
            prev_valid = k < d.kp;
            prev_vi = vi;
        }
        if (nblk > 0) {
            fold((S - 1) / DFOLD);                                      // the last period
            flush(prev_valid, prev_vi);
        }
        if (failed && lane == 0) atomicExch(&g_tcd_error, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(DCOLS));
}

// one CTA per subgrid of one plan (plan index idx[b] or first + b; image b of sub)
__global__ void __launch_bounds__(DNT, 2)
degridder_tcw_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ sub,
                     const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                     const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    degridder_tcw_body<false>(g, g.sub[sid], sub + (size_t)blockIdx.x * DPIX * 2, flags, aterms, taper, vis_out);
}

// fused: one CTA per subgrid, read from the grid
__global__ void __launch_bounds__(DNT, 2)
degridder_tcw_fused_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ grid,
                           const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                           const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    allow_dependents();
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    degridder_tcw_body<true>(g, g.sub[sid], grid, flags, aterms, taper, vis_out);
    complete_after_primary();
}

}  // namespace

idg_status launch_degridder_tcw_fused(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                      const void *aterms, const float *taper, void *vis_out, void *stream) {
    if (g.L != DL) return fail(IDG_ERR_UNSUPPORTED, "the tensor-core degridder is built for L = 32");
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute(degridder_tcw_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, D_SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core degridder smem attribute");
    degridder_tcw_fused_kernel<<<(unsigned)set.count, DNT, D_SMEM, s>>>(g, set.idx, set.first, (const float4 *)grid,
                                                                         flags, (const float4 *)aterms, taper,
                                                                         (float4 *)vis_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core fused degridder launch");
    return IDG_OK;
}

cudaError_t prepare_tcw_batch_kernels() {
    cudaError_t e = prepare_gridder_tcw_batch();
    if (e == cudaSuccess) e = prepare_sep_batch_kernels();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(degridder_tcw_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, D_SMEM);
    return e;
}

// a batch's launch of the fused kernel over one job's items (the shared-memory attribute
// is set by prepare_tcw_batch_kernels, outside graph capture); pdl: see launch_pdl
idg_status launch_degridder_tcw_job(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *vis_out, void *stream, bool pdl) {
    if (g.L != DL) return fail(IDG_ERR_UNSUPPORTED, "the tensor-core degridder is built for L = 32");
    if (set.count <= 0) return IDG_OK;
    const cudaError_t e = launch_pdl(degridder_tcw_fused_kernel, (unsigned)set.count, DNT, D_SMEM, (cudaStream_t)stream,
                                     pdl, g, set.idx, set.first, (const float4 *)grid, flags, (const float4 *)aterms,
                                     taper, (float4 *)vis_out);
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "tensor-core degridder job launch");
}


idg_status launch_degridder_tcw(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                const void *aterms, const float *taper, void *vis_out, void *stream) {
    if (g.L != DL) return fail(IDG_ERR_UNSUPPORTED, "the tensor-core degridder is built for L = 32");
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute(degridder_tcw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, D_SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core degridder smem attribute");
    degridder_tcw_kernel<<<(unsigned)set.count, DNT, D_SMEM, s>>>(g, set.idx, set.first, (const float4 *)sub, flags,
                                                                   (const float4 *)aterms, taper, (float4 *)vis_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core degridder launch");
    return IDG_OK;
}

idg_status read_tcd_error(int *code) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(code, g_tcd_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tcd_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    return IDG_OK;
}

}  // namespace idg
