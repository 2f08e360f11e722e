// Gridder on the 5th-generation tensor cores (tcgen05), L = 32.
//
// The direct sum of Eq. (ShiftedDirectImaging) is a complex contraction over
// the visibilities of a subgrid:  I[pix][pol] = sum_k E[pix][k] V[k][pol],
// E = exp(+i phi).  As a real GEMM, A[pix][2k + r] = (Re E, Im E)[r] and
//   B[2k][2q] = Re V_q,  B[2k+1][2q] = -Im V_q,  B[2k][2q+1] = Im V_q,  B[2k+1][2q+1] = Re V_q,
// so D = A B holds (Re, Im) of the four polarisations in 8 columns.
//
// Precision.  E is formed on the CUDA cores (phase, sin/cos) and split into
// FP16 parts E = E_hi + E_lo (E_hi = fp16(E), E_lo = fp16(E - E_hi), the
// difference exact); V, scaled by a power of two per subgrid so that its
// largest component lies in [2^9, 2^10), is split the same way.  One B tile
// [V_hi | V_lo] (N = 16) serves two MMAs per 128-pixel tile and group of 8
// visibilities (K = 16): E_hi [V_hi | V_lo] and E_lo [V_hi | V_lo] into the
// same accumulator, whose columns 0..7 + 8..15 are the result.  The tensor
// cores accumulate in FP32 without rounding to nearest (each step can lose up
// to an ulp, biased towards zero), so every WS_FOLD groups (256 visibilities,
// one staged batch, so that the fold and the batch barrier fall together) the
// accumulators are added into an FP32 sum in shared memory and restarted.
//
// Schedule.  One CTA per subgrid: eight producer warps form the phasors and
// write their FP16 hi/lo rows straight into tensor memory (tcgen05.st; warp w
// owns lanes 32 (w % 4) ..); a ninth warp issues the MMAs with A read from
// tensor memory.  Hand-off is by mbarriers, not CTA barriers:
// full[h] (8 producer arrivals) -> MMAs -> commit -> empty[h].
// Tensor memory per CTA (256 columns, two CTAs per SM):
//   columns   0..127  accumulators, tile mt at 16 mt
//   columns 128..255  two A stages of 4 tiles, tile lt of stage h at 128 + 64 h + 16 lt
//                     (8 columns hi, 8 lo; column c holds k = 2c and 2c + 1)
// At a fold the producers wait for the MMAs, add the accumulators into the
// shared-memory sum and release the MMA warp (folded), which restarts them
// from zero.  Every wait is bounded; after a failed wait a thread skips every
// later wait, so control flow stays uniform and the kernel ends; the error word
// is set and no output is written.
#include "batch_jobs.cuh"
#include "device_common.cuh"
#include "fft_impl.cuh"
#include "tc_common.cuh"

namespace idg {

// device error word of the tensor-core gridder (0 = ok); read and cleared by
// idg_device_errors
__device__ int g_tc_error = 0;

namespace {

using namespace dev;
using namespace tc;

constexpr int TC_L = 32;
constexpr int TC_PIX = TC_L * TC_L;              // 1024
constexpr int B_TILE = kTile16;                  // 512 B: 16 rows x 16 FP16
constexpr int FOLD_BYTES = 8 * TC_PIX * 4;       // [8][1024] FP32
constexpr int WS_NP = 256;                       // producer threads
constexpr int WS_NT = WS_NP + 32;                // + the MMA warp
constexpr int WS_VB = 256;                       // visibilities per staged batch (one per producer)
constexpr int WS_GROUPS = WS_VB / 8;
constexpr int WS_FOLD = 32;                      // groups between folds = one batch (two accumulations per group)
constexpr int WS_COLS = 256;
constexpr int WS_B_BATCH = WS_GROUPS * B_TILE;   // 16 KB
constexpr int WS_SMEM = 2 * WS_B_BATCH + 2 * WS_VB * 16 + FOLD_BYTES;
constexpr int FFT_P = TC_L + 1;                  // padded row pitch of the transform planes (float2)
static_assert(4 * TC_L * FFT_P * 8 <= 2 * WS_B_BATCH + 2 * WS_VB * 16, "transform planes fit over the B buffers");

__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" :: "n"(WS_NP) : "memory"); }

// One subgrid d of geometry g (taper and A-terms applied): into o[L][L][4], or with
// FUSED transformed in shared memory and added into the grid o[layer][N][N][4]
// (Algorithm 1: direct sum, image-domain kernel, "FFT", add to the master grid).
template <bool FUSED>
__device__ __forceinline__ void gridder_tcw_body(const Geometry &g, const DevSubgrid d,
                                                 const float4 *__restrict__ vis, const uint8_t *__restrict__ flags,
                                                 const float4 *__restrict__ aterms, const float *__restrict__ taper,
                                                 float4 *__restrict__ o) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;                                         // 2 batches x 4 KB
    float4 *s_coef = (float4 *)(smem + 2 * WS_B_BATCH);         // 2 batches x 64
    float *s_fold = (float *)(smem + 2 * WS_B_BATCH + 2 * WS_VB * 16);   // [8][1024]
    float2 *s_fft = (float2 *)smem;                 // FUSED epilogue: [4][L][L + 1], over the B and coefficient buffers
    bool failed_out = false;                        // a producer's bounded wait gave up
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[2], s_empty[2], s_foldbar, s_folded, s_drain;
    __shared__ float s_red[8];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == 8;
    const int total_groups = (d.kp + 7) / 8;
    const int n_batches = (d.kp + WS_VB - 1) / WS_VB;

    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "n"(WS_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int h = 0; h < 2; ++h) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" :: "r"(smem_u32(&s_full[h])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_empty[h])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_foldbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" :: "r"(smem_u32(&s_folded)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_drain)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // per-subgrid scale of V (producers)
    float vmax = 0.0f;
    if (!mma_warp)
        for (int k = tid; k < d.kp; k += WS_NP) {
            int t, c;
            const size_t vi = vis_index(g, d, k, t, c);
            if (!(flags && flags[vi])) {
                const float4 a = vis[2 * vi], b = vis[2 * vi + 1];
                vmax = fmaxf(vmax, fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                                         fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w)))));
            }
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0 && !mma_warp) s_red[warp] = vmax;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (mma_warp) {
        if (lane == 0) {
            bool failed = false;
            uint32_t folded_phase = 0;
            for (int gc = 0; gc < total_groups; ++gc) {
                const uint8_t *Bt = sB + ((gc / WS_GROUPS) & 1) * WS_B_BATCH + (gc % WS_GROUPS) * B_TILE;
                const uint64_t db = smem_desc(smem_u32(Bt));
                if (gc > 0 && gc % WS_FOLD == 0) {        // the producers have read the accumulators
                    wait_or_fail(smem_u32(&s_folded), folded_phase, failed);
                    folded_phase ^= 1u;
                }
                const uint32_t acc_hi = (gc % WS_FOLD == 0) ? 0u : 1u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    wait_or_fail(smem_u32(&s_full[h]), (uint32_t)(gc & 1), failed);
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int lt = 0; lt < 4; ++lt) {
                        const uint32_t dt = tmem + (uint32_t)(16 * (4 * h + lt));
                        const uint32_t at = tmem + (uint32_t)(128 + 64 * h + 16 * lt);
                        mma_ta(dt, at, db, acc_hi);
                        mma_ta(dt, at + 8, db, 1u);
                    }
                    commit(smem_u32(&s_empty[h]));
                }
                if ((gc + 1) % WS_FOLD == 0 || gc + 1 == total_groups) commit(smem_u32(&s_foldbar));
            }
            if (total_groups == 0) commit(smem_u32(&s_foldbar));
            commit(smem_u32(&s_drain));
            bool drained = false;
            wait_or_fail(smem_u32(&s_drain), 0u, drained);     // bounded: let own MMAs finish before the free
            if (failed) atomicExch(&g_tc_error, 1);
            failed_out = failed;
        }
    } else {
        const int q4 = warp & 3, ltw = warp >> 2;
        float m = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) m = fmaxf(m, s_red[w]);
        int e2 = 0;
        if (m > 0.0f) frexpf(m, &e2);
        const float scale = ldexpf(1.0f, 10 - e2);
        const float inv_scale = ldexpf(1.0f, e2 - 10);
        // pixel s = 2 h + i of this thread: tile 4 h + ltw + 2 i, row 32 q4 + lane
        float Yv[4], NP[4];
        int PIX[4];
        const float Xc = (float)(lane - TC_L / 2);   // pixel 128 mt + 32 q4 + lane lies in column lane
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
            const int mt = 4 * (s4 >> 1) + ltw + 2 * (s4 & 1);
            const int pix = 128 * mt + 32 * q4 + lane;
            PIX[s4] = pix;
            Yv[s4] = (float)((pix >> 5) - TC_L / 2);
            NP[s4] = g.nprime[pix];
        }
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16);
        bool failed = false;
        uint32_t fold_phase = 0;
        int n_folds = 0;
        for (int bt = 0; bt < n_batches; ++bt) {
            const int bb = bt & 1;
            uint8_t *sBb = sB + bb * WS_B_BATCH;
            float4 *coef = s_coef + bb * WS_VB;
            if (tid < WS_VB) {      // stage visibility tid of the batch: coefficients and its B column pairs
                const int k = bt * WS_VB + tid;
                float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (k < d.kp) {
                    int t, c;
                    const size_t vi = vis_index(g, d, k, t, c);
                    const PhaseCoef pc = phase_coef(g, d, t, c);
                    cf = make_float4(pc.a, pc.b, pc.c, 0.f);
                    if (!(flags && flags[vi])) {
                        const float4 a = vis[2 * vi], b = vis[2 * vi + 1];
                        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                    }
                }
                coef[tid] = cf;
                const int grp = tid >> 3, j = tid & 7;
                uint8_t *Bt = sBb + grp * B_TILE;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float re = v[2 * q] * scale, im = v[2 * q + 1] * scale;
                    const __half re_h = __float2half_rn(re), im_h = __float2half_rn(im);
                    const __half re_l = __float2half_rn(re - __half2float(re_h));
                    const __half im_l = __float2half_rn(im - __half2float(im_h));
                    *(__half *)(Bt + kmaj_off(2 * q, 2 * j)) = re_h;
                    *(__half *)(Bt + kmaj_off(2 * q, 2 * j + 1)) = __hneg(im_h);
                    *(__half *)(Bt + kmaj_off(2 * q + 1, 2 * j)) = im_h;
                    *(__half *)(Bt + kmaj_off(2 * q + 1, 2 * j + 1)) = re_h;
                    *(__half *)(Bt + kmaj_off(8 + 2 * q, 2 * j)) = re_l;
                    *(__half *)(Bt + kmaj_off(8 + 2 * q, 2 * j + 1)) = __hneg(im_l);
                    *(__half *)(Bt + kmaj_off(8 + 2 * q + 1, 2 * j)) = im_l;
                    *(__half *)(Bt + kmaj_off(8 + 2 * q + 1, 2 * j + 1)) = re_l;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            producers_sync();
            const int ng = min(WS_GROUPS, total_groups - bt * WS_GROUPS);
            for (int gi = 0; gi < ng; ++gi) {
                const int gc = bt * WS_GROUPS + gi;
                // the thread's four pixels share the column x = lane, so a X is formed once per visibility
                float aX[8], cb[8], cc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 cf = coef[gi * 8 + j];
                    aX[j] = cf.x * Xc;
                    cb[j] = cf.y;
                    cc[j] = cf.z;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (gc >= 1) wait_or_fail(smem_u32(&s_empty[h]), (uint32_t)((gc - 1) & 1), failed);
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int s4 = 2 * h + i;
                        uint32_t e[16];      // 8 hi (k = 2j, 2j + 1 = cos, sin of visibility j), then 8 lo
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float phase = fmaf(cb[j], Yv[s4], fmaf(cc[j], NP[s4], aX[j]));
                            float sn, cs;
                            __sincosf(phase, &sn, &cs);
                            split_e(cs, sn, e[j], e[8 + j]);
                        }
                        tmem_st16(lane_base + (uint32_t)(128 + 64 * h + 16 * (ltw + 2 * i)), e);
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&s_full[h]));
                }
                if ((gc + 1) % WS_FOLD == 0 && gc + 1 < total_groups) {
                    wait_or_fail(smem_u32(&s_foldbar), fold_phase, failed);
                    fold_phase ^= 1u;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4) {
                        uint32_t r[16];
                        const int mt = 4 * (s4 >> 1) + ltw + 2 * (s4 & 1);
                        tmem_ld16(lane_base + (uint32_t)(16 * mt), r);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float v = __uint_as_float(r[c]) + __uint_as_float(r[8 + c]);
                            float &f = s_fold[c * TC_PIX + PIX[s4]];
                            f = n_folds ? f + v : v;
                        }
                    }
                    ++n_folds;
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&s_folded));
                }
            }
            producers_sync();     // every producer is done with this batch's coefficients
        }
        wait_or_fail(smem_u32(&s_foldbar), fold_phase, failed);   // the last accumulation (or none)
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (failed) {
            if (lane == 0) atomicExch(&g_tc_error, 1);
        } else {
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
                const int pix = PIX[s4];
                const int mt = 4 * (s4 >> 1) + ltw + 2 * (s4 & 1);
                uint32_t r[16];
                tmem_ld16(lane_base + (uint32_t)(16 * mt), r);
                float sv[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float v = total_groups ? __uint_as_float(r[c]) + __uint_as_float(r[8 + c]) : 0.0f;
                    if (n_folds) v += s_fold[c * TC_PIX + pix];
                    sv[c] = v * inv_scale;
                }
                M22 P;
#pragma unroll
                for (int c = 0; c < 4; ++c) P.m[c] = make_float2(sv[2 * c], sv[2 * c + 1]);
                if (aterms) {
                    const size_t base = ((size_t)d.slot * g.n_stations) * TC_PIX;
                    const M22 Ap = load_m22(aterms + 2 * (base + (size_t)d.st_p * TC_PIX + pix));
                    const M22 Aq = load_m22(aterms + 2 * (base + (size_t)d.st_q * TC_PIX + pix));
                    P = herm_mul_mul(Ap, P, Aq);
                }
                if (FUSED) {
                    // the (-1)^(x+y) centring factor, into the transform planes
                    const int x = pix & (TC_L - 1), y = pix >> 5;
                    const float tw = ((x + y) & 1) ? -taper[pix] : taper[pix];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        s_fft[(q * TC_L + y) * FFT_P + x] = make_float2(tw * P.m[q].x, tw * P.m[q].y);
                } else {
                    const float tw = taper[pix];
                    o[2 * pix] = make_float4(tw * P.m[0].x, tw * P.m[0].y, tw * P.m[1].x, tw * P.m[1].y);
                    o[2 * pix + 1] = make_float4(tw * P.m[2].x, tw * P.m[2].y, tw * P.m[3].x, tw * P.m[3].y);
                }
            }
        }
        failed_out = failed;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (FUSED) {
        // every thread: transform the planes, then add with the (-1)^(i+j) factor and 1/L^2
        if (!__syncthreads_or(failed_out)) {
            fft2_planar<TC_L, -1>(s_fft, tid, WS_NT);
            const float inv = 1.0f / (float)TC_PIX;
            float4 *dst = o + (size_t)d.layer * g.N * g.N * 2;
            for (int pix = tid; pix < TC_PIX; pix += WS_NT) {
                const int i = pix >> 5, j = pix & (TC_L - 1);
                const float sg = ((i + j) & 1) ? -inv : inv;
                const float2 p0 = s_fft[(0 * TC_L + i) * FFT_P + j], p1 = s_fft[(1 * TC_L + i) * FFT_P + j];
                const float2 p2 = s_fft[(2 * TC_L + i) * FFT_P + j], p3 = s_fft[(3 * TC_L + i) * FFT_P + j];
                const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
                red_add_f4(dst + 2 * gp, make_float4(sg * p0.x, sg * p0.y, sg * p1.x, sg * p1.y));
                red_add_f4(dst + 2 * gp + 1, make_float4(sg * p2.x, sg * p2.y, sg * p3.x, sg * p3.y));
            }
        }
    }
    __syncthreads();
    if (mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(WS_COLS));
}

// one CTA per subgrid of one plan (plan index idx[b] or first + b)
__global__ void __launch_bounds__(WS_NT, 2)
gridder_tcw_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                   const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                   const float *__restrict__ taper, float4 *__restrict__ out) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    gridder_tcw_body<false>(g, g.sub[sid], vis, flags, aterms, taper, out + (size_t)blockIdx.x * TC_PIX * 2);
}

// fused: one CTA per subgrid, transformed and added into grid (accumulated)
__global__ void __launch_bounds__(WS_NT, 2)
gridder_tcw_fused_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                         const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                         const float *__restrict__ taper, float4 *__restrict__ grid) {
    allow_dependents();
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    gridder_tcw_body<true>(g, g.sub[sid], vis, flags, aterms, taper, grid);
    complete_after_primary();
}

}  // namespace

idg_status launch_gridder_tcw_fused(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *grid, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (g.L != TC_L) return fail(IDG_ERR_UNSUPPORTED, "the tensor-core gridder is built for L = 32");
    if (set.count <= 0) return IDG_OK;
    cudaError_t e = cudaFuncSetAttribute(gridder_tcw_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WS_SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core gridder smem attribute");
    gridder_tcw_fused_kernel<<<(unsigned)set.count, WS_NT, WS_SMEM, s>>>(g, set.idx, set.first, (const float4 *)vis,
                                                                          flags, (const float4 *)aterms, taper,
                                                                          (float4 *)grid);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core fused gridder launch");
    return IDG_OK;
}

cudaError_t prepare_gridder_tcw_batch() {
    return cudaFuncSetAttribute(gridder_tcw_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WS_SMEM);
}

// a batch's launch of the fused kernel over one job's items (the shared-memory attribute
// is set by prepare_tcw_batch_kernels, outside graph capture); pdl: see launch_pdl
idg_status launch_gridder_tcw_job(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                  const void *aterms, const float *taper, void *grid, void *stream, bool pdl) {
    if (g.L != TC_L) return fail(IDG_ERR_UNSUPPORTED, "the tensor-core gridder is built for L = 32");
    if (set.count <= 0) return IDG_OK;
    const cudaError_t e = launch_pdl(gridder_tcw_fused_kernel, (unsigned)set.count, WS_NT, WS_SMEM, (cudaStream_t)stream,
                                     pdl, g, set.idx, set.first, (const float4 *)vis, flags, (const float4 *)aterms,
                                     taper, (float4 *)grid);
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "tensor-core gridder job launch");
}


idg_status launch_gridder_tcw(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *out, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (g.L != TC_L) return fail(IDG_ERR_UNSUPPORTED, "the tensor-core gridder is built for L = 32");
    if (set.count <= 0) return IDG_OK;
    cudaError_t e = cudaFuncSetAttribute(gridder_tcw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WS_SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core gridder smem attribute");
    gridder_tcw_kernel<<<(unsigned)set.count, WS_NT, WS_SMEM, s>>>(g, set.idx, set.first, (const float4 *)vis, flags,
                                                                    (const float4 *)aterms, taper, (float4 *)out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core gridder launch");
    return IDG_OK;
}

idg_status read_device_errors(int *code, void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int zero = 0, mine = 0, dft = 0;
    e = cudaMemcpyFromSymbol(&mine, g_tc_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    int deg = 0, sep = 0, sepd = 0, self = 0, cl = 0;
    idg_status st = read_dft_error(&dft);
    if (st == IDG_OK) st = read_tcd_error(&deg);
    if (st == IDG_OK) st = read_sep_error(&sep);
    if (st == IDG_OK) st = read_sepd_error(&sepd);
    if (st == IDG_OK) st = read_selftest_error(&self);
    if (st == IDG_OK) st = read_classical_error(&cl);
    if (st != IDG_OK) return st;
    *code = mine | dft | deg | sep | sepd | self | cl;     // bit 0: a wait gave up; bit 1: a device check
    return IDG_OK;
}

}  // namespace idg
