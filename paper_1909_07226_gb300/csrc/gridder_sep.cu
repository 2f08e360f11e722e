// Separable gridder on the tensor cores (tcgen05), L = 32.
//
// The subgrid image of Eq. (ShiftedDirectImaging) is
//   I_q(x, y) = sum_k V_kq exp(i (a_k X + b_k Y + c_k n'(x, y))),
// with X = x - L/2, Y = y - L/2 and c_k = 2 pi (w_k - w0).  Splitting
// n'(x, y) = s(x) + t(y) + r(x, y), s and t the row and column through the
// centre pixel, the phasor factors into
//   Ex_k(x) = exp(i (a_k X + c_k s(x))),  Ey_k(y) = exp(i (b_k Y + c_k t(y))),
// times exp(i c_k r(x, y)).  The remainder r is fourth order in (l, m); where
// theta = max |c_k| max |r| is small (the plan checks theta <= 1.38e-3, so that
// theta^2 / 2 <= 2^-20) the factor is taken to first order,
// exp(i c r) = 1 + i c r + O(theta^2 / 2), so
//   I_q(x, y) = S0_q(x, y) + i r(x, y) S1_q(x, y),
//   S_mq(x, y) = sum_k [V_kq Ey_k(y)] [c_k^m Ex_k(x)],   m = 0, 1,
// a complex matrix product over the visibilities: rows (q, y), 128 of them,
// columns (m, x), 64.  Per visibility the CUDA cores form 128 + 64 phasor
// products instead of the L^2 = 1024 of the direct sum, and the tensor cores
// do the contraction.
//
// GEMM.  A[(q, y)][2 k + r] = (Re, Im)[r] of V_kq Ey_k(y) (tensor memory);
// B holds the real 2 x 2 embedding of beta = (c_k sigma)^m Ex_k(x): row
// (m, x, re) = (Re beta, -Im beta), row (m, x, im) = (Im beta, Re beta) over
// K = (k, r), so D[(q, y)][(m, x, re/im)] = (Re, Im) S_mq.  sigma is a power of
// two with max |c_k| sigma <= 1.
//
// Precision.  Both operands are split into FP16 hi + lo parts (A after a
// power-of-two scale per subgrid).  The m = 0 block takes A_hi B_hi +
// A_hi B_lo + A_lo B_hi; the m = 1 block, which contributes at most theta
// relative, takes A_hi B_hi only.  One MMA of N = 192 computes
// A_hi [B_hi (128 rows) | B_lo (m = 0, 64 rows)], a second of N = 64 adds
// A_lo B_hi (m = 0) to the correction columns.  The tensor cores accumulate
// without rounding to nearest, so every FOLD groups of 8 visibilities the
// accumulators are added into FP32 sums in shared memory (RN) and restarted;
// two accumulator sets alternate so the MMAs never wait for a fold.
//
// Schedule.  One CTA per subgrid, one CTA per SM: sixteen producer warps and
// one MMA warp.  A stage is four groups of 8 visibilities: per stage each
// producer writes the 8 A entries of its row (q = warp % 4, y = lane) for
// group warp / 4 into tensor memory (one 16-column store) and one B entry pair
// (x, re/im, j) per group into shared memory (one core matrix per warp and
// store, no bank conflicts), twelve independent phasor chains per thread.
// Visibilities are staged 512 at a time; the next batch is loaded into
// registers while the current one is processed.
// Tensor memory (512 columns):
//   accumulator set p at 192 p: main (m, x, re/im) 0..127, correction (m = 0) 128..191
//   A stage s at 384 + 64 s, group i at + 16 i: 8 columns hi, 8 lo
// Every wait is bounded; after a failed wait a thread skips every later wait,
// the error word is set and no output is written.
#include "batch_jobs.cuh"
#include "device_common.cuh"
#include "fft_impl.cuh"
#include "tc_common.cuh"

namespace idg {

// device error word of the separable gridder (0 = ok); read and cleared by
// idg_device_errors
__device__ int g_sep_error = 0;

namespace {

using namespace dev;
using namespace tc;

constexpr int SL = 32;
constexpr int SPIX = SL * SL;
constexpr int NPW = 16;                        // producer warps
constexpr int NP = NPW * 32;                   // producer threads
constexpr int NT = NP + 32;                    // + the MMA warp
constexpr int VB = NP;                         // visibilities per staged batch (one per producer)
constexpr int GB = VB / 8;                     // groups per batch
constexpr int FOLD = 64;                       // groups per accumulation period
constexpr int SG = 4;                          // groups of 8 visibilities per stage
constexpr int STAGES = 2;
constexpr int B_GROUP = 192 * 32;              // B of one group: 192 rows x 16 K FP16 (hi 128 rows, then lo 64)
constexpr int B_STAGE = SG * B_GROUP;
constexpr int COEF_OFF = STAGES * B_STAGE;     // [2][VB] float4 (a, b, c, 0)
constexpr int VIS_OFF = COEF_OFF + 2 * VB * 16;   // [2][VB][4] float2 (scaled V)
constexpr int FOLD_OFF = VIS_OFF + 2 * VB * 32;   // [32][NP] float: folded sums of each producer
constexpr int SEP_SMEM = FOLD_OFF + 32 * NP * 4;
constexpr int FFT_P = SL + 1;
constexpr uint32_t ACC_STRIDE = 192, A_COL = 384;
constexpr uint32_t IDESC_N192 = idesc_m128(192), IDESC_N64 = idesc_m128(64);
static_assert(4 * SL * FFT_P * 8 <= FOLD_OFF, "transform planes fit over the stage buffers");
static_assert(A_COL + 16 * SG * STAGES <= 512, "tensor memory");
static_assert(FOLD % SG == 0 && GB % SG == 0, "periods and batches are whole stages");

__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" :: "n"(NP) : "memory"); }

// One subgrid d of geometry g (taper and A-terms applied): into o[L][L][4], or with
// FUSED transformed in shared memory and added into the grid o[layer][N][N][4]
// (Algorithm 1: direct sum, image-domain kernel, "FFT", add to the master grid).
template <bool FUSED>
__device__ __forceinline__ void gridder_sep_body(const Geometry &g, const DevSubgrid d,
                                                 const float4 *__restrict__ vis, const uint8_t *__restrict__ flags,
                                                 const float4 *__restrict__ aterms, const float *__restrict__ taper,
                                                 float4 *__restrict__ o) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;
    float4 *s_coef = (float4 *)(smem + COEF_OFF);
    float2 *s_vis = (float2 *)(smem + VIS_OFF);
    float2 *s_fft = (float2 *)smem;                 // [4][L][L + 1] after the main loop
    float *s_fold = (float *)(smem + FOLD_OFF);     // [32][NP]: m = 0 sums (16), then m = 1 (16)
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[STAGES], s_empty[STAGES], s_foldbar[2], s_folded[2], s_drain;
    __shared__ float s_red[NPW];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == NPW;
    const int total_groups = (d.kp + 7) / 8;
    const int n_batches = (d.kp + VB - 1) / VB;
    const int n_per = (total_groups + FOLD - 1) / FOLD;

    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "n"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&s_full[s]), NPW);
            mbar_init(smem_u32(&s_empty[s]), 1);
        }
        for (int p = 0; p < 2; ++p) {
            mbar_init(smem_u32(&s_foldbar[p]), 1);
            mbar_init(smem_u32(&s_folded[p]), NPW);
        }
        mbar_init(smem_u32(&s_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // per-subgrid scale of V (producers)
    float vmax = 0.0f;
    if (!mma_warp)
        for (int k = tid; k < d.kp; k += NP) {
            int t, c;
            const size_t vi = vis_index(g, d, k, t, c);
            if (!(flags && flags[vi])) {
                const float4 a = vis[2 * vi], b = vis[2 * vi + 1];
                vmax = fmaxf(vmax, fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                                         fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w)))));
            }
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    if (lane == 0 && !mma_warp) s_red[warp] = vmax;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    bool failed = false;
    float inv_scale = 1.0f;
    const int q = warp & 3, sl = warp >> 2;         // lane quarter (polarisation) and column slice of the fold

    if (mma_warp) {
        if (lane == 0) {
            const int n_stages = (total_groups + SG - 1) / SG;
            for (int st = 0; st < n_stages; ++st) {
                const int s = st % STAGES;
                wait_or_fail(smem_u32(&s_full[s]), (uint32_t)((st / STAGES) & 1), failed);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int ng = min(SG, total_groups - st * SG);
                for (int i = 0; i < ng; ++i) {
                    const int gc = st * SG + i, P = gc / FOLD, p = P & 1;
                    const bool first = gc % FOLD == 0;
                    if (first && P >= 2) {
                        wait_or_fail(smem_u32(&s_folded[p]), (uint32_t)(((P - 2) >> 1) & 1), failed);
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    }
                    const uint64_t db = smem_desc(smem_u32(sB + s * B_STAGE + i * B_GROUP));
                    const uint32_t at = tmem + A_COL + 64u * (uint32_t)s + 16u * (uint32_t)i;
                    const uint32_t dt = tmem + ACC_STRIDE * (uint32_t)p;
                    mma_ta_i(dt, at, db, IDESC_N192, first ? 0u : 1u);
                    mma_ta_i(dt + 128u, at + 8u, db, IDESC_N64, 1u);
                    if (gc % FOLD == FOLD - 1 || gc == total_groups - 1) commit(smem_u32(&s_foldbar[p]));
                }
                commit(smem_u32(&s_empty[s]));
            }
            commit(smem_u32(&s_drain));
            bool drained = false;
            wait_or_fail(smem_u32(&s_drain), 0u, drained);     // bounded: let own MMAs finish before the free
        }
        failed = __shfl_sync(0xffffffffu, failed, 0);
    } else {
        float m = 0.0f;
#pragma unroll
        for (int w = 0; w < NPW; ++w) m = fmaxf(m, s_red[w]);
        int e2 = 0;
        if (m > 0.0f) frexpf(m, &e2);
        const float scale = ldexpf(1.0f, 10 - e2);
        inv_scale = ldexpf(1.0f, e2 - 10);
        // A rows (q, y = lane) of group warp / 4 of each stage
        const int ga = warp >> 2;
        const float Yv = (float)(lane - SL / 2);
        const float ty = g.sep[SL + lane];
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        // B entries: x = 4 (warp & 7) + (lane & 3), re/im = (lane >> 2) & 1, j = 4 (warp >> 3) + (lane >> 3)
        const int xb = 4 * (warp & 7) + (lane & 3), cb = (lane >> 2) & 1, jb = 4 * (warp >> 3) + (lane >> 3);
        const float Xv = (float)(xb - SL / 2);
        const float sx = g.sep[xb];
        const float csig = g.c_scale;
        const int n0 = 2 * xb + cb;
        const uint32_t off_h0 = kmaj_off(n0, 2 * jb), off_h1 = kmaj_off(64 + n0, 2 * jb);
        const uint32_t off_l0 = kmaj_off(128 + n0, 2 * jb);

        // staging: visibility tid of batch b, loaded into registers one batch ahead
        float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
        double pu = 0.0, pv = 0.0, pw = 0.0, psc = 0.0;
        bool pin = false, pflag = false;
        auto load_batch = [&](int b) {
            const int k = b * VB + tid;
            pin = k < d.kp;
            pflag = false;
            if (pin) {
                int t, c;
                const size_t vi = vis_index(g, d, k, t, c);
                const double *xw = g.uvw + ((size_t)d.bl * g.n_t + t) * 3;
                pu = xw[0];
                pv = xw[1];
                pw = xw[2];
                psc = g.scale[c];
                pflag = flags && flags[vi];
                if (!pflag) {
                    pa = vis[2 * vi];
                    pb = vis[2 * vi + 1];
                }
            }
        };
        auto store_batch = [&](int bb) {
            float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 v[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (pin) {
                cf.x = (float)((pu * psc - d.u0) * g.k_uv);
                cf.y = (float)((pv * psc - d.v0) * g.k_uv);
                cf.z = (float)((pw * psc - d.w0) * 6.283185307179586476925286766559);
                if (!pflag) {
                    v[0] = make_float2(pa.x * scale, pa.y * scale);
                    v[1] = make_float2(pa.z * scale, pa.w * scale);
                    v[2] = make_float2(pb.x * scale, pb.y * scale);
                    v[3] = make_float2(pb.z * scale, pb.w * scale);
                }
            }
            s_coef[bb * VB + tid] = cf;
            float4 *dv = (float4 *)(s_vis + (size_t)(bb * VB + tid) * 4);
            dv[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
            dv[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
        };

        auto fold = [&](int P) {
            const int p = P & 1;
            wait_or_fail(smem_u32(&s_foldbar[p]), (uint32_t)((P >> 1) & 1), failed);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // this thread's row (q, y = lane), columns of x in [8 sl, 8 sl + 8): sums at s_fold[c][tid]
            uint32_t r[16], rc[16];
            const uint32_t base = lane_base + ACC_STRIDE * (uint32_t)p + 16u * (uint32_t)sl;
            tmem_ld16(base, r);                      // main, m = 0
            tmem_ld16(base + 128u, rc);              // correction, m = 0
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float v = __uint_as_float(r[c]) + __uint_as_float(rc[c]);
                float &f = s_fold[c * NP + tid];
                f = P ? f + v : v;
            }
            tmem_ld16(base + 64u, r);                // main, m = 1
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float &f = s_fold[(16 + c) * NP + tid];
                f = P ? f + __uint_as_float(r[c]) : __uint_as_float(r[c]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_folded[p]));
        };

        load_batch(0);
        store_batch(0);
        producers_sync();
        int next_fold = 0;
        for (int b = 0; b < n_batches; ++b) {
            const int bb = b & 1;
            if (b + 1 < n_batches) load_batch(b + 1);
            const float4 *coef = s_coef + bb * VB;
            const float2 *vb = s_vis + (size_t)bb * VB * 4;
            const int nst = (min(GB, total_groups - b * GB) + SG - 1) / SG;
            for (int si = 0; si < nst; ++si) {
                const int st = b * (GB / SG) + si;
                const int s = st % STAGES;
                if (st >= STAGES) wait_or_fail(smem_u32(&s_empty[s]), (uint32_t)(((st / STAGES) - 1) & 1), failed);
                // B entry pairs, one per group: beta = Ex_k(x) (m = 0, hi and lo) and c_k sigma Ex_k(x) (m = 1, hi)
                uint8_t *Bs = sB + s * B_STAGE;
#pragma unroll
                for (int i = 0; i < SG; ++i) {
                    const float4 cf = coef[8 * (SG * si + i) + jb];
                    float sn, cs;
                    __sincosf(fmaf(cf.z, sx, cf.x * Xv), &sn, &cs);
                    const float vx = cb ? sn : cs, vy = cb ? cs : -sn;
                    uint32_t h0, l0;
                    split_e(vx, vy, h0, l0);
                    const float cz = cf.z * csig;
                    const uint32_t h1 = pack_f16x2(cz * vx, cz * vy);
                    *(uint32_t *)(Bs + i * B_GROUP + off_h0) = h0;
                    *(uint32_t *)(Bs + i * B_GROUP + off_h1) = h1;
                    *(uint32_t *)(Bs + i * B_GROUP + off_l0) = l0;
                }
                // A entries of group ga: V_kq Ey_k(y) for its 8 visibilities
                uint32_t e[16];
                const int kb = 8 * (SG * si + ga);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 cf = coef[kb + j];
                    float sn, cs;
                    __sincosf(fmaf(cf.z, ty, cf.y * Yv), &sn, &cs);
                    const float2 v = vb[(kb + j) * 4 + q];
                    split_e(fmaf(v.x, cs, -v.y * sn), fmaf(v.x, sn, v.y * cs), e[j], e[8 + j]);
                }
                tmem_st16(lane_base + A_COL + 64u * (uint32_t)s + 16u * (uint32_t)ga, e);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&s_full[s]));
                // fold period next_fold half-way through the following one
                if (next_fold < n_per - 1 && (st + 1) * SG == (next_fold + 1) * FOLD + FOLD / 2) {
                    fold(next_fold);
                    ++next_fold;
                }
            }
            if (b + 1 < n_batches) {
                store_batch(bb ^ 1);
                producers_sync();
            }
        }
        while (next_fold < n_per) {
            fold(next_fold);
            ++next_fold;
        }
        if (failed && lane == 0) atomicExch(&g_sep_error, 1);
        producers_sync();      // every producer is past the stage and batch buffers
        if (!failed) {
            // I = S0 + i r S1 / sigma, unscaled, into the polarisation planes
            const float rs = 1.0f / csig;
#pragma unroll
            for (int xi = 0; xi < 8; ++xi) {
                const int x = 8 * sl + xi;
                const float rr = g.sep[2 * SL + lane * SL + x] * rs;
                float s0r = 0.f, s0i = 0.f, s1r = 0.f, s1i = 0.f;
                if (n_per) {
                    s0r = s_fold[(2 * xi) * NP + tid];
                    s0i = s_fold[(2 * xi + 1) * NP + tid];
                    s1r = s_fold[(16 + 2 * xi) * NP + tid];
                    s1i = s_fold[(17 + 2 * xi) * NP + tid];
                }
                const float re = fmaf(-rr, s1i, s0r) * inv_scale;
                const float im = fmaf(rr, s1r, s0i) * inv_scale;
                s_fft[(q * SL + lane) * FFT_P + x] = make_float2(re, im);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (!__syncthreads_or(failed)) {
        // image-domain kernel per pixel: taper * A_p^H I A_q (with the centring factor when FUSED)
        for (int pix = tid; pix < SPIX; pix += NT) {
            const int y = pix >> 5, x = pix & (SL - 1);
            M22 P;
#pragma unroll
            for (int c = 0; c < 4; ++c) P.m[c] = s_fft[(c * SL + y) * FFT_P + x];
            if (aterms) {
                const size_t base = ((size_t)d.slot * g.n_stations) * SPIX;
                const M22 Ap = load_m22(aterms + 2 * (base + (size_t)d.st_p * SPIX + pix));
                const M22 Aq = load_m22(aterms + 2 * (base + (size_t)d.st_q * SPIX + pix));
                P = herm_mul_mul(Ap, P, Aq);
            }
            if (FUSED) {
                const float tw = ((x + y) & 1) ? -taper[pix] : taper[pix];
#pragma unroll
                for (int c = 0; c < 4; ++c) s_fft[(c * SL + y) * FFT_P + x] = make_float2(tw * P.m[c].x, tw * P.m[c].y);
            } else {
                const float tw = taper[pix];
                o[2 * pix] = make_float4(tw * P.m[0].x, tw * P.m[0].y, tw * P.m[1].x, tw * P.m[1].y);
                o[2 * pix + 1] = make_float4(tw * P.m[2].x, tw * P.m[2].y, tw * P.m[3].x, tw * P.m[3].y);
            }
        }
        if (FUSED) {
            __syncthreads();
            fft2_planar<SL, -1>(s_fft, tid, NT);
            const float inv = 1.0f / (float)SPIX;
            float4 *dst = o + (size_t)d.layer * g.N * g.N * 2;
            for (int pix = tid; pix < SPIX; pix += NT) {
                const int i = pix >> 5, j = pix & (SL - 1);
                const float sg = ((i + j) & 1) ? -inv : inv;
                const float2 p0 = s_fft[(0 * SL + i) * FFT_P + j], p1 = s_fft[(1 * SL + i) * FFT_P + j];
                const float2 p2 = s_fft[(2 * SL + i) * FFT_P + j], p3 = s_fft[(3 * SL + i) * FFT_P + j];
                const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
                atomicAdd(dst + 2 * gp, make_float4(sg * p0.x, sg * p0.y, sg * p1.x, sg * p1.y));
                atomicAdd(dst + 2 * gp + 1, make_float4(sg * p2.x, sg * p2.y, sg * p3.x, sg * p3.y));
            }
        }
    }
    __syncthreads();
    if (mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(512));
}

// one CTA per subgrid of one plan (plan index idx[b] or first + b): subgrid images
__global__ void __launch_bounds__(NT, 1)
gridder_sep_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                   const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                   const float *__restrict__ taper, float4 *__restrict__ out) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    gridder_sep_body<false>(g, g.sub[sid], vis, flags, aterms, taper, out + (size_t)blockIdx.x * SPIX * 2);
}

// fused: one CTA per subgrid, transformed and added into the grid
__global__ void __launch_bounds__(NT, 1)
gridder_sep_fused_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                         const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                         const float *__restrict__ taper, float4 *__restrict__ grid) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    gridder_sep_body<true>(g, g.sub[sid], vis, flags, aterms, taper, grid);
}

}  // namespace

idg_status launch_gridder_sep(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *out, void *stream) {
    if (g.L != SL || !g.separable) return fail(IDG_ERR_UNSUPPORTED, "the separable gridder needs L = 32 and a separable plan");
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute(gridder_sep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SEP_SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "separable gridder smem attribute");
    gridder_sep_kernel<<<(unsigned)set.count, NT, SEP_SMEM, s>>>(g, set.idx, set.first, (const float4 *)vis, flags,
                                                                 (const float4 *)aterms, taper, (float4 *)out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "separable gridder launch");
    return IDG_OK;
}

idg_status launch_gridder_sep_fused(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *grid, void *stream) {
    if (g.L != SL || !g.separable) return fail(IDG_ERR_UNSUPPORTED, "the separable gridder needs L = 32 and a separable plan");
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute(gridder_sep_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SEP_SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "separable gridder smem attribute");
    gridder_sep_fused_kernel<<<(unsigned)set.count, NT, SEP_SMEM, s>>>(g, set.idx, set.first, (const float4 *)vis,
                                                                       flags, (const float4 *)aterms, taper,
                                                                       (float4 *)grid);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "separable fused gridder launch");
    return IDG_OK;
}

idg_status read_sep_error(int *code) {
    int zero = 0, v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_sep_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_sep_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the separable gridder error word");
    *code = v;
    return IDG_OK;
}

}  // namespace idg
