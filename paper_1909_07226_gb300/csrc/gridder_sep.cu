// Separable gridder on the tensor cores (tcgen05), L = 32, 24 and 16.
//
// The subgrid image of Eq. (ShiftedDirectImaging) is
//   I_q(x, y) = sum_k V_kq exp(i (a_k X + b_k Y + c_k n'(x, y))),
// with X = x - L/2, Y = y - L/2 and c_k = 2 pi (w_k - w_s) (w_s the subgrid's w
// offset, see the epilogue).  Splitting n'(x, y) = s(x) + t(y) + r(x, y), s and t
// a row and a column of n' (the plan's reference row and column j0: s(x) =
// n'(x, j0), t(y) = n'(j0, y) - n'(j0, j0)), the phasor factors into
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
// accumulator is added into FP32 sums in shared memory (RN) and restarted.
// The producers read it as soon as the period's MMAs are done and release it
// before adding, so the MMAs wait only for the tensor-memory loads; the rest
// of the tensor memory holds two A stages.
//
// Schedule.  One CTA per subgrid, one CTA per SM: sixteen producer warps and
// one MMA warp.  A stage is eight groups of 8 visibilities: every stage ends
// in a tensor-memory wait, a proxy fence and a barrier arrival per warp, and
// with eight groups (rather than four) that fixed cost is spread over twice
// the work, 9 % off the gridder's time.  Per stage each producer, for each of
// its groups warp / 4 and warp / 4 + 4:
//   - writes the 8 A entries of its row (polarisation lane / 8, pixel row
//     8 (warp % 4) + lane % 8) into tensor memory, one 16-column store.  It
//     forms Ey for two of the visibilities and takes the others from the
//     lanes of the same row by shuffles;
//   - forms the B entries of pixel column 8 (warp % 4) + lane % 8 for the
//     adjacent visibilities 2 (lane / 8) and 2 (lane / 8) + 1 of the group,
//     and writes them as one 8-byte store per row block (a warp's store
//     covers 256 contiguous bytes, free of bank conflicts).
// Visibilities are staged 512 at a time; the next batch is loaded into
// registers while the current one is processed.
// Tensor memory (512 columns):
//   accumulator: main (m, re/im, x) 0..127, correction (m = 0) 128..191
//   A stage s at 192 + 128 s, group i at + 16 i: 8 columns hi, 8 lo
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

constexpr int NPW = 16;                        // producer warps
constexpr int NP = NPW * 32;                   // producer threads
constexpr int NT = NP + 32;                    // + the MMA warp
constexpr int VB = NP;                         // visibilities per staged batch (one per producer)
constexpr int GB = VB / 8;                     // groups per batch
constexpr int FOLD = 64;                       // groups per accumulation period
constexpr int SG = 8;                          // groups of 8 visibilities per stage
constexpr int STAGES = 2;
static_assert(FOLD / SG >= STAGES, "a period spans at least STAGES stages");
static_assert((STAGES & (STAGES - 1)) == 0, "STAGES is a power of two");
static_assert(FOLD % SG == 0 && GB % SG == 0, "periods and batches are whole stages");

// Layout for subgrid size L (32, 24 or 16).  A has 128 rows: lane quarter yq holds pixel
// rows y = (L / 4) yq + ylo for ylo < L / 4 at lanes 8 q + ylo (lanes with ylo >= L / 4
// carry zeros: ylo = 6, 7 at L = 24, ylo >= 4 at L = 16).  B has 6 L rows per group: (m = 0, re), (m = 0, im), (m = 1, re),
// (m = 1, im), then the lo parts of m = 0 re and im, L rows each.
template <int L>
struct SepG {
    static constexpr int SL = L, SPIX = L * L, YQ = L / 4;
    static constexpr int B_GROUP = 6 * L * 32;   // B of one group: 6 L rows x 16 K FP16
    static constexpr int B_STAGE = SG * B_GROUP;
    // coefficients as two float pairs, [2][VB] (b, c) for the Ey side, then [2][VB] (a, c)
    // for the Ex side: the shared-memory pipe is close to its limit in the main loop and its
    // cost is the bytes each thread reads (a float4 where two floats are used costs twice)
    static constexpr int COEF_OFF = STAGES * B_STAGE;
    static constexpr int VIS_OFF = COEF_OFF + 2 * VB * 16;   // [2][VB][4] float2 (scaled V)
    static constexpr int FOLD_OFF = VIS_OFF + 2 * VB * 32;   // [32][NP] float: folded sums of each producer
    static constexpr int SMEM = FOLD_OFF + 32 * NP * 4;
    static constexpr int FFT_P = L + 1;
    // the subgrid's A-terms after the main loop: [2 stations][L^2] 2 x 2 complex, beside the
    // transform planes, over the stage and coefficient buffers
    static constexpr int AT_OFF = 4 * L * FFT_P * 8;
    static constexpr uint32_t AT_BYTES = SPIX * 32;
    // accumulator: main (m, re/im, x) at 0 .. 4 L, correction (m = 0) at 4 L .. 6 L; then the
    // A stages
    static constexpr uint32_t A_COL = 6 * L;
    static constexpr uint32_t IDESC_NB = idesc_m128(6 * L), IDESC_NC = idesc_m128(2 * L);
    static constexpr int NSL = L / 8;             // 16-column slices of the m = 0 block (fold)
    static constexpr int XS = L / 4;              // x values per producer in the epilogue
    static_assert(L == 32 || L == 24 || L == 16, "subgrid sizes of the separable kernels");
    static_assert(4 * L * FFT_P * 8 <= FOLD_OFF, "transform planes fit over the stage buffers");
    static_assert(SMEM + 1024 <= 227 * 1024, "dynamic and static shared memory of one CTA");
    static_assert(AT_OFF % 16 == 0 && AT_OFF + 2 * (int)AT_BYTES <= VIS_OFF, "A-terms over the stage and coefficient buffers");
    static_assert(A_COL % 16 == 0 && A_COL + 16 * SG * STAGES <= 512, "tensor memory");
    static_assert(NSL <= NPW / 4, "one fold slice per warp of a lane quarter");
};

__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" :: "n"(NP) : "memory"); }

// One subgrid d of geometry g (taper and A-terms applied): into o[L][L][4], or with
// FUSED transformed in shared memory and added into the grid o[layer][N][N][4]
// (Algorithm 1: direct sum, image-domain kernel, "FFT", add to the master grid).
template <int L, bool FUSED>
__device__ __forceinline__ void gridder_sep_body(const Geometry &g, const DevSubgrid d,
                                                 const float4 *__restrict__ vis, const uint8_t *__restrict__ flags,
                                                 const float4 *__restrict__ aterms, const float *__restrict__ taper,
                                                 float4 *__restrict__ o) {
    using C = SepG<L>;
    constexpr int SL = C::SL, SPIX = C::SPIX, YQ = C::YQ, B_GROUP = C::B_GROUP, B_STAGE = C::B_STAGE;
    constexpr int COEF_OFF = C::COEF_OFF, VIS_OFF = C::VIS_OFF, FOLD_OFF = C::FOLD_OFF, FFT_P = C::FFT_P;
    constexpr int AT_OFF = C::AT_OFF, XS = C::XS;
    constexpr uint32_t AT_BYTES = C::AT_BYTES, A_COL = C::A_COL;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;
    float2 *s_cb = (float2 *)(smem + COEF_OFF);          // [2][VB] (b, c)
    float2 *s_ca = s_cb + 2 * VB;                         // [2][VB] (a, c)
    float2 *s_vis = (float2 *)(smem + VIS_OFF);
    float2 *s_fft = (float2 *)smem;                 // [4][L][L + 1] after the main loop
    float *s_fold = (float *)(smem + FOLD_OFF);     // [32][NP]: m = 0 sums (16), then m = 1 (16)
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[STAGES], s_empty[STAGES], s_foldbar, s_folded, s_drain, s_atbar;
    __shared__ float s_red[2][NPW];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == NPW;
    const int total_groups = (d.kp + 7) / 8;
    const int n_batches = (d.kp + VB - 1) / VB;     // = accumulation periods (FOLD = GB)

    // staging (producers): visibility tid of batch b, loaded into registers one batch ahead;
    // the first batch's loads go out before the set-up below, so their latency overlaps it
    float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa, puv = pa, pws = pa;
    float2 pw = make_float2(0.f, 0.f);
    bool pin = false, pflag = false;
    const float4 *uvw2 = (const float4 *)g.uvw_f2;
    const float4 *sc2 = (const float4 *)g.scale_f2;
    auto load_batch = [&](int b) {
        const int k = b * VB + tid;
        pin = k < d.kp;
        pflag = false;
        if (pin) {
            int t, c;
            const size_t vi = vis_index(g, d, k, t, c);
            const size_t bt = (size_t)d.bl * g.n_t + t;
            puv = uvw2[2 * bt];
            const float4 w4 = uvw2[2 * bt + 1];
            pw = make_float2(w4.x, w4.y);
            pws = sc2[c];
            pflag = flags && flags[vi];
            pa = vis[2 * vi];          // loaded whatever the flag: the load does not wait for it
            pb = vis[2 * vi + 1];
        }
    };
    if (!mma_warp) load_batch(0);

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
        mbar_init(smem_u32(&s_foldbar), 1);
        mbar_init(smem_u32(&s_folded), NPW);
        mbar_init(smem_u32(&s_drain), 1);
        mbar_init(smem_u32(&s_atbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    bool failed = false, at_issued = false;
    // the taper of this thread's epilogue pixels, loaded at the end of its main loop
    constexpr int NPIX = (SPIX + NT - 1) / NT;
    float tw_pre[NPIX];
    auto load_taper = [&]() {
#pragma unroll
        for (int i = 0; i < NPIX; ++i) tw_pre[i] = tid + i * NT < SPIX ? taper[tid + i * NT] : 0.0f;
    };
    const int yq = warp & 3, sl = warp >> 2;        // lane quarter (rows 32 yq ..) and fold column slice

    if (mma_warp) {
        if (lane == 0) {
            // descriptors and tensor-memory addresses advance by constants: stage s, group i at
            // B + s B_STAGE + i B_GROUP (the descriptor's address field counts 16-byte units)
            const uint64_t db0 = smem_desc(smem_u32(sB));
            const int n_stages = (total_groups + SG - 1) / SG;
            constexpr int SPP = FOLD / SG;                  // stages per accumulation period
            for (int st = 0; st < n_stages; ++st) {
                const int s = st & (STAGES - 1);
                const bool first = st % SPP == 0, last = st % SPP == SPP - 1 || st == n_stages - 1;
                if (first && st > 0) {         // the producers have read the previous period
                    wait_or_fail(smem_u32(&s_folded), (uint32_t)(((st / SPP) - 1) & 1), failed);
                }
                wait_or_fail(smem_u32(&s_full[s]), (uint32_t)((st / STAGES) & 1), failed);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int ng = min(SG, total_groups - st * SG);
                const uint64_t dbs = db0 + (uint64_t)((s * B_STAGE) >> 4);
                const uint32_t ats = tmem + A_COL + 16u * SG * (uint32_t)s;
#pragma unroll
                for (int i = 0; i < SG; ++i) {
                    if (i < ng) {
                        mma_ta_i(tmem, ats + 16u * i, dbs + (uint64_t)((i * B_GROUP) >> 4), C::IDESC_NB,
                                 (first && i == 0) ? 0u : 1u);
                        mma_ta_i(tmem + 4u * SL, ats + 16u * i + 8u, dbs + (uint64_t)((i * B_GROUP) >> 4), C::IDESC_NC,
                                 1u);
                    }
                }
                if (last) commit(smem_u32(&s_foldbar));
                commit(smem_u32(&s_empty[s]));
            }
            commit(smem_u32(&s_drain));
            bool late = false;
            wait_or_fail(smem_u32(&s_drain), 0u, late);     // bounded: let own MMAs finish before the free
            if (late) failed = true;
            // the tensor cores are done with the stage buffers: bring the subgrid's A-terms (A_p,
            // A_q) into them while the producers fold and form the image
            if (aterms && !failed) {
                const float4 *base = aterms + 2 * ((size_t)d.slot * g.n_stations) * SPIX;
                mbar_expect_tx(smem_u32(&s_atbar), 2 * AT_BYTES);
                bulk_g2s(smem_u32(smem + AT_OFF), base + 2 * (size_t)d.st_p * SPIX, AT_BYTES, smem_u32(&s_atbar));
                bulk_g2s(smem_u32(smem + AT_OFF + AT_BYTES), base + 2 * (size_t)d.st_q * SPIX, AT_BYTES,
                         smem_u32(&s_atbar));
                at_issued = true;
            }
        }
        failed = __shfl_sync(0xffffffffu, failed, 0);
        load_taper();
    } else {
        // A rows: r = 32 yq + lane holds polarisation qa = lane / 8 of pixel row y = YQ yq + lane % 8
        // (rows with lane % 8 >= YQ are zero)
        const int qa = lane >> 3, ylo = lane & 7;
        const bool row_ok = YQ == 8 || ylo < YQ;
        const int yrow = YQ * yq + (row_ok ? ylo : 0);
        const int ga = warp >> 2;                   // group of the stage whose A entries this warp writes
        const uint32_t lane_base = tmem + ((uint32_t)(32 * yq) << 16);
        // Ey of row y for visibilities 2 qa and 2 qa + 1 of the group: computed here, shared by shuffles
        const float Yv = (float)(yrow - SL / 2);
        const float ty = g.sep[SL + yrow];
        // B entries: x = 8 (warp & 3) + lane % 8, visibility j = 4 jh + lane / 8 of group i, where
        // (i, jh) = (combo / 2, combo % 2) for combo = 2 (warp / 4) + t, t = 0, 1
        const int xb = 8 * (warp & 3) + (lane & 7), jl = lane >> 3;
        const bool x_ok = SL == 32 || xb < SL;      // the same for the whole warp (L is a multiple of 8)
        const float Xv = (float)(xb - SL / 2);
        const float sx = g.sep[x_ok ? xb : 0];
        const float csig = g.c_scale;
        const uint16_t m1h = 0xBC00u;      // FP16 -1

        // phase coefficients of the staged visibility: u (f/c) k_uv - u0 k_uv and so on, from
        // float pairs with error-free products and sums, rounded once to FP32
        float4 cf_next = make_float4(0.f, 0.f, 0.f, 0.f);
        auto form_coef = [&]() {
            cf_next = make_float4(0.f, 0.f, 0.f, 0.f);
            if (pin) {
                cf_next.x = pair_coef(puv.x, puv.y, pws.x, pws.y, d.a0h, d.a0l);
                cf_next.y = pair_coef(puv.z, puv.w, pws.x, pws.y, d.b0h, d.b0l);
                cf_next.z = pair_coef(pw.x, pw.y, pws.z, pws.w, d.csh, d.csl);
            }
        };
        // coefficients and raw V of the batch; the batch's largest |component| into s_red[bb]
        auto store_batch = [&](int bb) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (pin && !pflag) {
                a = pa;
                b = pb;
            }
            s_cb[bb * VB + tid] = make_float2(cf_next.y, cf_next.z);
            s_ca[bb * VB + tid] = make_float2(cf_next.x, cf_next.z);
            float4 *dv = (float4 *)(s_vis + (size_t)(bb * VB + tid) * 4);
            dv[0] = a;
            dv[1] = b;
            float m = fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                            fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w))));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
            if (lane == 0) s_red[bb][warp] = m;
        };
        float inv_sc0 = 1.0f, inv_sc1 = 1.0f;        // 1 / scale of the last even and odd batch

        auto fold = [&](int P) {
            wait_or_fail(smem_u32(&s_foldbar), (uint32_t)(P & 1), failed);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // this thread's row, columns 16 sl .. of the m = 0 block (main + correction) and of m = 1;
            // the accumulator is released right after the loads
            constexpr bool all_fold = C::NSL == NPW / 4;
            if (!all_fold && sl >= C::NSL) {      // no slice of the m = 0 block for this warp
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&s_folded));
                return;
            }
            uint32_t r[16], rc[16], r1[16];
            const uint32_t base = lane_base + 16u * (uint32_t)sl;
            tmem_ld16(base, r);
            tmem_ld16(base + 4u * SL, rc);
            tmem_ld16(base + 2u * SL, r1);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_folded));
            const float is = (P & 1) ? inv_sc1 : inv_sc0;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float v = (__uint_as_float(r[c]) + __uint_as_float(rc[c])) * is;
                float &f = s_fold[c * NP + tid];
                f = P ? f + v : v;
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float v = __uint_as_float(r1[c]) * is;
                float &f = s_fold[(16 + c) * NP + tid];
                f = P ? f + v : v;
            }
        };

        form_coef();
        store_batch(0);
        producers_sync();
        int next_fold = 0;
        for (int b = 0; b < n_batches; ++b) {
            const int bb = b & 1;
            // this batch's power-of-two scale: largest |component| of V in [2^9, 2^10)
            float m = 0.0f;
#pragma unroll
            for (int w = 0; w < NPW; ++w) m = fmaxf(m, s_red[bb][w]);
            int e2 = 0;
            if (m > 0.0f) frexpf(m, &e2);
            const float scale = ldexpf(1.0f, 10 - e2);
            if (bb) inv_sc1 = ldexpf(1.0f, e2 - 10);
            else inv_sc0 = ldexpf(1.0f, e2 - 10);
            if (b + 1 < n_batches) load_batch(b + 1);
            const float2 *cb = s_cb + bb * VB, *ca = s_ca + bb * VB;
            const float2 *vb = s_vis + (size_t)bb * VB * 4;
            const int nst = (min(GB, total_groups - b * GB) + SG - 1) / SG;
            for (int si = 0; si < nst; ++si) {
                const int st = b * (GB / SG) + si;
                const int s = st % STAGES;
                if (st >= STAGES) wait_or_fail(smem_u32(&s_empty[s]), (uint32_t)(((st / STAGES) - 1) & 1), failed);
                // the MMAs of stage st - STAGES are done: when that was the last stage of period
                // next_fold, read it out now (the next period's first MMA waits for it)
                if (next_fold < n_batches - 1 && st - STAGES == (next_fold + 1) * (FOLD / SG) - 1) {
                    fold(next_fold);
                    ++next_fold;
                }
                // A entries of groups ga + 4 gg: scale V_kq Ey_k(y) for its 8 visibilities
#pragma unroll
                for (int gg = 0; gg < SG / 4; ++gg) {
                    const int kb = 8 * (SG * si + ga + 4 * gg);
                    float ec[2], es[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 cf = cb[kb + 2 * qa + h];
                        float sn, cs;
                        __sincosf(fmaf(cf.y, ty, cf.x * Yv), &sn, &cs);
                        ec[h] = cs * scale;
                        es[h] = sn * scale;
                    }
                    uint32_t e[16];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int src = 8 * (j >> 1) + ylo;
                        const float cs = __shfl_sync(0xffffffffu, (j & 1) ? ec[1] : ec[0], src);
                        const float sn = __shfl_sync(0xffffffffu, (j & 1) ? es[1] : es[0], src);
                        const float2 v = vb[(kb + j) * 4 + qa];
                        split_e_m(fmaf(v.x, cs, -v.y * sn), fmaf(v.x, sn, v.y * cs), m1h, e[j], e[8 + j]);
                        if (!row_ok) e[j] = e[8 + j] = 0u;
                    }
                    tmem_st16(lane_base + A_COL + 16u * SG * (uint32_t)s + 16u * (uint32_t)(ga + 4 * gg), e);
                }
                // B entries: beta = Ex_k(x) (m = 0: hi and lo) and c_k sigma Ex_k(x) (m = 1: hi), rows
                // (m, re, x) = (Re beta, -Im beta) and (m, im, x) = (Im beta, Re beta)
                uint8_t *Bs = sB + s * B_STAGE;
#pragma unroll
                for (int gg = 0; gg < SG / 4; ++gg) {
                    if (!x_ok) break;
                    // visibilities j0 = 2 jl and j0 + 1 of group i = warp / 4 + 4 gg sit in adjacent K
                    // slots of each row: one 8-byte store per row
                    const int i = (warp >> 2) + 4 * gg, j0 = 2 * jl;
                    uint32_t w[6][2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const float2 cf = ca[8 * (SG * si + i) + j0 + t];
                        float sn, cs;
                        __sincosf(fmaf(cf.y, sx, cf.x * Xv), &sn, &cs);
                        // the im row (sn, cs) is the re row (cs, -sn) with its halves swapped and the
                        // new low half negated: exact, as FP16 rounding is symmetric
                        uint32_t hr, lr;
                        split_e_m(cs, -sn, m1h, hr, lr);
                        const float cz = cf.y * csig;
                        const uint32_t h1r = pack_f16x2(cz * cs, -cz * sn);
                        w[0][t] = hr;
                        w[1][t] = __byte_perm(hr, 0u, 0x1032u) ^ 0x8000u;
                        w[2][t] = h1r;
                        w[3][t] = __byte_perm(h1r, 0u, 0x1032u) ^ 0x8000u;
                        w[4][t] = lr;
                        w[5][t] = __byte_perm(lr, 0u, 0x1032u) ^ 0x8000u;
                    }
                    uint8_t *Bg = Bs + i * B_GROUP + (uint32_t)(xb >> 3) * kSBO + (uint32_t)(jl >> 1) * kLBO +
                                  (uint32_t)(xb & 7) * 16 + (uint32_t)(jl & 1) * 8;
                    // row blocks of L (L / 8 kSBO): m = 0 re, m = 0 im, m = 1 re, m = 1 im, then the lo
                    // parts of m = 0 re and im (rows 4 L + x, 5 L + x)
#pragma unroll
                    for (int q = 0; q < 6; ++q) *(uint2 *)(Bg + (SL / 8) * q * kSBO) = make_uint2(w[q][0], w[q][1]);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&s_full[s]));
            }
            if (b + 1 < n_batches) {
                form_coef();
                store_batch(bb ^ 1);
                producers_sync();
            }
        }
        // the epilogue's global reads first: taper, and r(x, y) of this thread's x range
        load_taper();
        const int x0 = XS * sl;                     // this thread's x range in the epilogue
        float rr_pre[XS];
#pragma unroll
        for (int xi = 0; xi < XS; ++xi) rr_pre[xi] = g.sep[2 * SL + yrow * SL + x0 + xi];
        while (next_fold < n_batches) {
            fold(next_fold);
            ++next_fold;
        }
        if (failed && lane == 0) atomicExch(&g_sep_error, 1);
        producers_sync();      // every producer is past the stage and batch buffers and has folded
        if (!failed && row_ok) {
            // I = S0 + i r S1 / sigma into the polarisation planes.  Column C of the m = 0 block
            // (re: C = x, im: C = L + x) was folded by the thread of slice C / 16 of this row,
            // warp 4 (C / 16) + yq, as its entry C % 16.
            const float rs = 1.0f / csig;
#pragma unroll
            for (int xi = 0; xi < XS; ++xi) {
                const int x = x0 + xi, cre = x, cim = SL + x;
                const int tre = (4 * (cre >> 4) + yq) * 32 + lane, tim = (4 * (cim >> 4) + yq) * 32 + lane;
                float s0r = 0.f, s0i = 0.f, s1r = 0.f, s1i = 0.f;
                if (n_batches) {
                    s0r = s_fold[(cre & 15) * NP + tre];
                    s0i = s_fold[(cim & 15) * NP + tim];
                    s1r = s_fold[(16 + (cre & 15)) * NP + tre];
                    s1i = s_fold[(16 + (cim & 15)) * NP + tim];
                }
                const float rr = rr_pre[xi] * rs;
                s_fft[(qa * SL + yrow) * FFT_P + x] = make_float2(fmaf(-rr, s1i, s0r), fmaf(rr, s1r, s0i));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (!__syncthreads_or(failed)) {
        if (aterms) {
            bool late = false;
            wait_or_fail(smem_u32(&s_atbar), 0u, late);
            if (late) atomicExch(&g_sep_error, 1);
        }
        // image-domain kernel per pixel: taper * A_p^H I A_q (with the centring factor when FUSED)
#pragma unroll
        for (int ip = 0; ip < NPIX; ++ip) {
            const int pix = tid + ip * NT;
            if (pix >= SPIX) break;
            const int y = pix / SL, x = pix % SL;
            M22 P;
#pragma unroll
            for (int c = 0; c < 4; ++c) P.m[c] = s_fft[(c * SL + y) * FFT_P + x];
            if (d.dws != 0.0f) {      // the sums used w_s: the rest of the w offset, exp(i 2 pi (w_s - w0) n')
                float sn, cs;
                sincospif(d.dws * g.nprime[pix], &sn, &cs);     // (dws in half turns: exact reduction)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    P.m[c] = make_float2(P.m[c].x * cs - P.m[c].y * sn, P.m[c].x * sn + P.m[c].y * cs);
            }
            if (aterms) {
                const float4 *at = (const float4 *)(smem + AT_OFF);
                const M22 Ap = load_m22(at + 2 * pix);
                const M22 Aq = load_m22(at + 2 * (SPIX + pix));
                P = herm_mul_mul(Ap, P, Aq);
            }
            if (FUSED) {
                const float tw = ((x + y) & 1) ? -tw_pre[ip] : tw_pre[ip];
#pragma unroll
                for (int c = 0; c < 4; ++c) s_fft[(c * SL + y) * FFT_P + x] = make_float2(tw * P.m[c].x, tw * P.m[c].y);
            } else {
                const float tw = tw_pre[ip];
                o[2 * pix] = make_float4(tw * P.m[0].x, tw * P.m[0].y, tw * P.m[1].x, tw * P.m[1].y);
                o[2 * pix + 1] = make_float4(tw * P.m[2].x, tw * P.m[2].y, tw * P.m[3].x, tw * P.m[3].y);
            }
        }
        if (FUSED) {
            __syncthreads();
            if constexpr (SL == 32)
                fft2_planar_pairs32<-1>(s_fft, tid);
            else
                fft2_planar<SL, -1>(s_fft, tid, NT);
            const float inv = 1.0f / (float)SPIX;
            float4 *dst = o + (size_t)d.layer * g.N * g.N * 2;
            for (int pix = tid; pix < SPIX; pix += NT) {
                const int i = pix / SL, j = pix % SL;
                const float sg = ((i + j) & 1) ? -inv : inv;
                const float2 p0 = s_fft[(0 * SL + i) * FFT_P + j], p1 = s_fft[(1 * SL + i) * FFT_P + j];
                const float2 p2 = s_fft[(2 * SL + i) * FFT_P + j], p3 = s_fft[(3 * SL + i) * FFT_P + j];
                const size_t gp = (size_t)(d.r0 + i) * g.N + (d.q0 + j);
                red_add_f4(dst + 2 * gp, make_float4(sg * p0.x, sg * p0.y, sg * p1.x, sg * p1.y));
                red_add_f4(dst + 2 * gp + 1, make_float4(sg * p2.x, sg * p2.y, sg * p3.x, sg * p3.y));
            }
        }
    }
    __syncthreads();
    if (at_issued) {      // the copies have landed before the CTA's shared memory is released
        bool late = false;
        wait_or_fail(smem_u32(&s_atbar), 0u, late);
    }
    if (mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(512));
}

// one CTA per subgrid of one plan (plan index idx[b] or first + b): subgrid images
template <int L>
__global__ void __launch_bounds__(NT, 1)
gridder_sep_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                   const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                   const float *__restrict__ taper, float4 *__restrict__ out) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    gridder_sep_body<L, false>(g, g.sub[sid], vis, flags, aterms, taper, out + (size_t)blockIdx.x * L * L * 2);
}

// fused: one CTA per subgrid, transformed and added into the grid
template <int L>
__global__ void __launch_bounds__(NT, 1)
gridder_sep_fused_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ vis,
                         const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                         const float *__restrict__ taper, float4 *__restrict__ grid) {
    allow_dependents();
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    gridder_sep_body<L, true>(g, g.sub[sid], vis, flags, aterms, taper, grid);
    complete_after_primary();
}

template <int L>
idg_status launch_sep_set(bool fused, const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                          const void *aterms, const float *taper, void *out, cudaStream_t s) {
    auto kern = fused ? gridder_sep_fused_kernel<L> : gridder_sep_kernel<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SepG<L>::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "separable gridder smem attribute");
    kern<<<(unsigned)set.count, NT, SepG<L>::SMEM, s>>>(g, set.idx, set.first, (const float4 *)vis, flags,
                                                       (const float4 *)aterms, taper, (float4 *)out);
    e = cudaGetLastError();
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, fused ? "separable fused gridder launch" : "separable gridder launch");
}

}  // namespace

bool separable_size(int L) { return L == 32 || L == 24 || L == 16; }

cudaError_t prepare_gridder_sep_batch() {
    cudaError_t e = cudaFuncSetAttribute(gridder_sep_fused_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SepG<32>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gridder_sep_fused_kernel<24>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SepG<24>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gridder_sep_fused_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SepG<16>::SMEM);
    return e;
}

// a batch's launch of the fused kernel over one job's items (the shared-memory attribute
// is set by prepare_tcw_batch_kernels, outside graph capture); pdl: see launch_pdl
idg_status launch_gridder_sep_job(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                  const void *aterms, const float *taper, void *grid, void *stream, bool pdl) {
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned n = (unsigned)set.count;
    const float4 *v = (const float4 *)vis, *at = (const float4 *)aterms;
    float4 *o = (float4 *)grid;
    cudaError_t e;
    switch (g.L) {
    case 32: e = launch_pdl(gridder_sep_fused_kernel<32>, n, NT, SepG<32>::SMEM, s, pdl, g, set.idx, set.first, v, flags, at, taper, o); break;
    case 24: e = launch_pdl(gridder_sep_fused_kernel<24>, n, NT, SepG<24>::SMEM, s, pdl, g, set.idx, set.first, v, flags, at, taper, o); break;
    case 16: e = launch_pdl(gridder_sep_fused_kernel<16>, n, NT, SepG<16>::SMEM, s, pdl, g, set.idx, set.first, v, flags, at, taper, o); break;
    default: return fail(IDG_ERR_UNSUPPORTED, "the separable gridder needs L = 32, 24 or 16");
    }
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "separable gridder job launch");
}

idg_status launch_gridder_sep(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *out, void *stream) {
    if (!separable_size(g.L) || !g.separable)
        return fail(IDG_ERR_UNSUPPORTED, "the separable gridder needs L = 32, 24 or 16 and a separable plan");
    if (set.count <= 0) return IDG_OK;
    switch (g.L) {
    case 32: return launch_sep_set<32>(false, g, set, vis, flags, aterms, taper, out, (cudaStream_t)stream);
    case 24: return launch_sep_set<24>(false, g, set, vis, flags, aterms, taper, out, (cudaStream_t)stream);
    default: return launch_sep_set<16>(false, g, set, vis, flags, aterms, taper, out, (cudaStream_t)stream);
    }
}

idg_status launch_gridder_sep_fused(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *grid, void *stream) {
    if (!separable_size(g.L) || !g.separable)
        return fail(IDG_ERR_UNSUPPORTED, "the separable gridder needs L = 32, 24 or 16 and a separable plan");
    if (set.count <= 0) return IDG_OK;
    switch (g.L) {
    case 32: return launch_sep_set<32>(true, g, set, vis, flags, aterms, taper, grid, (cudaStream_t)stream);
    case 24: return launch_sep_set<24>(true, g, set, vis, flags, aterms, taper, grid, (cudaStream_t)stream);
    default: return launch_sep_set<16>(true, g, set, vis, flags, aterms, taper, grid, (cudaStream_t)stream);
    }
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
