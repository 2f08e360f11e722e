// Separable degridder on the tensor cores (tcgen05), L = 32, 24 and 16.
//
// The visibilities of Algorithm 2 from the corrected subgrid image P_q(x, y)
// (taper and A_p P A_q^H applied) are
//   y_kq = sum_{x,y} P_q(x, y) exp(-i (a_k X + b_k Y + c_k n'(x, y))).
// With the split n' = s(x) + t(y) + r(x, y) used by the separable gridder and
// exp(-i c r) = 1 - i c r + O(theta^2 / 2) (theta = max |c| max |r|, checked
// by the plan),
//   y_kq = sum_y Ey*_k(y) [T0_kq(y) - i c_k T1_kq(y)],
//   T_mkq(y) = sum_x Ex*_k(x) Q_mq(x, y),  Q0 = P, Q1 = P r,
//   Ex*_k(x) = exp(-i (a_k X + c_k s(x))),  Ey*_k(y) = exp(-i (b_k Y + c_k t(y))).
// Both terms are one complex matrix product on the tensor cores,
//   T_kq(y) = sum_x Ex*_k(x) Q0_q(x, y) + sum_x (-i c_k Ex*_k(x)) Q1_q(x, y),
// with rows (re/im, visibility) of a tile of 64 visibilities, columns (q, y),
// 128 of them, and K = (x, re/im) twice (m = 0, then m = 1).  The sum over y
// with the visibility's own phasors, y_kq = sum_y Ey*_k(y) T_kq(y), runs on
// the CUDA cores (FP32, round to nearest), one thread per tile row.
//
// GEMM.  A holds the real 2 x 2 embedding of a = Ex*_k(x) (m = 0) and of
// a = -i c_k sigma Ex*_k(x) (m = 1, sigma a power of two with max |c| sigma
// <= 1): row k (re) = (Re a, -Im a), row 64 + k (im) = (Im a, Re a) over
// K = (x, re/im).  B[(q, y)] = (Re, Im) of Q0 = s P and of Q1 = s r P / sigma
// (s a power of two per subgrid), so both products carry the same scale.  The
// m = 0 operands are split into FP16 hi + lo and take A_hi B_hi + A_hi B_lo +
// A_lo B_hi; the m = 1 term (at most theta relative) takes A_hi B_hi.  Per K
// step of 16 (8 x): four MMAs of N = 128.  The accumulation is 16 MMAs long,
// so no folds are needed.
//
// Schedule.  One CTA per subgrid, one CTA per SM.  All warps first form the
// image (split from the grid and inverse transform in shared memory when
// FUSED, while two bulk copies bring the subgrid's A-terms), the corrections,
// the scale and B (shared memory, fixed for the subgrid).  Then per tile: a
// coefficient warp stages the visibilities' phase coefficients (float pairs,
// error-free FP32 products and sums); eight producer warps write A (shared
// memory, one core matrix per warp store); the consumers form the tile's Ey*
// table while its MMAs run;
// the MMA warp issues the 16 MMAs into one of four accumulators; eight consumer
// warps read their rows' columns, sum over y, pair the re and im rows of each
// visibility through shared memory and write the visibilities.  The A stages
// (two, freed by the MMAs) and the coefficient and accumulator stages (four,
// freed by the consumers) are separate, so producers, MMAs and consumers
// overlap across tiles.  Tensor memory: accumulator e at 128 e.
// Every wait is bounded; after a failed wait a thread skips every later wait,
// the error word is set and no output is written.
#include "batch_jobs.cuh"
#include "device_common.cuh"
#include "fft_impl.cuh"
#include "tc_common.cuh"

namespace idg {

// device error word of the separable degridder (0 = ok); read and cleared by
// idg_device_errors
__device__ int g_sepd_error = 0;

namespace {

using namespace dev;
using namespace tc;

constexpr int NPW = 8, NCW = 8;                 // producer and consumer warps
constexpr int NP = NPW * 32, NC = NCW * 32;
constexpr int MMA_WARP = NPW + NCW;
constexpr int COEF_WARP = MMA_WARP + 1;        // stages the per-visibility coefficients (float pairs)
constexpr int NT = NP + NC + 64;
constexpr int TV = 64;                          // visibilities per tile (rows 2 k + re/im)
constexpr int AST = 2;                          // A stages (gated by the MMAs)
constexpr int EST = 4;                          // Ey*, coefficient stages and accumulators (gated by the consumers)
constexpr int T4K = 128 * 32;                   // 128 rows x 16 K FP16
constexpr int CF_BYTES = EST * TV * 16;         // coefficients: [EST][TV] float4 (a, b, c, index)
constexpr int PART_BYTES = 2 * 2 * 2 * 4 * TV * 4;   // consumer exchange: [2 tiles][re, im][h][4][TV] float
static_assert(AST == 2 && EST == 4, "stage arithmetic below");
static_assert(EST * 128 <= 512, "accumulators in tensor memory");

// Layout for subgrid size L (32, 24 or 16)
template <int L>
struct SepD {
    static constexpr int SL = L, SPIX = L * L;
    static constexpr int KT = L / 8;                // K steps of 16 (8 x, re/im) over the L x
    // B (fixed per subgrid), each [KT][4 L rows (q, y), padded to 128]: Q0 hi, Q0 lo, Q1 hi
    static constexpr int B0H_OFF = 0, B0L_OFF = B0H_OFF + KT * T4K, B1H_OFF = B0L_OFF + KT * T4K;
    static constexpr int A_OFF = B1H_OFF + KT * T4K;   // A: [AST][m = 0 hi, m = 0 lo, m = 1 hi][KT][128 rows]
    static constexpr int A_STAGE = 3 * KT * T4K;
    static constexpr int EY_OFF = A_OFF + AST * A_STAGE;   // Ey*: [2][L / 2 y pairs][TV] float4 (consumers)
    static constexpr int EY_STAGE = L * TV * 8;
    static constexpr int CF_OFF = EY_OFF + 2 * EY_STAGE;
    static constexpr int PART_OFF = CF_OFF + CF_BYTES;
    static constexpr int SMEM = PART_OFF + PART_BYTES;
    static constexpr int FFT_P = L + 1;
    // the subgrid's A-terms (A_p, A_q: [2][L^2] 2 x 2 complex), fetched by bulk copies at the
    // start of the prologue beside the transform planes (A stages and Ey* table are free until
    // the tiles)
    static constexpr int AT_OFF = A_OFF + 4 * L * FFT_P * 8;
    static constexpr uint32_t AT_BYTES = SPIX * 32;       // one station
    static constexpr uint32_t IDESC_N = idesc_m128(4 * L);
    // B tasks of the prologue: (q, y block of 8, x chunk of 4), one core matrix each
    static constexpr int YB = L / 8, XC = L / 4, NTASK = 4 * YB * XC;
    static constexpr int NWT = (NTASK + MMA_WARP - 1) / MMA_WARP;
    static constexpr int EYP = L * TV / NC / 2;     // Ey* pairs per consumer thread
    static_assert(L == 32 || L == 24 || L == 16, "subgrid sizes of the separable kernels");
    static_assert(4 * L * FFT_P * 8 <= AST * A_STAGE, "transform planes fit over the A stages");
    static_assert(AT_OFF % 16 == 0 && AT_OFF + 2 * (int)AT_BYTES <= CF_OFF, "A-terms before the coefficient stages");
    static_assert(3 * KT * T4K >= SPIX * 32, "the subgrid's grid rows fit in the B area");
    static_assert(L <= 32, "one grid row per lane of warp 0");
    static_assert(4 * L <= 128 && (4 * L) % 16 == 0, "B rows (q, y) in one MMA");
    static_assert(L * TV % (2 * NC) == 0 && (L / 2) % 4 == 0, "Ey* pairs spread evenly over the consumers");
    static_assert(L % 8 == 0 && 4 * NPW >= L, "x columns over the producer warps");
};

__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 2, %0;" :: "n"(NC) : "memory"); }

// Visibilities of subgrid d of geometry g from its image src[L][L][4], or with
// FUSED from the grid src[layer][N][N][4]: split and transformed in shared memory
// first (Algorithm 2: split from the master grid, "IFFT", image-domain kernel, sum).
template <int L, bool FUSED>
__device__ __forceinline__ void degridder_sep_body(const Geometry &g, const DevSubgrid d,
                                                   const float4 *__restrict__ src, const uint8_t *__restrict__ flags,
                                                   const float4 *__restrict__ aterms, const float *__restrict__ taper,
                                                   float4 *__restrict__ vis_out) {
    using C = SepD<L>;
    constexpr int SL = C::SL, SPIX = C::SPIX, KT = C::KT, B0H_OFF = C::B0H_OFF, B0L_OFF = C::B0L_OFF;
    constexpr int B1H_OFF = C::B1H_OFF, A_OFF = C::A_OFF, A_STAGE = C::A_STAGE, EY_OFF = C::EY_OFF;
    constexpr int CF_OFF = C::CF_OFF, PART_OFF = C::PART_OFF, FFT_P = C::FFT_P, AT_OFF = C::AT_OFF;
    constexpr uint32_t AT_BYTES = C::AT_BYTES;
    extern __shared__ __align__(1024) uint8_t smem[];
    float2 *s_fft = (float2 *)(smem + A_OFF);       // [4][L][L + 1] during the prologue
    float4 *s_coef = (float4 *)(smem + CF_OFF);
    float4 *s_ey = (float4 *)(smem + EY_OFF);
    float *s_part = (float *)(smem + PART_OFF);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_afull[AST], s_aempty[AST], s_eyfull[EST], s_eyempty[EST], s_dfull[EST],
        s_dempty[EST], s_drain, s_atbar, s_gbar;
    __shared__ float s_red[NT / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = (d.kp + TV - 1) / TV;

    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "n"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (warp == 0) {
        // barriers by lane 0; the copies are then issued by the whole warp, one per lane: the
        // subgrid's 32 grid rows (1 KB each, contiguous in the grid) into the B area, which is
        // free until B is formed at the end of the prologue, and the two stations' A-terms
        if (lane == 0) {
            for (int s = 0; s < AST; ++s) {
                mbar_init(smem_u32(&s_afull[s]), NPW);
                mbar_init(smem_u32(&s_aempty[s]), 1);
            }
            for (int e = 0; e < EST; ++e) {
                mbar_init(smem_u32(&s_eyfull[e]), 1);
                mbar_init(smem_u32(&s_eyempty[e]), NCW);
                mbar_init(smem_u32(&s_dfull[e]), 1);
                mbar_init(smem_u32(&s_dempty[e]), NCW);
            }
            mbar_init(smem_u32(&s_drain), 1);
            mbar_init(smem_u32(&s_atbar), 1);
            mbar_init(smem_u32(&s_gbar), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if (FUSED) mbar_expect_tx(smem_u32(&s_gbar), SL * SL * 32);
            if (aterms) mbar_expect_tx(smem_u32(&s_atbar), 2 * AT_BYTES);
        }
        __syncwarp();
        if (FUSED && lane < SL) {
            const float4 *gsrc = src + (size_t)d.layer * g.N * g.N * 2;
            bulk_g2s(smem_u32(smem + B0H_OFF + lane * SL * 32), gsrc + 2 * ((size_t)(d.r0 + lane) * g.N + d.q0),
                     SL * 32, smem_u32(&s_gbar));
        }
        if (aterms && lane < 2) {
            const float4 *base = aterms + 2 * ((size_t)d.slot * g.n_stations) * SPIX;
            bulk_g2s(smem_u32(smem + AT_OFF + lane * AT_BYTES), base + 2 * (size_t)(lane ? d.st_q : d.st_p) * SPIX,
                     AT_BYTES, smem_u32(&s_atbar));
        }
    }

    // the coefficient warp loads its first tile's coordinates now, so that they have
    // arrived when the tiles start
    struct Raw {
        float4 uv, sc;
        float2 w;
        uint32_t vi;
        bool in, flag;
    };
    const float4 *uvw2 = (const float4 *)g.uvw_f2;
    const float4 *sc2 = (const float4 *)g.scale_f2;
    auto load_raw = [&](Raw &r, int k) {
        r.in = k < d.kp;
        r.flag = false;
        if (r.in) {
            int tt, c;
            const size_t vi = vis_index(g, d, k, tt, c);
            const size_t bt = (size_t)d.bl * g.n_t + tt;
            r.uv = uvw2[2 * bt];
            const float4 w4 = uvw2[2 * bt + 1];
            r.w = make_float2(w4.x, w4.y);
            r.sc = sc2[c];
            r.vi = (uint32_t)vi;
            r.flag = flags && flags[vi];
        }
    };
    Raw r0 = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), make_float2(0.f, 0.f), 0u, false,
              false},
        r1 = r0;
    if (warp == COEF_WARP && n_tiles > 0) {
        load_raw(r0, lane);
        load_raw(r1, lane + 32);
    }
    // the prologue's other global reads, issued while the copies run: the taper of this
    // thread's pixels and the remainder r(x, y) of its B entries
    constexpr int NPIX = (SPIX + NT - 1) / NT;
    float tw_pre[NPIX];
#pragma unroll
    for (int i = 0; i < NPIX; ++i) tw_pre[i] = tid + i * NT < SPIX ? taper[tid + i * NT] : 0.0f;
    constexpr int NWT = C::NWT;
    float rr_pre[NWT];
#pragma unroll
    for (int i = 0; i < NWT; ++i) {
        const int wt = warp + MMA_WARP * i;
        const int yb = (wt / C::XC) % C::YB, xc = wt % C::XC;
        rr_pre[i] = warp < MMA_WARP && wt < C::NTASK
                        ? g.sep[2 * SL + (8 * yb + (lane >> 2)) * SL + 4 * xc + (lane & 3)]
                        : 0.0f;
    }
    __syncthreads();      // the copies' barriers are initialised

    // ---- prologue: the corrected image P = taper A_p I A_q^H into the planes
    if (FUSED) {
        bool late = false;
        wait_or_fail(smem_u32(&s_gbar), 0u, late);
        if (late) atomicExch(&g_sepd_error, 1);
        const float4 *rows = (const float4 *)(smem + B0H_OFF);
        for (int pix = tid; pix < SPIX; pix += NT) {
            const int i = pix / SL, j = pix % SL;
            const float sg = ((i + j) & 1) ? -1.0f : 1.0f;
            const float4 a = rows[2 * pix], b = rows[2 * pix + 1];
            s_fft[(0 * SL + i) * FFT_P + j] = make_float2(sg * a.x, sg * a.y);
            s_fft[(1 * SL + i) * FFT_P + j] = make_float2(sg * a.z, sg * a.w);
            s_fft[(2 * SL + i) * FFT_P + j] = make_float2(sg * b.x, sg * b.y);
            s_fft[(3 * SL + i) * FFT_P + j] = make_float2(sg * b.z, sg * b.w);
        }
        __syncthreads();
        if constexpr (SL == 32)
            fft2_planar_pairs32<+1>(s_fft, tid);
        else
            fft2_planar<SL, +1>(s_fft, tid, NT);
    }
    if (aterms) {
        bool late = false;
        wait_or_fail(smem_u32(&s_atbar), 0u, late);
        if (late) atomicExch(&g_sepd_error, 1);
    }
    float m = 0.0f;
#pragma unroll
    for (int ip = 0; ip < NPIX; ++ip) {
        const int pix = tid + ip * NT;
        if (pix >= SPIX) break;
        const int y = pix / SL, x = pix % SL;
        M22 P;
        if (FUSED) {      // (-1)^(x+y) / L^2 of the transform
            const float sg = ((x + y) & 1) ? -1.0f / SPIX : 1.0f / SPIX;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = s_fft[(q * SL + y) * FFT_P + x];
                P.m[q] = make_float2(sg * v.x, sg * v.y);
            }
        } else {
            P = load_m22(src + 2 * pix);
        }
        if (d.dws != 0.0f) {      // the sums use w_s: the rest of the w offset, exp(-i 2 pi (w_s - w0) n')
            float sn, cs;
            sincospif(d.dws * g.nprime[pix], &sn, &cs);     // (dws in half turns: exact reduction)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                P.m[q] = make_float2(P.m[q].x * cs + P.m[q].y * sn, P.m[q].y * cs - P.m[q].x * sn);
        }
        if (aterms) {
            const float4 *at = (const float4 *)(smem + AT_OFF);
            const M22 Ap = load_m22(at + 2 * pix);
            const M22 Aq = load_m22(at + 2 * (SPIX + pix));
            P = mul_mul_herm(Ap, P, Aq);
        }
        const float tw = tw_pre[ip];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 v = make_float2(tw * P.m[q].x, tw * P.m[q].y);
            s_fft[(q * SL + y) * FFT_P + x] = v;
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) s_red[warp] = m;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    m = 0.0f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) m = fmaxf(m, s_red[w]);
    int e2 = 0;
    if (m > 0.0f) frexpf(m, &e2);
    const float scale = ldexpf(1.0f, 10 - e2);
    const float inv_scale = ldexpf(1.0f, e2 - 10);
    // B: Q0 = scale P (hi and lo), Q1 = scale r P / sigma (hi), rows L q + y; one core matrix
    // (8 rows y, 4 x) per warp store: warp-task wt = (q, y block, x chunk of 4)
    if (warp < MMA_WARP) {
        const float rs = scale / g.c_scale;
#pragma unroll
        for (int i = 0; i < NWT; ++i) {
            const int wt = warp + MMA_WARP * i;
            if (wt >= C::NTASK) break;
            const int q = wt / (C::YB * C::XC), yb = (wt / C::XC) % C::YB, xc = wt % C::XC;
            const int y = 8 * yb + (lane >> 2), x = 4 * xc + (lane & 3);
            const float2 p = s_fft[(q * SL + y) * FFT_P + x];
            const float rr = rr_pre[i] * rs;
            uint32_t h0, l0;
            split_e(p.x * scale, p.y * scale, h0, l0);
            const uint32_t h1 = pack_f16x2(p.x * rr, p.y * rr);
            const uint32_t off = (uint32_t)(C::YB * q + yb) * kSBO + (uint32_t)(xc & 1) * kLBO + (uint32_t)(lane >> 2) * 16 +
                                 (uint32_t)(lane & 3) * 4;
            const int kk = xc >> 1;
            *(uint32_t *)(smem + B0H_OFF + kk * T4K + off) = h0;
            *(uint32_t *)(smem + B0L_OFF + kk * T4K + off) = l0;
            *(uint32_t *)(smem + B1H_OFF + kk * T4K + off) = h1;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();      // B complete; the planes (over the A stages) are free

    bool failed = false;
    if (warp == MMA_WARP) {
        if (lane == 0) {
            const uint64_t da0 = smem_desc(smem_u32(smem + A_OFF));
            const uint64_t db0 = smem_desc(smem_u32(smem + B0H_OFF));
            for (int t = 0; t < n_tiles; ++t) {
                const int s = t & 1, e = t & 3;
                wait_or_fail(smem_u32(&s_afull[s]), (uint32_t)((t >> 1) & 1), failed);
                if (t >= EST) wait_or_fail(smem_u32(&s_dempty[e]), (uint32_t)(((t >> 2) - 1) & 1), failed);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dt = tmem + 128u * (uint32_t)e;
#pragma unroll
                for (int kk = 0; kk < KT; ++kk) {
                    const uint64_t da = da0 + (uint64_t)((s * A_STAGE + kk * T4K) >> 4);     // m = 0 hi
                    const uint64_t db = db0 + (uint64_t)((kk * T4K) >> 4);                  // Q0 hi
                    mma_ss_i(dt, da, db, C::IDESC_N, kk > 0 ? 1u : 0u);
                    mma_ss_i(dt, da, db + (uint64_t)((KT * T4K) >> 4), C::IDESC_N, 1u);        // Q0 lo
                    mma_ss_i(dt, da + (uint64_t)((KT * T4K) >> 4), db, C::IDESC_N, 1u);        // m = 0 lo
                    mma_ss_i(dt, da + (uint64_t)((2 * KT * T4K) >> 4), db + (uint64_t)((2 * KT * T4K) >> 4),
                             C::IDESC_N, 1u);                                                // m = 1 hi x Q1 hi
                }
                commit(smem_u32(&s_aempty[s]));
                commit(smem_u32(&s_dfull[e]));
            }
            commit(smem_u32(&s_drain));
            bool drained = false;
            wait_or_fail(smem_u32(&s_drain), 0u, drained);     // bounded: let own MMAs finish before the free
        }
        failed = __shfl_sync(0xffffffffu, failed, 0);
    } else if (warp < NPW) {
        // ---- producers: coefficients, A (2 x 2 embedding of Ex*) and the Ey* table per tile.
        // A rows are (re/im, k): row k = (Re E, -Im E), row 64 + k = (Im E, Re E).  Lane = 4 k_lo + x_lo:
        // warp w owns x = 4 w + x_lo (K step w / 2, chunk w % 2) and writes visibilities 8 kg + k_lo
        const int klo = lane >> 2, xlo = lane & 3, x = 4 * warp + xlo;
        const bool x_ok = SL == 32 || 4 * warp < SL;    // warps past the last x only keep the protocol
        const float Xv = (float)(x - SL / 2), sx = g.sep[x_ok ? x : 0], csig = g.c_scale;
        const uint32_t a_off = (uint32_t)(warp >> 1) * T4K + (uint32_t)(warp & 1) * kLBO + (uint32_t)klo * 16 +
                               (uint32_t)xlo * 4;
        for (int t = 0; t < n_tiles; ++t) {
            const int s = t & 1, e = t & 3;
            if (t >= AST) wait_or_fail(smem_u32(&s_aempty[s]), (uint32_t)(((t >> 1) - 1) & 1), failed);
            wait_or_fail(smem_u32(&s_eyfull[e]), (uint32_t)((t >> 2) & 1), failed);      // the tile's coefficients
            const float4 *cf = s_coef + e * TV;
            uint8_t *As = smem + A_OFF + s * A_STAGE;
#pragma unroll 2
            for (int kg = 0; kg < TV / 8; ++kg) {
                if (!x_ok) break;
                const float4 c = cf[8 * kg + klo];
                float sn, cs;
                __sincosf(fmaf(c.z, sx, c.x * Xv), &sn, &cs);
                // m = 0: a = E = cs - i sn: row re = (cs, sn), row im = (-sn, cs); the im row is the re
                // row with halves swapped and the new low half negated (exact for FP16 parts)
                uint32_t hr, lr;
                split_e(cs, sn, hr, lr);
                const uint32_t hm = __byte_perm(hr, 0u, 0x1032u) ^ 0x8000u;
                const uint32_t lm = __byte_perm(lr, 0u, 0x1032u) ^ 0x8000u;
                // m = 1: a = -i c sigma E = -c sigma (sn + i cs): row re = (-c sigma sn, c sigma cs)
                const float cz = c.z * csig;
                const uint32_t h1r = pack_f16x2(-cz * sn, cz * cs);
                const uint32_t h1m = __byte_perm(h1r, 0u, 0x1032u) ^ 0x8000u;
                const uint32_t o_re = a_off + (uint32_t)kg * kSBO, o_im = o_re + 8 * kSBO;
                *(uint32_t *)(As + o_re) = hr;
                *(uint32_t *)(As + o_im) = hm;
                *(uint32_t *)(As + KT * T4K + o_re) = lr;
                *(uint32_t *)(As + KT * T4K + o_im) = lm;
                *(uint32_t *)(As + 2 * KT * T4K + o_re) = h1r;
                *(uint32_t *)(As + 2 * KT * T4K + o_im) = h1m;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_afull[s]));
        }
        if (failed && lane == 0) atomicExch(&g_sepd_error, 1);
    } else if (warp == COEF_WARP) {
        // ---- coefficients: lane l stages visibilities l and l + 32 of each tile: (a, b, c) from
        // float pairs (error-free FP32 products and sums, rounded once) and the output index (flag
        // in bit 31); the coordinates of the next tile are loaded while this one is formed, and a
        // stage is reused once the consumers release it (the first tile's were loaded before
        // the prologue)
        auto form = [&](const Raw &r) {
            float4 cf = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xFFFFFFFFu));   // beyond K_p: no output
            if (r.in) {
                cf.x = pair_coef(r.uv.x, r.uv.y, r.sc.x, r.sc.y, d.a0h, d.a0l);
                cf.y = pair_coef(r.uv.z, r.uv.w, r.sc.x, r.sc.y, d.b0h, d.b0l);
                cf.z = pair_coef(r.w.x, r.w.y, r.sc.z, r.sc.w, d.csh, d.csl);
                cf.w = __uint_as_float(r.vi | (r.flag ? 0x80000000u : 0u));
            }
            return cf;
        };
        for (int t = 0; t < n_tiles; ++t) {
            const int e = t & 3;
            const float4 c0 = form(r0), c1 = form(r1);
            if (t + 1 < n_tiles) {
                load_raw(r0, (t + 1) * TV + lane);
                load_raw(r1, (t + 1) * TV + lane + 32);
            }
            if (t >= EST) wait_or_fail(smem_u32(&s_eyempty[e]), (uint32_t)(((t >> 2) - 1) & 1), failed);
            s_coef[e * TV + lane] = c0;
            s_coef[e * TV + lane + 32] = c1;
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_eyfull[e]));
        }
        if (failed && lane == 0) atomicExch(&g_sepd_error, 1);
    } else {
        // ---- consumers: row 32 (warp % 4) + lane = (re/im = row / 64, k = row % 64) of the tile,
        // polarisations 2 h, 2 h + 1; the re and im rows of a visibility meet through s_part
        const int qq = warp & 3, h = (warp - NPW) >> 2;
        const int ci = qq >> 1, kl = 32 * (qq & 1) + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * qq) << 16);
        // Ey* entries: visibility ke = ctid % TV, rows y = 2 p, 2 p + 1 of the pairs p = ctid / TV + 4 j
        // (ctid = consumer thread index); entry (p, k) = (cs_2p, cs_2p+1, -sn_2p, -sn_2p+1)
        const int ctid = tid - NP, ke = ctid & (TV - 1), p0 = ctid >> 6;
        constexpr int EYP = C::EYP;               // pairs per thread
        float tys[2 * EYP];
#pragma unroll
        for (int j = 0; j < EYP; ++j) {
            tys[2 * j] = g.sep[SL + 2 * (p0 + 4 * j)];
            tys[2 * j + 1] = g.sep[SL + 2 * (p0 + 4 * j) + 1];
        }
        for (int t = 0; t < n_tiles; ++t) {
            const int s = t & 1, e = t & 3;
            wait_or_fail(smem_u32(&s_eyfull[e]), (uint32_t)((t >> 2) & 1), failed);
            // Ey*_k(y) = exp(-i (b_k Y + c_k t(y))) of the tile (entry y TV + k), while its MMAs run
            float4 *eyw = s_ey + s * (SL / 2 * TV);     // [L / 2 pairs][TV]
            {
                const float4 c = s_coef[e * TV + ke];
#pragma unroll
                for (int j = 0; j < EYP; ++j) {
                    const int pp = p0 + 4 * j;
                    float sn0, cs0, sn1, cs1;
                    __sincosf(fmaf(c.z, tys[2 * j], c.y * (float)(2 * pp - SL / 2)), &sn0, &cs0);
                    __sincosf(fmaf(c.z, tys[2 * j + 1], c.y * (float)(2 * pp + 1 - SL / 2)), &sn1, &cs1);
                    eyw[pp * TV + ke] = make_float4(cs0, cs1, -sn0, -sn1);
                }
            }
            consumers_sync();
            wait_or_fail(smem_u32(&s_dfull[e]), (uint32_t)((t >> 2) & 1), failed);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const ulonglong2 *ey = (const ulonglong2 *)eyw;
            // [q'][(sum er T, sum ei T)], each as packed partial sums over the even and odd rows y
            f2_t accp[2][2];
#pragma unroll
            for (int q2 = 0; q2 < 2; ++q2) accp[q2][0] = accp[q2][1] = 0ull;
#pragma unroll 1
            for (int yc = 0; yc < SL / 8; ++yc) {    // rows y in [8 yc, 8 yc + 8)
                uint32_t r[2][8];
#pragma unroll
                for (int qp = 0; qp < 2; ++qp)       // columns 32 (2 h + q') + y
                    tmem_ld8_nowait(lane_base + 128u * (uint32_t)e + (uint32_t)(SL * (2 * h + qp) + 8 * yc), r[qp]);
                ulonglong2 ep[4];
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) ep[pp] = ey[(4 * yc + pp) * TV + kl];
#pragma unroll
                for (int qp = 0; qp < 2; ++qp) {
                    tmem_wait_ld8(r[qp]);
#pragma unroll
                    for (int pp = 0; pp < 4; ++pp) {
                        const f2_t v = f2_pack(__uint_as_float(r[qp][2 * pp]), __uint_as_float(r[qp][2 * pp + 1]));
                        accp[qp][0] = f2_fma(ep[pp].x, v, accp[qp][0]);
                        accp[qp][1] = f2_fma(ep[pp].y, v, accp[qp][1]);
                    }
                }
            }
            float acc[2][2];
#pragma unroll
            for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float lo, hi;
                    f2_unpack(accp[q2][c], lo, hi);
                    acc[q2][c] = lo + hi;
                }
            const float4 cfk = s_coef[e * TV + kl];
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(smem_u32(&s_dempty[e]));
                mbar_arrive(smem_u32(&s_eyempty[e]));
            }
            // exchange with the other row of the visibility: the re row holds (er Tr, ei Tr),
            // the im row (er Ti, ei Ti); Re(E T) = er Tr - ei Ti, Im(E T) = er Ti + ei Tr
            float *part = s_part + (size_t)(s * 2 + ci) * (2 * 4 * TV) + (size_t)h * 4 * TV;
#pragma unroll
            for (int q2 = 0; q2 < 2; ++q2) {
                part[(2 * q2) * TV + kl] = acc[q2][0];
                part[(2 * q2 + 1) * TV + kl] = acc[q2][1];
            }
            consumers_sync();
            const float *other = s_part + (size_t)(s * 2 + (ci ^ 1)) * (2 * 4 * TV) + (size_t)h * 4 * TV;
            // this thread writes polarisation q' = ci of the pair
            const int qp = ci;
            const float own0 = ci ? acc[1][0] : acc[0][0];
            const float own1 = ci ? acc[1][1] : acc[0][1];
            const float oth0 = other[(2 * qp) * TV + kl], oth1 = other[(2 * qp + 1) * TV + kl];
            const float a0 = ci ? oth0 : own0, a1 = ci ? oth1 : own1;     // er Tr, ei Tr
            const float b0 = ci ? own0 : oth0, b1 = ci ? own1 : oth1;     // er Ti, ei Ti
            const uint32_t vw = __float_as_uint(cfk.w);       // index (< 2^31 - 1), bit 31 = flagged
            if (!(vw & 0x80000000u) && !failed) {
                ((float2 *)vis_out)[4 * (size_t)vw + 2 * h + qp] = make_float2((a0 - b1) * inv_scale, (b0 + a1) * inv_scale);
            } else if (vw != 0xFFFFFFFFu && !failed) {
                ((float2 *)vis_out)[4 * (size_t)(vw & 0x7FFFFFFFu) + 2 * h + qp] = make_float2(0.f, 0.f);   // flagged
            }
        }
        if (failed && lane == 0) atomicExch(&g_sepd_error, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == MMA_WARP) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(512));
}

// one CTA per subgrid of one plan (plan index idx[b] or first + b; image b of sub)
template <int L>
__global__ void __launch_bounds__(NT, 1)
degridder_sep_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ sub,
                     const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                     const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    degridder_sep_body<L, false>(g, g.sub[sid], sub + (size_t)blockIdx.x * L * L * 2, flags, aterms, taper, vis_out);
}

// fused: one CTA per subgrid, read from the grid
template <int L>
__global__ void __launch_bounds__(NT, 1)
degridder_sep_fused_kernel(Geometry g, const int32_t *__restrict__ idx, int64_t first, const float4 *__restrict__ grid,
                           const uint8_t *__restrict__ flags, const float4 *__restrict__ aterms,
                           const float *__restrict__ taper, float4 *__restrict__ vis_out) {
    allow_dependents();
    const int sid = idx ? idx[blockIdx.x] : (int)(first + blockIdx.x);
    degridder_sep_body<L, true>(g, g.sub[sid], grid, flags, aterms, taper, vis_out);
    complete_after_primary();
}

template <int L>
idg_status launch_sepd_set(bool fused, const Geometry &g, const SubgridSet &set, const void *src, const uint8_t *flags,
                           const void *aterms, const float *taper, void *vis_out, cudaStream_t s) {
    auto kern = fused ? degridder_sep_fused_kernel<L> : degridder_sep_kernel<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SepD<L>::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "separable degridder smem attribute");
    kern<<<(unsigned)set.count, NT, SepD<L>::SMEM, s>>>(g, set.idx, set.first, (const float4 *)src, flags,
                                                       (const float4 *)aterms, taper, (float4 *)vis_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? IDG_OK
                            : cuda_fail(e, fused ? "separable fused degridder launch" : "separable degridder launch");
}

}  // namespace

cudaError_t prepare_sep_batch_kernels() {
    cudaError_t e = prepare_gridder_sep_batch();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(degridder_sep_fused_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SepD<32>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(degridder_sep_fused_kernel<24>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SepD<24>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(degridder_sep_fused_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SepD<16>::SMEM);
    return e;
}


idg_status launch_degridder_sep(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                const void *aterms, const float *taper, void *vis_out, void *stream) {
    if (!separable_size(g.L) || !g.separable)
        return fail(IDG_ERR_UNSUPPORTED, "the separable degridder needs L = 32, 24 or 16 and a separable plan");
    if (set.count <= 0) return IDG_OK;
    switch (g.L) {
    case 32: return launch_sepd_set<32>(false, g, set, sub, flags, aterms, taper, vis_out, (cudaStream_t)stream);
    case 24: return launch_sepd_set<24>(false, g, set, sub, flags, aterms, taper, vis_out, (cudaStream_t)stream);
    default: return launch_sepd_set<16>(false, g, set, sub, flags, aterms, taper, vis_out, (cudaStream_t)stream);
    }
}

// a batch's launch of the fused kernel over one job's items (the shared-memory attribute
// is set by prepare_tcw_batch_kernels, outside graph capture); pdl: see launch_pdl
idg_status launch_degridder_sep_job(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *vis_out, void *stream, bool pdl) {
    if (set.count <= 0) return IDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned n = (unsigned)set.count;
    const float4 *gr = (const float4 *)grid, *at = (const float4 *)aterms;
    float4 *o = (float4 *)vis_out;
    cudaError_t e;
    switch (g.L) {
    case 32: e = launch_pdl(degridder_sep_fused_kernel<32>, n, NT, SepD<32>::SMEM, s, pdl, g, set.idx, set.first, gr, flags, at, taper, o); break;
    case 24: e = launch_pdl(degridder_sep_fused_kernel<24>, n, NT, SepD<24>::SMEM, s, pdl, g, set.idx, set.first, gr, flags, at, taper, o); break;
    case 16: e = launch_pdl(degridder_sep_fused_kernel<16>, n, NT, SepD<16>::SMEM, s, pdl, g, set.idx, set.first, gr, flags, at, taper, o); break;
    default: return fail(IDG_ERR_UNSUPPORTED, "the separable degridder needs L = 32, 24 or 16");
    }
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, "separable degridder job launch");
}

idg_status launch_degridder_sep_fused(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                      const void *aterms, const float *taper, void *vis_out, void *stream) {
    if (!separable_size(g.L) || !g.separable)
        return fail(IDG_ERR_UNSUPPORTED, "the separable degridder needs L = 32, 24 or 16 and a separable plan");
    if (set.count <= 0) return IDG_OK;
    switch (g.L) {
    case 32: return launch_sepd_set<32>(true, g, set, grid, flags, aterms, taper, vis_out, (cudaStream_t)stream);
    case 24: return launch_sepd_set<24>(true, g, set, grid, flags, aterms, taper, vis_out, (cudaStream_t)stream);
    default: return launch_sepd_set<16>(true, g, set, grid, flags, aterms, taper, vis_out, (cudaStream_t)stream);
    }
}

idg_status read_sepd_error(int *code) {
    int zero = 0, v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_sepd_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_sepd_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the separable degridder error word");
    *code = v;
    return IDG_OK;
}

}  // namespace idg
