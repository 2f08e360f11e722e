// Private declarations shared by the library's translation units.
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/idg.h"

namespace idg {

constexpr double kSpeedOfLight = 299792458.0;   // m/s
constexpr int kDescFields = IDG_DESC_FIELDS;

// Work description of one subgrid on the device (112 B, 16-B aligned).
struct alignas(16) DevSubgrid {
    int32_t bl, slot, t0, nt, c0, nc, q0, r0, layer, kp, st_p, st_q;
    double u0, v0, w0;     // centre of the subgrid in wavelengths (Sect. 3.3)
    // the phase offsets of the centre as float pairs (hi + lo = the FP64 value to
    // about 2^-48): u0 k_uv, v0 k_uv and 2 pi w0
    float a0h, a0l, b0h, b0l, c0h, c0l;
    // the separable kernels' w offset w_s (w0, or the middle of the subgrid's w range
    // when it needs that to meet the remainder bound): 2 pi w_s as a float pair, and
    // 2 (w_s - w0), the phase in half turns per unit of n' they apply to the subgrid image
    float csh, csl, dws;
};
static_assert(sizeof(DevSubgrid) == 112, "DevSubgrid layout");

// Geometry and pointers the kernels read; passed by value to every launch.
struct Geometry {
    int L, N, n_t, n_chan, n_stations;
    double S;             // N * cell: image size in direction cosines
    double k_uv;          // 2 pi S / L: phase per pixel index per wavelength
    const DevSubgrid *sub;     // [n_sub], plan order
    const int32_t *order;      // [n_sub], device work order (plan indices)
    const double *uvw;         // [n_bl][n_t][3] metres
    const double *scale;       // [n_chan] f / c
    // float-pair copies (hi + lo = the FP64 value to about 2^-48) for coefficient
    // arithmetic without FP64 instructions, 16-B aligned: uvw_f2[8 (bl n_t + t) ..]
    // = (u hi, u lo, v hi, v lo, w hi, w lo, 0, 0) in metres; scale_f2[4 c ..] =
    // (k_uv f/c hi, lo, 2 pi f/c hi, lo)
    const float *uvw_f2;
    const float *scale_f2;
    const float *nprime;       // [L][L] n' = sqrt(1 - l^2 - m^2) - 1
    double ds;                 // channel scale step (f_{c+1} - f_c)/c for uniformly spaced channels
    int recurrence;            // 1: phasors by channel recurrence (IDG_PHASOR_RECURRENCE)
    int anchor;                // channels per recurrence run (re-anchor interval)
    // separable split n'(x, y) = s(x) + t(y) + r(x, y): s(x) = n'(x, j0),
    // t(y) = n'(j0, y) - n'(j0, j0) (j0 the reference row and column that makes
    // max |r| smallest), r the remainder; sep = [s[L] | t[L] | r[L][L]] (FP64
    // differences rounded to FP32)
    const float *sep;
    // 1: the launch's subgrids meet the bound max |c_k| max |r| of the first-order w
    // remainder (the plan's own value: every subgrid does; the composite calls set it
    // per launch for the separable part of a plan)
    int separable;
    float c_scale;             // power of two with max |c_k| c_scale <= 1 over the separable subgrids (c_k = 2 pi (w - w_s))
    float r_scale;             // power of two with max |r(x, y)| r_scale <= 1
};

// Host planner output.
struct PlanResult {
    std::vector<int32_t> desc;   // kDescFields per subgrid, plan order
    int64_t n_dropped = 0;
    int32_t n_w = 1;
    int32_t k_min = 0;
};

struct PlanParams {
    const double *uvw;
    const double *freqs;
    const int32_t *aterm_offsets;
    int n_bl, n_t, n_chan, n_slots;
    int L, N;
    double cell, w_step, beta;
    int t_max;
    int n_threads;
};

// Sect. 3.2 partition; deterministic and independent of n_threads.
PlanResult make_plan(const PlanParams &p);

}  // namespace idg

struct idg_plan {
    idg_plan_options opts;
    idg_plan_stats stats;
    int n_bl, n_t, n_chan, n_stations, n_slots, L, N;
    double cell, w_step, S;
    std::vector<int32_t> desc;          // host copy, plan order
    std::vector<int32_t> baselines;     // [n_bl][2]
    int device = -1;
    // device metadata (owned)
    idg::DevSubgrid *d_sub = nullptr;
    int32_t *d_order = nullptr;
    double *d_uvw = nullptr;
    double *d_scale = nullptr;
    float *d_uvw_f2 = nullptr;             // float-pair copies for the coefficient arithmetic
    float *d_scale_f2 = nullptr;
    float *d_nprime = nullptr;             // [L][L] n', then the separable tables [2 L + L^2]
    double sep_theta = 0.0;                // max |c_k| max |r(x, y)|: phase of the separable remainder
    int sep_j0 = 0;                        // reference row and column of the separable split
    // per subgrid (plan order): the separable kernels' w offset w_s (wavelengths), and
    // 1 where the remainder phase with it meets the bound (the separable kernels take it)
    std::vector<double> w_sep;
    std::vector<uint8_t> sep_sub;
    // [n + 1] number of separable subgrids before each position of the work, plan and
    // span orders (the work order and each span list the separable subgrids first)
    std::vector<int64_t> sep_prefix_order, sep_prefix_plan, sep_prefix_span;
    // pieces: the composite calls may take a subgrid outside the bound as kt x kc blocks of
    // its timesteps and channels, each within the bound with its own w_s, at the subgrid's
    // position with its taper and A-terms (the sums are linear in the visibilities, so the
    // pieces add up to the subgrid).  Their descriptors follow the plan's in d_sub.
    struct Piece {
        int32_t parent, t0, nt, c0, nc;
        double ws;
    };
    std::vector<Piece> pieces;
    std::vector<uint8_t> split_sub;        // [n_sub] 1: the composite calls take it in pieces
    std::vector<int32_t> kp_all;           // [n_sub + pieces] K_p of every d_sub entry
    // the composite calls' lists of d_sub entries when the plan has pieces: the separable
    // subgrids and the pieces, then the direct subgrids left (each part by K_p descending);
    // the same per span, span k at [fspan_first[k], fspan_first[k + 1])
    int32_t *d_fused_order = nullptr;
    int32_t *d_fused_span = nullptr;
    std::vector<int32_t> kp_fused_order, kp_fused_span;
    std::vector<int64_t> kp_prefix_fused, kp_prefix_fspan, sep_prefix_fused, sep_prefix_fspan;
    std::vector<int64_t> fspan_first;
    // IDG_ADDER_SORTED: the tiles of the grid that subgrids overlap, with those subgrids
    // (plan indices, ascending); see SortedTiles
    int32_t *d_tile_ids = nullptr;
    int32_t *d_tile_first = nullptr;
    int32_t *d_tile_sub = nullptr;
    int64_t n_tiles_sorted = 0;
    int64_t n_heavy_sorted = 0;
    float c_scale = 1.0f;
    float r_scale = 1.0f;
    bool any_dropped = false;
    double ds = 0.0;                        // uniform channel scale step (0 if not uniform)
    std::vector<int64_t> kp_prefix_plan;    // [n_sub + 1], sum of K_p in plan order
    std::vector<int64_t> kp_prefix_order;   // [n_sub + 1], sum of K_p in device work order
    std::vector<int32_t> kp_plan;           // [n_sub] K_p in plan order
    std::vector<int32_t> kp_order;          // [n_sub] K_p in device work order (separable subgrids
                                            // first, each part non-increasing)
    std::vector<int32_t> order;             // [n_sub] plan index of each work-order slot (host copy)
    // spans of whole baselines for the host-buffer calls: span k holds plan indices
    // [span_first[k], span_first[k + 1]) and baselines [span_bl[k], span_bl[k + 1]);
    // span_order lists each span's separable subgrids, then the others, each part by K_p
    // descending (positions as in plan order)
    std::vector<int64_t> span_first;
    std::vector<int32_t> span_bl;
    int32_t *d_span_order = nullptr;
    std::vector<int32_t> kp_span_order;
    std::vector<int64_t> kp_prefix_span;
    // default taper c[y][x] = a_y a_x of the PSWF window a of the plan's beta (device,
    // float32 [L][L]); used where a call passes a NULL taper
    float *d_taper = nullptr;
    float *d_ones = nullptr;               // [L][L] of 1.0f: the unit taper of the calibration's residual sums
    // the plan's own kernel choice per kernel (-1: the process-wide choice for its L);
    // the one part of a plan that may change after creation (idg_plan_set_kernel_variant,
    // idg_autotune), read once per call
    mutable std::atomic<int> variant[IDG_KERNEL_COUNT];

    idg_plan() {
        for (auto &v : variant) v.store(-1, std::memory_order_relaxed);
    }
    idg::Geometry geometry() const;
    // effective kernel variant of this plan for `kernel`
    int kernel_variant(int kernel) const;
    // the taper a call uses: its own, else the plan's default (NULL if the plan has none)
    const float *taper_or_default(const float *t) const { return t ? t : d_taper; }
};

namespace idg {

// device memory from the library's stream-ordered pool (kept across calls); free with
// cudaFreeAsync on the same stream
idg_status scratch_alloc(int device, size_t bytes, void *stream, void **p);

// thread-local error text
void set_error(const std::string &msg);
idg_status fail(idg_status st, const std::string &msg);
idg_status cuda_fail(int err, const char *what);

// event-based kernel timing (idg_profile_*); no-ops while disabled
struct ProfileScope {
    ProfileScope(int kernel, void *stream, double work);
    ~ProfileScope();
    int kernel;
    void *stream;
    void *ev[2];
    double work;
    bool on;
};

// A set of subgrids processed by one launch: block b works on plan index
// idx[b] (idx: device array) or, without idx, on first + b.  kp_host (host,
// count entries, may be null for the gridder) holds the members' K_p so a
// launcher can split the set into runs of equal work shape.
struct SubgridSet {
    const int32_t *idx;
    int64_t first;
    int64_t count;
    const int32_t *kp_host;
};

// kernel launchers (each returns IDG_OK or an error with the message set).
// variant < 0 selects the process-wide choice for L (see set_variant).
bool gridder_supported(int L);
int gridder_variant_count(int L);
const char *gridder_variant_name(int L, int v);
idg_status launch_gridder(const Geometry &g, const SubgridSet &set, int variant, const void *vis,
                          const uint8_t *flags, const void *aterms, const float *taper, void *subgrids,
                          void *stream);
int degridder_variant_count(int L);
const char *degridder_variant_name(int L, int v);
idg_status launch_degridder(const Geometry &g, const SubgridSet &set, int variant, const void *subgrids,
                            const uint8_t *flags, const void *aterms, const float *taper, void *vis_out,
                            void *stream);
idg_status launch_fft(int L, int64_t count, int direction, void *subgrids, void *stream);
idg_status launch_adder(const Geometry &g, const SubgridSet &set, const void *subgrids, void *grid, void *stream);
idg_status launch_splitter(const Geometry &g, const SubgridSet &set, const void *grid, void *subgrids, void *stream);
idg_status launch_adder_compensated(const Geometry &g, const SubgridSet &set, const void *subgrids, void *grid,
                                    void *comp, void *stream);
idg_status launch_fold_compensation(void *grid, const void *comp, size_t n_float4, void *stream);

// channel-recurrence forms (precision_mode = IDG_PHASOR_RECURRENCE)
idg_status launch_gridder_rec(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *subgrids, void *stream);
idg_status launch_degridder_rec(const Geometry &g, const SubgridSet &set, const void *subgrids,
                                const uint8_t *flags, const void *aterms, const float *taper, void *vis_out,
                                void *stream);

// tensor-core gridder (L = 32; FP16 hi/lo split products, FP32 accumulation in
// tensor memory) and the device error word of the bounded waits
// subgrid sizes the separable tensor-core kernels are built for (32, 24 and 16)
bool separable_size(int L);
// The fused (and one-CTA-per-subgrid) degridders pay a fixed prologue per subgrid, so a
// launch takes them only when at least half its visibilities lie in subgrids of at least
// this many: 512 for the direct tensor-core degridder; for the separable one, whose
// per-visibility cost is lower, 64 (on the precision workload's subgrids of 256 the fused
// separable degridder took 29.4 ms against 63.1 ms for splitter, transform and the
// packed-FP32 degridder).
constexpr int32_t kTcwFusedKpMin = 512;
constexpr int32_t kSepFusedKpMin = 64;
// separable tensor-core gridder (L = 32, 24 or 16, g.separable): subgrid images, or fused
// with the transform and the adder into grid
idg_status launch_gridder_sep(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *out, void *stream);
idg_status launch_gridder_sep_fused(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *grid, void *stream);
idg_status read_sep_error(int *code);
// separable tensor-core degridder (L = 32, 24 or 16, g.separable): from subgrid images, or
// fused with the splitter and the inverse transform from grid
idg_status launch_degridder_sep(const Geometry &g, const SubgridSet &set, const void *sub, const uint8_t *flags,
                                const void *aterms, const float *taper, void *vis_out, void *stream);
idg_status launch_degridder_sep_fused(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                      const void *aterms, const float *taper, void *vis_out, void *stream);
idg_status read_sepd_error(int *code);
idg_status launch_gridder_tcw(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *subgrids, void *stream);
idg_status read_device_errors(int *code, void *stream);
// tensor-core degridder (L = 32) and its device error word
idg_status launch_degridder_tcw(const Geometry &g, const SubgridSet &set, const void *subgrids, const uint8_t *flags,
                                const void *aterms, const float *taper, void *vis_out, void *stream);
idg_status read_tcd_error(int *code);
// error word of the bounded-wait self-test kernel (selftest.cu)
idg_status read_selftest_error(int *code);
// fused forms (L = 32): the gridder transforms each subgrid in shared memory and adds it
// into `grid` (accumulated); the degridder splits and transforms from `grid`
idg_status launch_gridder_tcw_fused(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *grid, void *stream);
idg_status launch_degridder_tcw_fused(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                      const void *aterms, const float *taper, void *vis_out, void *stream);
// the sorted (deterministic) adder's tiles: kTile x kTile grid pixels per layer; for each of
// the n_tiles tiles that subgrids overlap, its id (layer (ntx ntx) + ty ntx + tx, ntx =
// ceil(N / kTile)) and the plan indices of those subgrids, ascending, at
// tile_sub[tile_first[k] .. tile_first[k + 1]) (device arrays).  The rows of tiles whose
// list is longer than kHeavyEntries come last (n_heavy of them); each takes a cluster of
// kHeavyCluster CTAs
constexpr int kTile = 32;
constexpr int kHeavyEntries = 64;
constexpr int kHeavyCluster = 8;
struct SortedTiles {
    const int32_t *tile_ids;
    const int32_t *tile_first;
    const int32_t *tile_sub;
    int64_t n_tiles;
    int64_t n_heavy;
};
// adds the images of the set's subgrids (consecutive plan indices: set.first + i in scratch
// slot i) into the grid tile by tile in plan-index order
idg_status launch_adder_sorted(const Geometry &g, const SubgridSet &set, const void *sub, void *grid,
                               const SortedTiles &t, void *stream);
// the fused kernels of one job of a batch (the plan's geometry, a set of its d_sub entries),
// as a programmatic dependent launch when pdl (see tc_common.cuh)
idg_status launch_gridder_sep_job(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                  const void *aterms, const float *taper, void *grid, void *stream, bool pdl);
idg_status launch_degridder_sep_job(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *vis_out, void *stream, bool pdl);
idg_status launch_gridder_tcw_job(const Geometry &g, const SubgridSet &set, const void *vis, const uint8_t *flags,
                                  const void *aterms, const float *taper, void *grid, void *stream, bool pdl);
idg_status launch_degridder_tcw_job(const Geometry &g, const SubgridSet &set, const void *grid, const uint8_t *flags,
                                    const void *aterms, const float *taper, void *vis_out, void *stream, bool pdl);

// calibration (calibration.cu): residuals and cost over the visibilities of a subgrid
// set (res holds the model visibilities on entry), and the A-term gradient from the
// residual images R and the model images P of the set (chunk positions)
idg_status launch_calib_residual(const Geometry &g, const SubgridSet &set, const void *obs, const uint8_t *flags,
                                 void *res, double *cost, void *stream);
idg_status launch_calib_gradient(const Geometry &g, const SubgridSet &set, const void *R, const void *P,
                                 const void *aterms, const float *taper, void *grad, void *stream);

// classical gridding with oversampled A/W-projection kernels (classical.cu)
size_t classical_kernels_smem(int M, int O);
size_t classical_grid_smem(int L, int M);
idg_status launch_classical_planes(const Geometry &g, int64_t n_sub, double dw, struct int2 *range, void *stream);
idg_status launch_classical_kernels(const Geometry &g, int M, int O, double dw, const float *taper,
                                    const void *aterms, const double *nprime, const struct int2 *sets,
                                    int64_t n_sets, void *tables, void *stream);
idg_status launch_classical_grid(const Geometry &g, int M, int O, double dw, const struct int2 *work,
                                 const int *jmin, int64_t count, const void *tables, const void *vis,
                                 const uint8_t *flags, void *grid, void *stream);
idg_status read_classical_error(int *code);

// tensor-core subgrid transform (fft_mode = IDG_FFT_TC_SPLIT; L = 32)
bool dft_tc_supported(int L);
idg_status launch_dft_tc(int L, int64_t count, int direction, void *subgrids, void *stream);
idg_status read_dft_error(int *code);
// the plan's transform (FP32 shared-memory FFT or the tensor-core form)
idg_status launch_subgrid_fft(const idg_plan *p, int64_t count, int direction, void *subgrids, void *stream);

// fused batch kernel shapes (batch.cu)
int batch_variant_count(int kernel, int L);
const char *batch_variant_name(int kernel, int L, int v);

// process-wide kernel variant choice per (kernel, L); default 0
int get_variant(int kernel, int L);
void set_variant(int kernel, int L, int v);

}  // namespace idg
