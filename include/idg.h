/*
 * idg.h -- C ABI of a single-GPU (sm_103a) implementation of Image Domain
 * Gridding (van der Tol, Veenboer & Offringa, "Image Domain Gridding: a fast
 * method for convolutional resampling of visibilities", A&A 2018).
 *
 * The library implements the data-parallel part of the method: the partition
 * of the visibilities into subgrids (Sect. 3.2), the per-subgrid gridder and
 * degridder (Algorithms 1 and 2, inner loops; Eq. ShiftedDirectImaging), the
 * image-domain kernel of taper and per-station 2x2 A-terms (Sect. 3.4), the
 * batched subgrid transform ("FFT"/"IFFT" of Algorithms 1 and 2) and the adder
 * and splitter that move subgrids to and from the master uv grid.
 *
 * Conventions (all arrays C-contiguous, little-endian):
 *   visibility   complex64 (8 B: re, im float32) [n_bl][n_t][n_chan][4], pol
 *                order XX, XY, YX, YY = the 2x2 matrix [[XX, XY], [YX, YY]];
 *   uvw          float64 [n_bl][n_t][3], metres (uvw = x_q - x_p of baseline (p,q));
 *   frequency    float64 [n_chan], Hz (channel centres);
 *   baselines    int32 [n_bl][2], station pair (p, q);
 *   A-terms      complex64 [n_slots][n_stations][L][L][4], the Jones matrix of a
 *                station sampled at subgrid pixel (y, x); slot a covers the
 *                timesteps [aterm_offsets[a], aterm_offsets[a+1]);
 *   taper        float32 [L][L], real, centre pixel (L/2, L/2) normally 1;
 *   grid         complex64 [n_w][N][N][4], row index v, column index u;
 *                pixel q of an axis has uv coordinate (q - N/2)/S, S = N * cell;
 *   subgrid      complex64 [L][L][4] (uv or image domain).
 * Subgrid image pixel (y, x) sits at l = (x - L/2) S / L, m = (y - L/2) S / L,
 * n' = sqrt(1 - l^2 - m^2) - 1 (Sect. 2, pixel positions; Alg. 1/2 use n').
 *
 * Gridding (Alg. 1, without the final full-grid FFT and taper division):
 *   I_p[y][x] = sum_k V_k exp(+2 pi i ((u_k - u0) l + (v_k - v0) m + (w_k - w0) n'))
 *   I_p <- taper * A_p^H I_p A_q                     (per pixel, 2x2 products)
 *   V_p[i][j] = L^-2 sum_{y,x} I_p[y][x] exp(-2 pi i ((j-L/2)(x-L/2) + (i-L/2)(y-L/2)) / L)
 *   grid[layer][r0 + i][q0 + j] += V_p[i][j]
 * Degridding (Alg. 2, after the full-image steps) is its exact adjoint:
 *   V_p = grid[layer][r0..][q0..];  I_p = L^-2 sum V_p exp(+2 pi i ...);
 *   I_p <- taper * A_p I_p A_q^H;  y_k = sum_{y,x} I_p exp(-2 pi i (...)).
 *
 * Ownership: the caller owns every data buffer; device pointers are plain CUDA
 * device (or managed) addresses, host pointers plain host memory.  A plan owns
 * its own host and device metadata and is immutable after creation, except for
 * its kernel choice (idg_plan_set_kernel_variant, idg_autotune), which each call
 * reads once when it starts; it may be used from several host threads and
 * streams at once, and one plan's kernel choice does not affect another plan.
 * Device calls are asynchronous and stream-ordered on the stream given (NULL =
 * legacy default stream); a call returns after enqueueing.  Host-buffer
 * variants synchronise.
 *
 * Errors: every entry point returns an idg_status; nothing crosses the ABI as
 * an exception.  idg_last_error() returns a thread-local description of the
 * last failure on the calling thread.  Invalid arguments are rejected before
 * any work is enqueued.  No entry point aborts the process.
 */
#ifndef IDG_GB300_IDG_H
#define IDG_GB300_IDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct idg_plan idg_plan;
typedef struct CUstream_st *idg_stream;   /* the same type as cudaStream_t */

typedef enum {
    IDG_OK = 0,
    IDG_ERR_INVALID_ARG = 1,    /* a size, pointer or value is out of range        */
    IDG_ERR_NO_MEMORY = 2,      /* host or device allocation failed                */
    IDG_ERR_CUDA = 3,           /* a CUDA runtime call or launch failed            */
    IDG_ERR_TIMEOUT = 4,        /* a bounded device wait gave up                   */
    IDG_ERR_DEVICE_CHECK = 5,   /* a device-side consistency check failed          */
    IDG_ERR_UNSUPPORTED = 6     /* valid, but not built into this library (e.g. L) */
} idg_status;

/* Plan options.  Fill with idg_plan_options_default() and change fields. */
typedef struct {
    double kernel_size;              /* beta: main-lobe width of the uv kernel in
                                        pixels; allowed shift from the subgrid
                                        centre is (L - beta + 1)/2 (Sect. 4.3).
                                        Default 7 (Sect. 5.3, Table 1).          */
    int max_timesteps_per_subgrid;   /* T_max, default 128                        */
    int precision_mode;              /* IDG_PHASOR_* (see below)                  */
    int fft_mode;                    /* IDG_FFT_*                                  */
    int adder_mode;                  /* IDG_ADDER_*                                */
    int n_host_threads;              /* planner threads, 0 = hardware concurrency */
} idg_plan_options;

enum { IDG_PHASOR_SINCOS = 0,      /* FP32 sin/cos of every phase                  */
       IDG_PHASOR_RECURRENCE = 1 };/* channel recurrence, re-anchored periodically  */
enum { IDG_FFT_FP32 = 0,           /* FP32 FFT in shared memory                     */
       IDG_FFT_TC_SPLIT = 1 };     /* centred DFT as two matrix products on the tensor
                                      cores, FP16 hi/lo split operands (three products
                                      per stage), FP32 accumulation; subgrid size 32
                                      only (IDG_ERR_UNSUPPORTED otherwise)          */
enum { IDG_ADDER_ATOMIC = 0,       /* 16-byte vector atomic adds                    */
       IDG_ADDER_COMPENSATED = 1,  /* atomics + exact TwoSum error into a compensation
                                      grid folded in at the end (O(eps) instead of
                                      O(n eps) summation error; grid-sized scratch) */
       IDG_ADDER_SORTED = 2 };     /* deterministic: the gridding runs in plan order, in
                                      chunks of consecutive subgrids; one CTA per 32 x 32
                                      grid tile sums the chunk's subgrids that overlap
                                      it in plan order (plan-held tile lists) and adds
                                      the sum with plain stores; a tile that more than
                                      64 subgrids of the plan overlap takes a cluster of
                                      8 CTAs, fixed segments of its list summed apart and
                                      added in rank order.  The grid is the same bit for
                                      bit on every run (for a given plan, device and
                                      range boundaries), with no atomics.  Batches add
                                      with atomics whatever the plan's adder.       */

typedef struct {
    int64_t n_subgrids;       /* P, number of blocks                              */
    int64_t n_vis_planned;    /* sum of K_p (flags are not known to the plan)     */
    int64_t n_vis_dropped;    /* visibilities whose support is off the grid       */
    int64_t max_kp;           /* largest K_p                                      */
    int32_t n_w_layers;       /* layers of the grid (1 without W-layers)          */
    int32_t w_layer_min;      /* k of layer 0: w0(layer) = (layer + min) * w_step */
    int32_t subgrid_size;     /* L                                                */
    int32_t grid_size;        /* N                                                */
    int32_t n_bl, n_t, n_chan, n_stations, n_slots;
    int32_t device;           /* CUDA device holding the plan's metadata          */
    int32_t separable;        /* 1: every subgrid meets the remainder bound and the
                                 separable tensor-core kernels take the whole plan
                                 (L = 32, 24 or 16), see idg_grid                  */
    double sep_phase;         /* max over subgrids of |2 pi (w - w_s)| * max |r(x, y)|
                                 in radians, r the part of n' = sqrt(1 - l^2 - m^2) - 1
                                 that is not n'(l, m0) + n'(m0, m) - n'(m0, m0), for
                                 the pixel row m0 that makes max |r| smallest; w_s is
                                 the subgrid's w offset w0 when that meets the bound
                                 (1.38e-3), else the middle of the subgrid's own w
                                 range (the separable kernels then apply
                                 exp(+-2 pi i (w_s - w0) n') to the subgrid image)  */
    int64_t n_sep_subgrids;   /* subgrids whose phase with their w_s meets the bound:
                                 the separable kernels take these, the direct kernels
                                 the rest (0 when L is not 32, 24 or 16)           */
    int64_t n_vis_sep;        /* sum of K_p over those subgrids                    */
    int64_t n_split_subgrids; /* subgrids outside the bound that the composite calls
                                 take in pieces: kt x kc blocks of their timesteps and
                                 channels, each within the bound with its own w_s, at
                                 the subgrid's position (the sums are linear in the
                                 visibilities, so the pieces add up to the subgrid);
                                 split where the direct kernels' extra cost per
                                 visibility outweighs a piece's fixed cost        */
    int64_t n_pieces;         /* number of those pieces                           */
    int64_t n_vis_split;      /* sum of K_p over the split subgrids                */
} idg_plan_stats;

/* Number of int32 fields per exported subgrid descriptor, and their order. */
#define IDG_DESC_FIELDS 10
enum { IDG_DESC_BASELINE = 0, IDG_DESC_SLOT, IDG_DESC_T0, IDG_DESC_NT, IDG_DESC_C0,
       IDG_DESC_NC, IDG_DESC_Q0, IDG_DESC_R0, IDG_DESC_LAYER, IDG_DESC_KP };

void idg_plan_options_default(idg_plan_options *opts);

/*
 * Partition the visibilities into subgrids (Sect. 3.2, Fig. 2) and upload the
 * plan's metadata (descriptors, uvw, channel scales) to the current device.
 *
 * Block rule (deterministic): per baseline (input order), per A-term slot, the
 * smallest number G of contiguous channel groups (the first n_chan mod G groups
 * one channel larger) such that every single timestep of every group fits by
 * size; then, per group, timesteps are added in order while the block still
 * fits and has at most T_max timesteps.  A block fits when every sample's grid
 * pixel position pu = u/lambda * S + N/2 (and pv) lies within (L - beta + 1)/2
 * of the centre Cu = floor((min + max)/2 + 1/2), the box [Cu - L/2, Cu + L/2)
 * lies inside [0, N) on both axes, and (with w_step > 0) its w spread is at
 * most w_step.  A lone timestep that does not fit is dropped and counted.
 * Layers: k = floor(mid_w / w_step + 1/2), w0 = k * w_step; w_step = 0 means
 * a single layer with w0 = 0.  Descriptors are ordered (baseline, slot, group,
 * first timestep).  The plan is bit-identical on every host (FP64, no fused
 * multiply-add).
 *
 * uvw_m          [n_bl][n_t][3] float64, host, metres, finite
 * freqs_hz       [n_chan] float64, host, > 0, finite
 * baselines      [n_bl][2] int32, host, station indices in [0, n_stations)
 * aterm_offsets  [n_slots + 1] int32, host, 0 = off[0] < off[1] < ... = n_t
 * subgrid_size   L, even, L >= kernel_size + 1
 * grid_size      N, even, N >= L
 * cell_size_rad  pixel size of the image, > 0 (S = N * cell)
 * w_step_lambda  >= 0, W-layer spacing in wavelengths (0: no W-layers)
 * opts           NULL for defaults
 * out            receives the plan (NULL on failure)
 * Errors: IDG_ERR_INVALID_ARG (message says which argument, or that the plan's
 *         subgrids, pieces or sorted-adder tile lists exceed 32-bit indices),
 *         IDG_ERR_NO_MEMORY, IDG_ERR_CUDA.
 */
idg_status idg_plan_create(const double *uvw_m, const double *freqs_hz, const int32_t *baselines,
                           const int32_t *aterm_offsets, int n_bl, int n_t, int n_chan,
                           int n_stations, int n_slots, int subgrid_size, int grid_size,
                           double cell_size_rad, double w_step_lambda,
                           const idg_plan_options *opts, idg_plan **out);

/* Summary numbers of a plan (host only). */
idg_status idg_plan_info(const idg_plan *plan, idg_plan_stats *out);

/* Copy the descriptors, IDG_DESC_FIELDS int32 per subgrid in plan order, into
   desc[cap_subgrids][IDG_DESC_FIELDS] (host).  Fails with IDG_ERR_INVALID_ARG
   if cap_subgrids < n_subgrids. */
idg_status idg_plan_export(const idg_plan *plan, int32_t *desc, int64_t cap_subgrids);

/* Release the plan and its device metadata.  The caller must ensure that no
   work using the plan is still in flight.  NULL is ignored. */
void idg_plan_destroy(idg_plan *plan);

/*
 * Gridding, Algorithm 1 (subgrid images, taper and A-terms, subgrid FFT, adder).
 * d_vis     device complex64 [n_bl][n_t][n_chan][4]
 * d_flags   device uint8 [n_bl][n_t][n_chan], nonzero = flagged (weight 0), or NULL
 * d_aterms  device complex64 [n_slots][n_stations][L][L][4], or NULL = identity
 * d_taper   device float32 [L][L], or NULL for the plan's default taper
 *           c[y][x] = a_y a_x, a the PSWF window of the plan's kernel_size as
 *           idg_taper_window(L, kernel_size, IDG_TAPER_PSWF) gives it (Sect. 4.1),
 *           rounded to float32 and kept on the plan's device
 * d_grid    device complex64 [n_w][N][N][4]; the result is ADDED (Alg. 1 starts
 *           from V = 0: zero it first), so several plans may sum into one grid.
 * Summation order on the grid is not fixed (atomic adds): results agree with
 * the FP64 definition to FP32 rounding, not bit for bit across runs.
 * Device scratch of at most 512 MiB is taken from the stream-ordered allocator
 * (plus one grid-sized compensation buffer with IDG_ADDER_COMPENSATED).
 * At L = 32, and at L = 24 and 16 when the plan is separable, with the default
 * kernel choice, IDG_FFT_FP32, IDG_PHASOR_SINCOS and IDG_ADDER_ATOMIC the whole call is
 * one fused tensor-core launch (image-domain sum, taper and A-terms, transform
 * and adder per subgrid in one CTA) and takes no subgrid scratch.  A plan with
 * only some subgrids within the remainder bound (0 < n_sep_subgrids < n_subgrids)
 * grids those, and the pieces of the subgrids it splits (n_split_subgrids), in
 * one separable launch, and the rest with the direct kernels (at L = 32 a second
 * fused launch; at 24 and 16 gridder, transform and adder through the scratch).
 * Without the fused separable launch (other modes or kernel choices) the
 * subgrids are not split: the separable ones go first, the others direct.
 */
idg_status idg_grid(const idg_plan *plan, const void *d_vis, const uint8_t *d_flags,
                    const void *d_aterms, const float *d_taper, void *d_grid, idg_stream stream);

/*
 * Degridding, Algorithm 2 (splitter, subgrid IFFT, taper and A-terms, degridder).
 * d_grid     device complex64 [n_w][N][N][4]
 * d_vis_out  device complex64 [n_bl][n_t][n_chan][4], OVERWRITTEN: flagged and
 *            dropped visibilities are set to 0.
 * Other arguments as for idg_grid.
 * At L = 32, and at L = 24 and 16 when the plan is separable, with the default
 * kernel choice, IDG_FFT_FP32 and IDG_PHASOR_SINCOS, when at least half the
 * visibilities lie in subgrids of 64 or more (separable kernels; 512 for the
 * direct tensor-core degridder), the call
 * is one fused tensor-core launch (splitter, transform, A-terms and taper, and
 * the visibility sums per subgrid in one CTA) without subgrid scratch.  A plan
 * with only some subgrids within the remainder bound degrids those (with the
 * pieces of the subgrids it splits, when the separable part runs fused) and the
 * rest in separate launches, each by the same rules.
 */
idg_status idg_degrid(const idg_plan *plan, const void *d_grid, const uint8_t *d_flags,
                      const void *d_aterms, const float *d_taper, void *d_vis_out,
                      idg_stream stream);

/*
 * Classical gridding with oversampled A/W-projection kernels (Sect. 2: the
 * convolutional gridding the paper compares image domain gridding against),
 * on the plan's subgrids, visibilities and grid layout, so the two can be set
 * side by side on the same data.  For every subgrid p (baseline (p, q), A-term
 * slot a) and W-projection plane j the call builds the kernel
 *   window  c[(i,j),(a,b)](y, x) = b[y][x] exp(2 pi i j w_plane_step n') conj(A_p[a][i]) A_q[b][j]
 *           on the support x support lattice l = (x - M/2) S / M (the gridding
 *           direction's A_p^H X A_q as a 4 x 4 operator on XX, XY, YX, YY),
 *   kernel  the window zero-padded to (M O)^2 and Fourier transformed:
 *           C(dv, du) = M^-2 sum c[y][x] exp(-2 pi i (du (x - M/2) + dv (y - M/2)) / M),
 *           tabulated at offsets d - M/2 + 1 - o / O (o = 0 .. O-1),
 * and grids each unflagged visibility: position pu = (u f/c) S + N/2 (pv
 * alike), support pixels floor(pu) - M/2 + 1 .. floor(pu) + M/2, table phase
 * o = floor(frac(pu) O + 1/2) (o = O moves the support one pixel on), plane
 * j = floor((w f/c - w0) / w_plane_step + 1/2) with w0 the subgrid's W-layer
 * offset; grid[layer][r][q] += C . y_k, support pixels outside the grid are
 * dropped.  Kernels are rebuilt for every subgrid, i.e. every A-term slot.
 * support         M, even, 2 .. 32 (with the subgrid size: (L + M + 3)^2 x 32
 *                 bytes of shared memory at most 200 KiB)
 * oversample      O, 1 .. 128; one kernel (O^2 M^2 x 16 complex64) <= 256 MiB
 * w_plane_step    >= 0 wavelengths; 0: no w-term in the kernels
 * d_aterms        complex64 [n_slots][n_stations][M][M][4], the Jones matrices on
 *                 the kernel lattice, or NULL (identity)
 * d_taper         float32 [M][M] window b, or NULL for the PSWF window of width
 *                 M: a_y a_x with a = idg_taper_window(M, M, IDG_TAPER_PSWF)
 * d_grid          ADDED into, as idg_grid.
 * Kernel tables take up to 2 GiB of stream-ordered scratch (chunks of subgrids);
 * with w_plane_step > 0 the call first reads each subgrid's plane range back to
 * the host (it synchronises `stream` once).
 */
idg_status idg_classical_grid(const idg_plan *plan, int support, int oversample, double w_plane_step,
                              const void *d_vis, const uint8_t *d_flags, const void *d_aterms, const float *d_taper,
                              void *d_grid, idg_stream stream);

/*
 * Residuals, cost and A-term gradient for calibration (Sect. 6: image domain
 * gridding computes the residuals and derivatives of a fit whose free
 * parameters are the A-terms, with a full image -- here its grid -- as model).
 * With y_k the model visibilities of d_grid under d_aterms (as idg_degrid):
 *   d_residual[k] = d_vis[k] - y_k for planned, unflagged k; 0 for flagged and
 *                   dropped k (OVERWRITTEN, layout of d_vis)
 *   *d_cost      += J = sum_k sum_pol |d_residual[k][pol]|^2 (one FP64 value in
 *                   device memory, ADDED; NULL: not computed)
 *   d_gradient   += dJ/dRe(A) + i dJ/dIm(A) for every A-term entry, complex64
 *                   [n_slots][n_stations][L][L][4] like d_aterms (ADDED: zero it
 *                   first, or sum several plans into one gradient).  For a
 *                   complex direction E, d/dh J(A + h E) = Re sum conj(G) E.
 *   Per subgrid of baseline (p, q) in slot a and pixel: G[a][p] += -2 R A_q B^H
 *   and G[a][q] += -2 R^H A_p B, with B = taper * (the model's subgrid image)
 *   and R = sum_k r_k exp(+2 pi i phi_k) (the gridder's direct sum of the
 *   residuals, without taper and A-terms).
 * d_aterms NULL differentiates at identity A-terms; d_taper NULL is the plan's
 * default taper.  Runs the plan's splitter, inverse transform, degridder and
 * gridder kernels (the stage forms, not the fused ones) plus a residual and a
 * gradient kernel, per chunk of subgrids with up to 512 MiB of stream-ordered
 * scratch.  Summation order is not fixed (atomic adds).
 */
idg_status idg_aterm_gradient(const idg_plan *plan, const void *d_grid, const void *d_vis, const uint8_t *d_flags,
                              const void *d_aterms, const float *d_taper, void *d_residual, void *d_gradient,
                              double *d_cost, idg_stream stream);

/*
 * The composite operations restricted to the plan's subgrids [first, first +
 * count) in plan order (0 <= first, first + count <= n_subgrids; count 0 does
 * nothing).  They run the kernels idg_grid / idg_degrid would choose for these
 * subgrids (fused where those are fused).  This is the unit of a partition of
 * the subgrids over several devices or processes (Sect. 3.2: subgrids are
 * independent, only their sum into the grid couples them): every part grids
 * its range into a grid of its own and the parts' grids are summed; for
 * degridding the ranges' visibilities are disjoint.
 * idg_grid_range   ADDS the range's subgrids into d_grid (as idg_grid).
 * idg_degrid_range writes the visibilities of the range's subgrids (flagged
 *                  ones as 0) and leaves every other element of d_vis_out as
 *                  it was (dropped visibilities included).
 * Arguments otherwise as for idg_grid / idg_degrid; IDG_ERR_INVALID_ARG for a
 * range outside the plan.
 */
idg_status idg_grid_range(const idg_plan *plan, int64_t first, int64_t count, const void *d_vis,
                          const uint8_t *d_flags, const void *d_aterms, const float *d_taper, void *d_grid,
                          idg_stream stream);
idg_status idg_degrid_range(const idg_plan *plan, int64_t first, int64_t count, const void *d_grid,
                            const uint8_t *d_flags, const void *d_aterms, const float *d_taper, void *d_vis_out,
                            idg_stream stream);

/*
 * The same two operations on HOST buffers (layouts as above): inputs are copied
 * to device memory taken from the library's stream-ordered pool, the operation
 * runs on `stream`, the result is copied back and the call returns when it is
 * in h_grid / h_vis_out.  The work is cut into spans of whole baselines (about
 * 256 MB of visibilities each, at least 4 when there are that many baselines);
 * a library-owned copy stream per device moves the visibilities of one span
 * while `stream` computes another (gridding: copy in ahead; degridding: copy
 * out behind), ordered by events.  Page-locked host memory gives the full copy
 * bandwidth and the overlap; pageable memory works with staged copies.
 * h_grid is OVERWRITTEN with the grid of these visibilities (the device grid
 * starts from zero); h_vis_out is overwritten as in idg_degrid.  h_taper NULL
 * selects the plan's default taper (as d_taper NULL in idg_grid).  Host buffers
 * must not be touched by the caller until the call returns.
 */
idg_status idg_grid_host(const idg_plan *plan, const void *h_vis, const uint8_t *h_flags,
                         const void *h_aterms, const float *h_taper, void *h_grid, idg_stream stream);
idg_status idg_degrid_host(const idg_plan *plan, const void *h_grid, const uint8_t *h_flags,
                           const void *h_aterms, const float *h_taper, void *h_vis_out,
                           idg_stream stream);

/*
 * Both directions on HOST buffers in one call: h_vis gridded into h_grid
 * (OVERWRITTEN, as idg_grid_host) and the model grid h_model [n_w][N][N][4]
 * degridded into h_vis_out (OVERWRITTEN, as idg_degrid_host), with the same
 * flags, A-terms and taper (h_taper NULL: the plan's default).  One copy stream
 * carries the visibility spans ahead of the gridding, the model grid while the
 * gridding still runs, the gridded grid back while the degridding runs, and the
 * model visibilities span by span behind the degridding, so that only the first
 * and last span's copies are exposed.  Device memory: two visibility-sized and
 * two grid-sized buffers from the stream-ordered pool.  Synchronises `stream`.
 */
idg_status idg_grid_degrid_host(const idg_plan *plan, const void *h_vis, const void *h_model, const uint8_t *h_flags,
                                const void *h_aterms, const float *h_taper, void *h_grid, void *h_vis_out,
                                idg_stream stream);

/*
 * Gridding that allocates no device memory (the paper has no counterpart: this
 * is a deployment variant of idg_grid).  Some callers cannot allocate device
 * memory when they grid -- a real-time pipeline that reserves its whole memory
 * budget up front, or a host framework whose own allocator already holds all
 * free device memory -- because a new allocation could fail mid-run or
 * implicitly synchronise the device.  This call runs the same kernels as
 * idg_grid but keeps the subgrid scratch in a fixed 64 MiB array compiled into
 * the library (held by every GPU that loads the library, until the process
 * exits).  It calls no allocator.
 *   - The plan must need at most 64 MiB of scratch: n_subgrids * L * L * 32
 *     bytes (2048 subgrids of L = 32, 3640 of L = 24, 8192 of L = 16).  A
 *     larger plan is rejected with IDG_ERR_INVALID_ARG and a message giving
 *     the need and the limit, before any work is enqueued.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it.  Under
 *     CUDA's lazy module loading that lookup also loads the array (64 MiB)
 *     onto the device, so the first call may fail for lack of memory or
 *     synchronise the device: make it before reserving the rest of the
 *     device's memory and before any stream capture on the device.  A call
 *     with a plan of no subgrids does only the lookup and serves as the
 *     warm-up.  The cached address stays valid while the device's context
 *     lives: calls after cudaDeviceReset are not supported.
 *   - The atomic and the sorted adder run here.  A plan created with
 *     IDG_ADDER_COMPENSATED needs a grid-sized compensation buffer and is
 *     refused with IDG_ERR_UNSUPPORTED before any work is enqueued.
 *   - All calls on one device share the array.  Calls whose work overlaps on
 *     the GPU (different streams without ordering between them) race on it:
 *     order them on one stream or with events.  The array keeps the last
 *     call's contents; every call overwrites the part it uses before reading
 *     it, so nothing needs clearing.
 * Arguments, layouts and the accumulation into d_grid are as for idg_grid.
 */
idg_status idg_grid_no_alloc(const idg_plan *plan, const void *d_vis, const uint8_t *d_flags,
                             const void *d_aterms, const float *d_taper, void *d_grid, idg_stream stream);

/*
 * Stage entry points over the plan's subgrids [first, first + count) in plan
 * order.  d_subgrids is a device complex64 [count][L][L][4] buffer owned by
 * the caller.  They expose the intermediate states of Algorithms 1 and 2.
 *
 * idg_grid_subgrids    direct sum + taper + A_p^H . A_q  (image domain)
 * idg_fft_subgrids     in-place centred transform, direction -1 (image -> uv,
 *                      Alg. 1) or +1 (uv -> image, Alg. 2), both scaled by L^-2
 * idg_add_subgrids     grid[layer][r0 + i][q0 + j] += subgrid[i][j] (atomic adds; the
 *                      sorted tile adder for IDG_ADDER_SORTED plans, so the same bits
 *                      on every call; compensated plans add with plain atomics here)
 * idg_split_subgrids   subgrid[i][j] = grid[layer][r0 + i][q0 + j]
 * idg_degrid_subgrids  taper + A_p . A_q^H, then the degridding sum, from image
 *                      domain subgrids; writes only the visibilities of these
 *                      subgrids (flagged ones as 0).
 */
idg_status idg_grid_subgrids(const idg_plan *plan, int64_t first, int64_t count, const void *d_vis,
                             const uint8_t *d_flags, const void *d_aterms, const float *d_taper,
                             void *d_subgrids, idg_stream stream);
idg_status idg_fft_subgrids(const idg_plan *plan, int64_t count, int direction, void *d_subgrids,
                            idg_stream stream);
idg_status idg_add_subgrids(const idg_plan *plan, int64_t first, int64_t count, const void *d_subgrids,
                            void *d_grid, idg_stream stream);
idg_status idg_split_subgrids(const idg_plan *plan, int64_t first, int64_t count, const void *d_grid,
                              void *d_subgrids, idg_stream stream);
idg_status idg_degrid_subgrids(const idg_plan *plan, int64_t first, int64_t count, const void *d_subgrids,
                               const uint8_t *d_flags, const void *d_aterms, const float *d_taper,
                               void *d_vis_out, idg_stream stream);

/*
 * Batched form: many independent jobs processed together.  A batch binds each
 * job's plan to its device buffers at creation.  The work items (job, subgrid)
 * of all jobs with the same subgrid size L form work classes: the subgrids
 * within the separable remainder bound with the pieces of those the plans
 * split (L = 32, 24, 16), and the other subgrids.  Each work item is the whole
 * per-subgrid pipeline in one CTA, the subgrid staying in shared memory:
 *   idg_batch_grid    direct sum, taper and A_p^H . A_q, FFT, add into grid
 *                     (accumulated, as idg_grid)
 *   idg_batch_degrid  split from grid, IFFT, taper and A_p . A_q^H, degrid sum
 *                     into vis_out (overwritten; flagged and dropped -> 0)
 * A class runs either the fused tensor-core kernels (the separable ones, and at
 * L = 32 the direct ones with the default batch variant "tcgen05_fused",
 * IDG_KERNEL_BATCH_*): one launch per job with one CTA per item, most
 * visibilities first, each launch allowed to begin while the previous one
 * ends (programmatic dependent launch: the jobs' outputs are disjoint, or
 * summed by atomic adds; the kernels still complete in stream order); or ONE
 * persistent launch over the class's items
 * ordered by cost (K_p, largest first), a few CTAs per SM pulling items from a
 * device counter: the packed-FP32 kernels, for the direct subgrids at L = 24,
 * 16 and 8 and for any class whose visibilities lie mostly in subgrids of
 * fewer than 64 (separable classes) or 512 (direct).  No device scratch is used.  With
 * IDG_BATCH_GRAPH the first call of each direction captures its launch
 * sequence into a CUDA graph, and later calls replay it (the buffers are fixed
 * by the batch, so the graph stays valid).
 * Supported: subgrid sizes 8, 16, 24, 32 and the direct phasor form.  The
 * plans and buffers must outlive the batch; calls on one batch must not
 * overlap (they share the work counters).
 * idg_job_buffers per job (device pointers, layouts as above):
 *   vis      gridding input (may be NULL for a degrid-only batch)
 *   vis_out  degridding output (may be NULL for a grid-only batch)
 *   flags    or NULL;  aterms  or NULL (identity);  taper  or NULL (the plan's
 *            default taper, as in idg_grid)
 *   grid     gridding output (accumulated) / degridding input
 * idg_batch_info returns the planned visibilities, the work items and the
 * number of work classes (n_launches).
 */
typedef struct idg_batch idg_batch;
typedef struct {
    const void *vis;
    void *vis_out;
    const uint8_t *flags;
    const void *aterms;
    const float *taper;
    void *grid;
} idg_job_buffers;
enum { IDG_BATCH_GRAPH = 1 };
idg_status idg_batch_create(const idg_plan *const *plans, const idg_job_buffers *buffers, int n_jobs, int flags,
                            idg_batch **out);
idg_status idg_batch_grid(idg_batch *batch, idg_stream stream);
idg_status idg_batch_degrid(idg_batch *batch, idg_stream stream);
idg_status idg_batch_info(const idg_batch *batch, int64_t *n_vis, int64_t *n_items, int *n_launches);
/* The batch's own autotuner: for every class that runs a persistent kernel (not
 * the tensor-core classes) and each direction, times one launch of every compiled
 * shape (pixels per thread, visibilities per thread, block size, CTAs per SM) on
 * `stream` and keeps the fastest for this batch; recorded graphs are dropped and
 * recorded again on the next call.  The trial launches ADD into the jobs' grids
 * and overwrite their vis_out: zero the grids after tuning.  ms[i] receives the
 * trial times in order (classes, grid then degrid, shapes) for i < cap (ms may be
 * NULL).  Synchronises `stream`. */
idg_status idg_batch_autotune(idg_batch *batch, double *ms, int cap, idg_stream stream);
void idg_batch_destroy(idg_batch *batch);

/*
 * Kernel timing.  While enabled, every kernel launch of the library is
 * bracketed by two CUDA events recorded on the launch stream.  idg_profile_read
 * waits for the recorded events, adds their elapsed times into per-kernel
 * totals and returns the totals since the last reset:
 *   launches[k]  number of launches of kernel k
 *   ms[k]        summed device time (event to event) in milliseconds
 *   work[k]      algorithmic work of those launches: visibility-pixel products
 *                (sum of K_p * L^2) for the gridder, the degridder and the two
 *                fused batch kernels (IDG_KERNEL_BATCH_*), bytes moved
 *                for the adder (read subgrid + read and write grid, 96 B per
 *                pixel), the splitter (64 B per pixel), the calibration's
 *                residual kernel (96 B per planned visibility: model and
 *                observed read, residual written, flags aside) and gradient
 *                kernel (256 B per subgrid pixel: R, P, A_p, A_q read, two
 *                gradient entries read and written), subgrids for the FFT,
 *                bytes of kernel tables written for the classical kernel
 *                builder, visibility-support-pixel products (visibilities x M^2)
 *                for the classical gridder.
 * Arrays have IDG_KERNEL_COUNT entries; any of them may be NULL.  Do not enable
 * timing while a stream is being captured into a CUDA graph.
 */
enum { IDG_KERNEL_GRIDDER = 0, IDG_KERNEL_FFT, IDG_KERNEL_ADDER, IDG_KERNEL_SPLITTER, IDG_KERNEL_DEGRIDDER,
       IDG_KERNEL_BATCH_GRID, IDG_KERNEL_BATCH_DEGRID, IDG_KERNEL_CALIB_RESIDUAL, IDG_KERNEL_CALIB_GRADIENT,
       IDG_KERNEL_CLASSICAL_KERNELS, IDG_KERNEL_CLASSICAL_GRID, IDG_KERNEL_COUNT };
void idg_profile_enable(int on);
idg_status idg_profile_read(int64_t *launches, double *ms, double *work, int reset);

/*
 * Kernel variants and the autotuner.  The gridder and the degridder come in
 * several compiled tile shapes per subgrid size L (pixels per thread,
 * visibilities per shared-memory batch, block size, pixel-group split), and so
 * do the fused batch kernels (IDG_KERNEL_BATCH_GRID / _DEGRID, chosen when a
 * batch is created); the other kernels have one.  The process-wide choice per (kernel, L) starts at
 * variant 0 and applies to every later call with that L.
 *   idg_kernel_variant_count   number of variants (0: no such kernel or L)
 *   idg_kernel_variant_name    a static string naming the variant, or NULL
 *   idg_set/get_kernel_variant set or read the choice (IDG_ERR_INVALID_ARG if
 *                              out of range)
 *   idg_autotune               times every variant of the gridder and (when
 *                              d_vis_scratch is given) the degridder on a
 *                              strided sample of at most max_subgrids (<= 0:
 *                              4096) of the plan's subgrids, on `stream`, and
 *                              selects the fastest for this plan (its own
 *                              kernel choice; other plans keep theirs).  Mean
 *                              milliseconds per launch of variant v go to
 *                              gridder_ms[v] / degridder_ms[v] for v < cap
 *                              (arrays may be NULL).  d_vis_scratch is a
 *                              visibility-sized device buffer that the trial
 *                              degrids overwrite.  Takes sample scratch from
 *                              the stream-ordered pool; returns after the
 *                              stream has finished the trials.
 */
int idg_kernel_variant_count(int kernel, int subgrid_size);
const char *idg_kernel_variant_name(int kernel, int subgrid_size, int variant);
idg_status idg_set_kernel_variant(int kernel, int subgrid_size, int variant);
int idg_get_kernel_variant(int kernel, int subgrid_size);
/* The kernel choice of one plan (IDG_KERNEL_GRIDDER or IDG_KERNEL_DEGRIDDER):
 * variant -1 (the default of a new plan) follows the process-wide choice for the
 * plan's L; 0 .. count-1 fixes the plan's own.  Calls made with the plan read
 * it once when they start.  idg_autotune stores its pick in the plan, not
 * process-wide.  idg_plan_get_kernel_variant returns the variant the plan's
 * calls use (-1 for a NULL plan or an unknown kernel). */
idg_status idg_plan_set_kernel_variant(idg_plan *plan, int kernel, int variant);
int idg_plan_get_kernel_variant(const idg_plan *plan, int kernel);
idg_status idg_autotune(const idg_plan *plan, const void *d_vis, const uint8_t *d_flags, const void *d_aterms,
                        const float *d_taper, void *d_vis_scratch, int64_t max_subgrids, double *gridder_ms,
                        double *degridder_ms, int cap, idg_stream stream);

/*
 * Device error words.  The tensor-core kernels (the L = 32 gridder and
 * degridder, the separable ones at L = 32, 24 and 16, variants named "tcgen05_...",
 * and the IDG_FFT_TC_SPLIT transform)
 * wait on shared-memory barriers for their matrix operations and bulk copies;
 * every wait has an iteration limit, after which the kernel records an error
 * in a device word, waits (bounded) for its own operations in flight, releases
 * its tensor memory and leaves its outputs unwritten.  idg_device_errors
 * synchronises `stream`, reads and clears the words, and returns
 * IDG_ERR_TIMEOUT if any wait gave up since the last call, else
 * IDG_ERR_DEVICE_CHECK if a device-side check failed (the classical gridder
 * skipped a visibility whose support left its subgrid's tile, which a valid
 * plan rules out), IDG_OK otherwise.  The words are per device and per process.
 */
idg_status idg_device_errors(idg_stream stream);

/*
 * Self-test of that failure path (no counterpart in the paper): enqueues on
 * `stream` one CTA that allocates tensor memory as the tensor-core kernels do,
 * waits on a shared-memory barrier that nothing arrives on, with a limit of
 * max_polls polls (1 .. 2^20, a few milliseconds at most), records the timeout
 * in its device error word and releases the tensor memory.  The next
 * idg_device_errors then returns IDG_ERR_TIMEOUT (and clears the word); the
 * device stays usable.  No matrix operation or copy is involved.
 * IDG_ERR_INVALID_ARG for max_polls out of range.
 */
idg_status idg_selftest_wait_timeout(int64_t max_polls, idg_stream stream);

/*
 * Anti-aliasing windows (Sect. 4.1-4.3 and the appendix; host, FP64, no GPU).
 *
 * The taper passed to the gridding calls is c[y][x] = a_y a_x with a 1D window a
 * of L samples; sample x sits at offset x - L/2 from the subgrid centre and the
 * main lobe (the image) spans samples [0, L).
 *
 * idg_taper_window(L, beta, kind, a_out, eps_out) writes the window
 * a_out[L] (host, may be NULL), normalised so that a_out[L/2] = 1, and its
 * aliasing level *eps_out (may be NULL; not both):
 *   IDG_TAPER_PSWF: a_x = psi_0(c = pi beta / 2, eta = 2 (x - L/2) / L), the zeroth
 *     prolate spheroidal wave function (Sect. 4.1); *eps_out = sqrt(1 - lambda_0),
 *     its side-lobe level as a classical-gridding window of support beta
 *     (Table 1, "Classical PSWF").  In FP64, 1 - lambda_0 loses digits for
 *     beta > 9 (eps < 1e-6).
 *   IDG_TAPER_IDG_OPTIMAL: the window that minimises the mean side-lobe energy
 *     of the effective window of image domain gridding over the allowed sample
 *     positions |s| <= (L - beta + 1) / 2 (Sect. 4.3, Eq. a_opt): the eigenvector
 *     of the smallest eigenvalue of Rbar = Qbar (Hadamard) Sbar (appendix);
 *     *eps_out = the square root of that eigenvalue.  Where that eigenvalue is
 *     below 1e-14 of the largest (eps below about 1e-7, beta >~ 12) the window
 *     is not determined in FP64: IDG_ERR_UNSUPPORTED.
 * idg_taper_aliasing(L, beta, a, eps_out) writes the side-lobe level of any
 * window a[L] in image domain gridding: sqrt(a^T Rbar a / a^T a).
 * Both fail with IDG_ERR_INVALID_ARG for odd L, L outside 2 .. 512, beta outside
 * (0, L + 1), an unknown kind, or missing pointers.
 */
enum { IDG_TAPER_PSWF = 0, IDG_TAPER_IDG_OPTIMAL = 1 };
idg_status idg_taper_window(int subgrid_size, double beta, int kind, double *a_out, double *eps_out);
idg_status idg_taper_aliasing(int subgrid_size, double beta, const double *a, double *eps_out);

/*
 * Image-side steps (Alg. 1 last line, Alg. 2 first lines; Sect. 3.5, 4.2), device
 * buffers, stream-ordered on `stream`:
 *
 * idg_image_from_grid(plan, d_grid, h_window, d_image, stream):
 *   d_image[y][x][pol] (complex64, N x N x 4, overwritten) =
 *     sum_k exp(+2 pi i w0_k n'(x, y)) sum_{q,r} d_grid[k][r][q][pol]
 *       exp(+2 pi i ((q - N/2)(x - N/2) + (r - N/2)(y - N/2)) / N) / (cbar(x) cbar(y)),
 *   over the plan's w-layers k (w0_k = (k + w_layer_min) w_step, 0 without layers),
 *   with l = (x - N/2) S / N, m = (y - N/2) S / N, n' = sqrt(1 - l^2 - m^2) - 1.
 *   cbar is the effective window at zero shift of the 1D window h_window[L] (host,
 *   the window of the taper c[y][x] = a_y a_x):
 *     cbar(x) = L^-1 sum_j a_j sum_{m=-L/2}^{L/2-1} exp(2 pi i m ((x - N/2)/N - (j - L/2)/L)),
 *   which makes a sample at a subgrid centre image to its exact fringe.  h_window
 *   NULL: no division.
 * idg_grid_from_image(plan, d_image, h_window, d_grid, stream): its adjoint,
 *   d_grid[k] (overwritten) = the centred forward transform (sign -) of
 *   d_image exp(-2 pi i w0_k n') / (conj cbar(x) conj cbar(y)).
 * Both take two scratch images (32 N^2 bytes each) from the stream-ordered pool, need N
 * a power of two in 32 .. 4096 (IDG_ERR_UNSUPPORTED otherwise) and fail with
 * IDG_ERR_INVALID_ARG for missing buffers, a window that is not finite or whose
 * cbar vanishes on the image, or a plan of another device.
 */
idg_status idg_image_from_grid(const idg_plan *plan, const void *d_grid, const double *h_window, void *d_image,
                               idg_stream stream);
idg_status idg_grid_from_image(const idg_plan *plan, const void *d_image, const double *h_window, void *d_grid,
                               idg_stream stream);

/* Text of a status code, and the last error message of the calling thread. */
const char *idg_status_string(idg_status status);
const char *idg_last_error(void);

/* Subgrid sizes L compiled into this library: writes up to cap values, returns
   how many there are. */
int idg_supported_subgrid_sizes(int32_t *sizes, int cap);

#ifdef __cplusplus
}
#endif

#endif /* IDG_GB300_IDG_H */
