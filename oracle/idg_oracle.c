/*
 * FP64 CPU oracle for Image Domain Gridding (van der Tol, Veenboer & Offringa,
 * "Image Domain Gridding: a fast method for convolutional resampling of
 * visibilities", A&A 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, step-by-step
 * statement of what the GPU library computes.  It shares no code, header,
 * table or helper with the library; only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  The library never calls it.
 *
 * Every step follows the paper in its own order:
 *   plan            Sect. 3.2 "Partitioning" + Fig. 2: blocks of one baseline,
 *                   a range of timesteps and a group of channels whose support
 *                   fits an L x L subgrid (allowed shift (L - beta + 1)/2,
 *                   Sect. 4.3);
 *   subgrid image   Eq. (ShiftedDirectImaging) / Algorithm 1 inner loops: direct
 *                   sum of y_pk exp(+2 pi i (du l + dv m + dw n')) per pixel,
 *                   then the image-domain kernel (taper and A-terms, Sect. 3.4
 *                   "Variations");
 *   subgrid FFT     Algorithm 1 "Transform subgrid to uv domain";
 *   adder           Algorithm 1 "Add subgrid to master grid";
 *   splitter        Algorithm 2 "initialize subgrid from master grid";
 *   subgrid IFFT    Algorithm 2 "Transform subgrid to image domain";
 *   degridder       Algorithm 2 inner loops: y_pk = sum over pixels of
 *                   exp(-2 pi i (du l + dv m + dw n')) c[i,j] I_p[i,j].
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - pixel positions l = (x - L/2) S / L, m = (y - L/2) S / L, the definition of
 *     Sect. 2 (l_i = -S/2 + i S/L), not the garbled forms inside Alg. 1/2;
 *   - n' = sqrt(1 - l^2 - m^2) - 1 (the algorithms' n', not Eq. ShiftedDirectImaging's n);
 *   - "FFT" = centred 2D DFT with exp(-2 pi i ...) towards uv, scaled by 1/L^2;
 *     "IFFT" = its exact adjoint (exp(+...), also 1/L^2);
 *   - polarised form (Sect. 3.4): gridding applies taper * A_p^H P A_q per pixel,
 *     degridding taper * A_p P A_q^H, P = [[XX, XY], [YX, YY]];
 *   - the subgrid centre pixel Cu = floor(mid + 1/2), corner q0 = Cu - L/2, with
 *     u0 = (Cu - N/2)/S; grid index grid[layer][v][u][pol];
 *   - w0 = 0 without W-layers; with a w-step, layer k = floor(mid_w / w_step + 1/2),
 *     w0 = k * w_step;
 *   - channel frequency centres are given; c = 299792458 m/s.
 *
 * Compile with -ffp-contract=off: the plan's integers must be reproducible
 * bit for bit, so no multiply-add may be fused.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_C_LIGHT 299792458.0
#define ORACLE_TWO_PI 6.283185307179586476925286766559

typedef double complex cplx;

/* Descriptor layout: 10 int32 per subgrid. */
enum { D_BL = 0, D_SLOT, D_T0, D_NT, D_C0, D_NC, D_Q0, D_R0, D_LAYER, D_KP, D_FIELDS };

typedef struct {
    double umin, umax, vmin, vmax, wmin, wmax;
} extent;

typedef struct {
    const double *uvw, *freqs;
    int n_t, n_chan;
    int L, N;
    double S, smax, w_step;
} plan_ctx;

/* pixel coordinates of visibility (b, t, c) on the master grid, Sect. 2 Eq. (2):
   u_k = u / lambda_q; the grid pixel q has u = (q - N/2)/S */
static void vis_pixel(const plan_ctx *P, int b, int t, int c, double *pu, double *pv, double *wl)
{
    const double *uvw = P->uvw + ((size_t)b * P->n_t + t) * 3;
    double sc = P->freqs[c] / ORACLE_C_LIGHT;
    *pu = (uvw[0] * sc) * P->S + 0.5 * P->N;
    *pv = (uvw[1] * sc) * P->S + 0.5 * P->N;
    *wl = uvw[2] * sc;
}

static extent extent_of(const plan_ctx *P, int b, int t, int c0, int nc)
{
    extent e = { INFINITY, -INFINITY, INFINITY, -INFINITY, INFINITY, -INFINITY };
    for (int c = c0; c < c0 + nc; ++c) {
        double pu, pv, wl;
        vis_pixel(P, b, t, c, &pu, &pv, &wl);
        if (pu < e.umin) e.umin = pu;
        if (pu > e.umax) e.umax = pu;
        if (pv < e.vmin) e.vmin = pv;
        if (pv > e.vmax) e.vmax = pv;
        if (wl < e.wmin) e.wmin = wl;
        if (wl > e.wmax) e.wmax = wl;
    }
    return e;
}

static extent extent_union(extent a, extent b)
{
    extent e;
    e.umin = a.umin < b.umin ? a.umin : b.umin;
    e.umax = a.umax > b.umax ? a.umax : b.umax;
    e.vmin = a.vmin < b.vmin ? a.vmin : b.vmin;
    e.vmax = a.vmax > b.vmax ? a.vmax : b.vmax;
    e.wmin = a.wmin < b.wmin ? a.wmin : b.wmin;
    e.wmax = a.wmax > b.wmax ? a.wmax : b.wmax;
    return e;
}

static double centre_pixel(double lo, double hi) { return floor((lo + hi) * 0.5 + 0.5); }

/* The support of every sample must stay within the allowed shift from the
   subgrid centre (Sect. 4.3: (L - beta + 1)/2); with W-layers, the w spread of
   a block must not exceed one w-step. */
static int fits_size(const plan_ctx *P, extent e)
{
    double cu = centre_pixel(e.umin, e.umax);
    double cv = centre_pixel(e.vmin, e.vmax);
    double s = cu - e.umin;
    if (e.umax - cu > s) s = e.umax - cu;
    if (cv - e.vmin > s) s = cv - e.vmin;
    if (e.vmax - cv > s) s = e.vmax - cv;
    if (!(s <= P->smax)) return 0;
    if (P->w_step > 0.0 && !(e.wmax - e.wmin <= P->w_step)) return 0;
    return 1;
}

/* ... and the subgrid box must lie inside the master grid. */
static int fits(const plan_ctx *P, extent e)
{
    if (!fits_size(P, e)) return 0;
    double cu = centre_pixel(e.umin, e.umax);
    double cv = centre_pixel(e.vmin, e.vmax);
    double h = 0.5 * P->L;
    if (!(cu - h >= 0.0 && cu + h <= (double)P->N)) return 0;
    if (!(cv - h >= 0.0 && cv + h <= (double)P->N)) return 0;
    return 1;
}

static int group_first_channel(int n_chan, int G, int g)
{
    int base = n_chan / G, extra = n_chan % G;
    return g * base + (g < extra ? g : extra);
}

static int group_size(int n_chan, int G, int g)
{
    return n_chan / G + (g < n_chan % G ? 1 : 0);
}

/*
 * Partition the visibilities into subgrids (Sect. 3.2).
 * Order: baseline, A-term slot, channel group, first timestep.
 * Returns the number of subgrids; writes at most `cap` descriptors.
 */
long oracle_plan(const double *uvw, const double *freqs, const int32_t *aterm_offsets,
                 int n_bl, int n_t, int n_chan, int n_slots,
                 int L, int N, double cell, double w_step, double beta, int t_max,
                 int32_t *desc, long cap, long *n_dropped, int *n_w, int *k_min)
{
    plan_ctx P;
    P.uvw = uvw; P.freqs = freqs; P.n_t = n_t; P.n_chan = n_chan;
    P.L = L; P.N = N; P.S = (double)N * cell; P.smax = ((double)L - beta + 1.0) * 0.5;
    P.w_step = w_step;

    long count = 0, dropped = 0;
    long kmin = 0, kmax = 0;
    int have_k = 0;
    int32_t *kbuf = NULL;   /* layer k of each stored descriptor, made relative at the end */
    if (cap > 0) kbuf = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);

    for (int b = 0; b < n_bl; ++b) {
        for (int a = 0; a < n_slots; ++a) {
            int ts = aterm_offsets[a], te = aterm_offsets[a + 1];
            /* smallest number of channel groups for which every single timestep
               of every group fits the subgrid by size */
            int G = 1;
            for (; G < n_chan; ++G) {
                int ok = 1;
                for (int t = ts; t < te && ok; ++t)
                    for (int g = 0; g < G && ok; ++g)
                        ok = fits_size(&P, extent_of(&P, b, t, group_first_channel(n_chan, G, g),
                                                     group_size(n_chan, G, g)));
                if (ok) break;
            }
            for (int g = 0; g < G; ++g) {
                int c0 = group_first_channel(n_chan, G, g), nc = group_size(n_chan, G, g);
                int t = ts;
                while (t < te) {
                    extent e = extent_of(&P, b, t, c0, nc);
                    if (!fits(&P, e)) {            /* a lone timestep off the grid: dropped */
                        dropped += nc;
                        ++t;
                        continue;
                    }
                    int t0 = t++;
                    while (t < te && (t - t0 + 1) <= t_max) {
                        extent e2 = extent_union(e, extent_of(&P, b, t, c0, nc));
                        if (!fits(&P, e2)) break;
                        e = e2;
                        ++t;
                    }
                    double cu = centre_pixel(e.umin, e.umax);
                    double cv = centre_pixel(e.vmin, e.vmax);
                    long k = 0;
                    if (w_step > 0.0) k = (long)floor((e.wmin + e.wmax) * 0.5 / w_step + 0.5);
                    if (!have_k || k < kmin) kmin = k;
                    if (!have_k || k > kmax) kmax = k;
                    have_k = 1;
                    if (count < cap) {
                        int32_t *d = desc + count * D_FIELDS;
                        d[D_BL] = b; d[D_SLOT] = a; d[D_T0] = t0; d[D_NT] = t - t0;
                        d[D_C0] = c0; d[D_NC] = nc;
                        d[D_Q0] = (int32_t)cu - L / 2; d[D_R0] = (int32_t)cv - L / 2;
                        d[D_LAYER] = 0; d[D_KP] = (t - t0) * nc;
                        kbuf[count] = (int32_t)k;
                    }
                    ++count;
                }
            }
        }
    }
    long stored = count < cap ? count : cap;
    for (long i = 0; i < stored; ++i) desc[i * D_FIELDS + D_LAYER] = (int32_t)(kbuf[i] - kmin);
    free(kbuf);
    *n_dropped = dropped;
    *n_w = have_k ? (int)(kmax - kmin + 1) : 1;
    *k_min = (int)kmin;
    return count;
}

/* ------------------------------------------------------------------------ */
/* gridding and degridding                                                   */

typedef struct {
    const double *uvw, *freqs;
    const int32_t *baselines;
    const float *taper;            /* [L][L] */
    const float complex *aterms;   /* [n_slots][n_st][L][L][4] or NULL (identity) */
    int n_t, n_chan, n_st, L, N, k_min;
    double S, w_step;
} idg_ctx;

/* offsets of the subgrid centre from the uv origin (Sect. 3.3: u_0p, v_0p, w_0p) */
static void subgrid_offsets(const idg_ctx *C, const int32_t *d, double *u0, double *v0, double *w0)
{
    *u0 = ((double)d[D_Q0] + 0.5 * C->L - 0.5 * C->N) / C->S;
    *v0 = ((double)d[D_R0] + 0.5 * C->L - 0.5 * C->N) / C->S;
    *w0 = C->w_step > 0.0 ? (double)(d[D_LAYER] + C->k_min) * C->w_step : 0.0;
}

static void pixel_lmn(const idg_ctx *C, int y, int x, double *l, double *m, double *n1)
{
    *l = ((double)x - 0.5 * C->L) * C->S / C->L;
    *m = ((double)y - 0.5 * C->L) * C->S / C->L;
    *n1 = sqrt(1.0 - (*l) * (*l) - (*m) * (*m)) - 1.0;
}

static void load_jones(const idg_ctx *C, int slot, int station, int y, int x, cplx J[4])
{
    if (!C->aterms) {
        J[0] = 1.0; J[1] = 0.0; J[2] = 0.0; J[3] = 1.0;
        return;
    }
    const float complex *a = C->aterms + ((((size_t)slot * C->n_st + station) * C->L + y) * C->L + x) * 4;
    for (int i = 0; i < 4; ++i) J[i] = (cplx)a[i];
}

/* 2x2 products, matrices stored [[0,1],[2,3]] */
static void mat_mul(const cplx A[4], const cplx B[4], cplx R[4])
{
    R[0] = A[0] * B[0] + A[1] * B[2];
    R[1] = A[0] * B[1] + A[1] * B[3];
    R[2] = A[2] * B[0] + A[3] * B[2];
    R[3] = A[2] * B[1] + A[3] * B[3];
}

static void mat_herm(const cplx A[4], cplx R[4])
{
    R[0] = conj(A[0]); R[1] = conj(A[2]); R[2] = conj(A[1]); R[3] = conj(A[3]);
}

/*
 * Subgrid images of the selected subgrids (Algorithm 1 up to the FFT):
 *   I_p[y][x] = sum_k y_k exp(+2 pi i (du l + dv m + dw n')),  unflagged k only,
 *   then I_p <- taper[y][x] * A_p^H I_p A_q  (gridding uses the adjoint kernel).
 * out: [n_ids][L][L][4] complex double.
 */
void oracle_subgrid_images(const double *uvw, const double *freqs, const int32_t *baselines,
                           const float complex *vis, const uint8_t *flags,
                           const float complex *aterms, const float *taper,
                           int n_t, int n_chan, int n_st, int L, int N, double cell,
                           double w_step, int k_min,
                           const int32_t *desc, const int32_t *ids, long n_ids, double complex *out)
{
    idg_ctx C = { uvw, freqs, baselines, taper, aterms, n_t, n_chan, n_st, L, N, k_min,
                  (double)N * cell, w_step };
#pragma omp parallel for schedule(dynamic)
    for (long s = 0; s < n_ids; ++s) {
        const int32_t *d = desc + (size_t)ids[s] * D_FIELDS;
        cplx *img = out + (size_t)s * L * L * 4;
        memset(img, 0, sizeof(cplx) * (size_t)L * L * 4);
        double u0, v0, w0;
        subgrid_offsets(&C, d, &u0, &v0, &w0);
        int b = d[D_BL];
        for (int t = d[D_T0]; t < d[D_T0] + d[D_NT]; ++t) {
            for (int c = d[D_C0]; c < d[D_C0] + d[D_NC]; ++c) {
                size_t k = ((size_t)b * n_t + t) * n_chan + c;
                if (flags && flags[k]) continue;
                const double *uvw_k = uvw + ((size_t)b * n_t + t) * 3;
                double sc = freqs[c] / ORACLE_C_LIGHT;
                double du = uvw_k[0] * sc - u0;
                double dv = uvw_k[1] * sc - v0;
                double dw = uvw_k[2] * sc - w0;
                cplx V[4];
                for (int p = 0; p < 4; ++p) V[p] = (cplx)vis[k * 4 + p];
                for (int y = 0; y < L; ++y) {
                    for (int x = 0; x < L; ++x) {
                        double l, m, n1;
                        pixel_lmn(&C, y, x, &l, &m, &n1);
                        double phase = ORACLE_TWO_PI * (du * l + dv * m + dw * n1);
                        cplx ph = cos(phase) + I * sin(phase);
                        cplx *px = img + ((size_t)y * L + x) * 4;
                        for (int p = 0; p < 4; ++p) px[p] += V[p] * ph;
                    }
                }
            }
        }
        int st_p = baselines[2 * b], st_q = baselines[2 * b + 1];
        for (int y = 0; y < L; ++y) {
            for (int x = 0; x < L; ++x) {
                cplx Ap[4], Aq[4], ApH[4], T[4], R[4];
                cplx *px = img + ((size_t)y * L + x) * 4;
                load_jones(&C, d[D_SLOT], st_p, y, x, Ap);
                load_jones(&C, d[D_SLOT], st_q, y, x, Aq);
                mat_herm(Ap, ApH);
                mat_mul(ApH, px, T);
                mat_mul(T, Aq, R);
                double c = (double)taper[y * L + x];
                for (int p = 0; p < 4; ++p) px[p] = c * R[p];
            }
        }
    }
}

/*
 * Centred 2D DFT of n subgrids [n][L][L][4], in place:
 *   out[i][j] = L^-2 sum_{y,x} in[y][x] exp(sign 2 pi i ((j - L/2)(x - L/2) + (i - L/2)(y - L/2)) / L)
 * sign = -1 towards the uv domain (Algorithm 1), +1 towards the image (Algorithm 2).
 * Written as the textbook sum, one dimension after the other.
 */
void oracle_dft2(double complex *data, long n, int L, int sign)
{
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)L);
    for (int k = 0; k < L; ++k) {
        double a = ORACLE_TWO_PI * (double)k / (double)L;
        w[k] = cos(a) + I * (double)sign * sin(a);
    }
#pragma omp parallel
    {
        cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)L * L * 4);
#pragma omp for schedule(static)
        for (long s = 0; s < n; ++s) {
            cplx *g = data + (size_t)s * L * L * 4;
            /* along x: tmp[y][j] = sum_x g[y][x] w^((j-L/2)(x-L/2)) */
            for (int y = 0; y < L; ++y)
                for (int j = 0; j < L; ++j)
                    for (int p = 0; p < 4; ++p) {
                        cplx acc = 0.0;
                        for (int x = 0; x < L; ++x) {
                            long e = (long)(j - L / 2) * (long)(x - L / 2);
                            int idx = (int)(((e % L) + L) % L);
                            acc += g[((size_t)y * L + x) * 4 + p] * w[idx];
                        }
                        tmp[((size_t)y * L + j) * 4 + p] = acc;
                    }
            /* along y, with the 1/L^2 normalisation */
            for (int i = 0; i < L; ++i)
                for (int j = 0; j < L; ++j)
                    for (int p = 0; p < 4; ++p) {
                        cplx acc = 0.0;
                        for (int y = 0; y < L; ++y) {
                            long e = (long)(i - L / 2) * (long)(y - L / 2);
                            int idx = (int)(((e % L) + L) % L);
                            acc += tmp[((size_t)y * L + j) * 4 + p] * w[idx];
                        }
                        g[((size_t)i * L + j) * 4 + p] = acc / ((double)L * (double)L);
                    }
        }
        free(tmp);
    }
    free(w);
}

/* Algorithm 1 "Add subgrid to master grid": grid[layer][r0+i][q0+j] += V_p[i][j],
   in the order given (deterministic). grid: [n_w][N][N][4] complex double. */
void oracle_add(const int32_t *desc, const int32_t *ids, long n_ids, const double complex *sub,
                int L, int N, double complex *grid)
{
    for (long s = 0; s < n_ids; ++s) {
        const int32_t *d = desc + (size_t)ids[s] * D_FIELDS;
        const cplx *V = sub + (size_t)s * L * L * 4;
        cplx *G = grid + (size_t)d[D_LAYER] * N * N * 4;
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j)
                for (int p = 0; p < 4; ++p)
                    G[(((size_t)(d[D_R0] + i)) * N + (d[D_Q0] + j)) * 4 + p] += V[((size_t)i * L + j) * 4 + p];
    }
}

/* Algorithm 2 "initialize subgrid from master grid". */
void oracle_split(const int32_t *desc, const int32_t *ids, long n_ids, const double complex *grid,
                  int L, int N, double complex *sub)
{
    for (long s = 0; s < n_ids; ++s) {
        const int32_t *d = desc + (size_t)ids[s] * D_FIELDS;
        cplx *V = sub + (size_t)s * L * L * 4;
        const cplx *G = grid + (size_t)d[D_LAYER] * N * N * 4;
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j)
                for (int p = 0; p < 4; ++p)
                    V[((size_t)i * L + j) * 4 + p] = G[(((size_t)(d[D_R0] + i)) * N + (d[D_Q0] + j)) * 4 + p];
    }
}

/*
 * Degridding of the selected subgrids from their image-domain subgrids
 * (Algorithm 2 after the IFFT):
 *   I_p <- taper[y][x] * A_p I_p A_q^H,
 *   y_k = sum_{y,x} I_p[y][x] exp(-2 pi i (du l + dv m + dw n')),  flagged k -> 0.
 * img: [n_ids][L][L][4]; vis_out: [n_bl][n_t][n_chan][4] complex double, only the
 * visibilities of the selected subgrids are written.
 */
void oracle_degrid_images(const double *uvw, const double *freqs, const int32_t *baselines,
                          const uint8_t *flags, const float complex *aterms, const float *taper,
                          int n_t, int n_chan, int n_st, int L, int N, double cell,
                          double w_step, int k_min,
                          const int32_t *desc, const int32_t *ids, long n_ids,
                          const double complex *img, double complex *vis_out)
{
    idg_ctx C = { uvw, freqs, baselines, taper, aterms, n_t, n_chan, n_st, L, N, k_min,
                  (double)N * cell, w_step };
#pragma omp parallel
    {
        cplx *P = (cplx *)malloc(sizeof(cplx) * (size_t)L * L * 4);
#pragma omp for schedule(dynamic)
        for (long s = 0; s < n_ids; ++s) {
            const int32_t *d = desc + (size_t)ids[s] * D_FIELDS;
            const cplx *src = img + (size_t)s * L * L * 4;
            int b = d[D_BL];
            int st_p = baselines[2 * b], st_q = baselines[2 * b + 1];
            for (int y = 0; y < L; ++y) {
                for (int x = 0; x < L; ++x) {
                    cplx Ap[4], Aq[4], AqH[4], T[4], R[4];
                    const cplx *px = src + ((size_t)y * L + x) * 4;
                    load_jones(&C, d[D_SLOT], st_p, y, x, Ap);
                    load_jones(&C, d[D_SLOT], st_q, y, x, Aq);
                    mat_herm(Aq, AqH);
                    mat_mul(Ap, px, T);
                    mat_mul(T, AqH, R);
                    double c = (double)taper[y * L + x];
                    for (int p = 0; p < 4; ++p) P[((size_t)y * L + x) * 4 + p] = c * R[p];
                }
            }
            double u0, v0, w0;
            subgrid_offsets(&C, d, &u0, &v0, &w0);
            for (int t = d[D_T0]; t < d[D_T0] + d[D_NT]; ++t) {
                for (int c = d[D_C0]; c < d[D_C0] + d[D_NC]; ++c) {
                    size_t k = ((size_t)b * n_t + t) * n_chan + c;
                    cplx acc[4] = { 0.0, 0.0, 0.0, 0.0 };
                    if (!(flags && flags[k])) {
                        const double *uvw_k = uvw + ((size_t)b * n_t + t) * 3;
                        double sc = freqs[c] / ORACLE_C_LIGHT;
                        double du = uvw_k[0] * sc - u0;
                        double dv = uvw_k[1] * sc - v0;
                        double dw = uvw_k[2] * sc - w0;
                        for (int y = 0; y < L; ++y) {
                            for (int x = 0; x < L; ++x) {
                                double l, m, n1;
                                pixel_lmn(&C, y, x, &l, &m, &n1);
                                double phase = -ORACLE_TWO_PI * (du * l + dv * m + dw * n1);
                                cplx ph = cos(phase) + I * sin(phase);
                                const cplx *px = P + ((size_t)y * L + x) * 4;
                                for (int p = 0; p < 4; ++p) acc[p] += px[p] * ph;
                            }
                        }
                    }
                    for (int p = 0; p < 4; ++p) vis_out[k * 4 + p] = acc[p];
                }
            }
        }
        free(P);
    }
}
