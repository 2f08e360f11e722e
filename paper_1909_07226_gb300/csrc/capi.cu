// C ABI: plan object, argument validation, device metadata and the composite
// gridding / degridding calls built from the stage kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>

#include "idg_internal.h"

namespace idg {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

idg_status fail(idg_status st, const std::string &msg) {
    set_error(msg);
    return st;
}

idg_status cuda_fail(int err, const char *what) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%d)", what, cudaGetErrorString((cudaError_t)err), err);
    set_error(buf);
    return err == cudaErrorMemoryAllocation ? IDG_ERR_NO_MEMORY : IDG_ERR_CUDA;
}

idg_status launch_subgrid_fft(const idg_plan *p, int64_t count, int direction, void *subgrids, void *stream) {
    if (p->opts.fft_mode == IDG_FFT_TC_SPLIT) return launch_dft_tc(p->L, count, direction, subgrids, stream);
    return launch_fft(p->L, count, direction, subgrids, stream);
}

// One stream-ordered memory pool per device for the subgrid scratch, kept
// alive (release threshold = max) so repeated calls do not return memory to
// the driver between steps.
static cudaMemPool_t scratch_pool(int device) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= 64) return nullptr;
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        pools[device] = pool;
    }
    return pools[device];
}

idg_status scratch_alloc(int device, size_t bytes, void *stream, void **p) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemPool_t pool = scratch_pool(device);
    if (!pool) return fail(IDG_ERR_CUDA, "cannot create the scratch memory pool");
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync(scratch)");
    return IDG_OK;
}

static constexpr size_t kScratchBudget = size_t(512) << 20;

static int64_t chunk_subgrids(const idg_plan *p) {
    const size_t per = (size_t)p->L * p->L * 4 * 8;
    int64_t c = (int64_t)(kScratchBudget / per);
    return std::max<int64_t>(1, std::min<int64_t>(c, p->stats.n_subgrids));
}

static idg_status check_device(const idg_plan *p) {
    if (p->device < 0) return fail(IDG_ERR_INVALID_ARG, "the plan was created without a CUDA device");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device)
        return fail(IDG_ERR_INVALID_ARG, "plan was created on device " + std::to_string(p->device) +
                                             " but the current device is " + std::to_string(dev));
    return IDG_OK;
}

// ---------------------------------------------------------------------------
// kernel timing

namespace {
std::mutex g_prof_mu;
bool g_prof_on = false;
struct ProfRec {
    int kernel;
    cudaEvent_t a, b;
    double work;
};
std::vector<ProfRec> g_prof_pending;
int64_t g_prof_launches[IDG_KERNEL_COUNT] = {};
double g_prof_ms[IDG_KERNEL_COUNT] = {};
double g_prof_work[IDG_KERNEL_COUNT] = {};
}  // namespace

ProfileScope::ProfileScope(int k, void *s, double w) : kernel(k), stream(s), ev{nullptr, nullptr}, work(w), on(false) {
    {
        std::lock_guard<std::mutex> lock(g_prof_mu);
        on = g_prof_on;
    }
    if (!on) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        on = false;       // no timing events inside a graph capture
        return;
    }
    if (cudaEventCreate((cudaEvent_t *)&ev[0]) != cudaSuccess || cudaEventCreate((cudaEvent_t *)&ev[1]) != cudaSuccess) {
        cudaGetLastError();
        on = false;
        return;
    }
    cudaEventRecord((cudaEvent_t)ev[0], (cudaStream_t)stream);
}

ProfileScope::~ProfileScope() {
    if (!on) return;
    cudaEventRecord((cudaEvent_t)ev[1], (cudaStream_t)stream);
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_pending.push_back({kernel, (cudaEvent_t)ev[0], (cudaEvent_t)ev[1], work});
}

}  // namespace idg

using namespace idg;

static constexpr double kTwoPi = 6.283185307179586476925286766559;

// x = hi + lo with hi = x rounded to FP32 and lo the rounded remainder (|x - hi - lo|
// <= 2^-48 |x| about); the kernels form phase coefficients from such pairs with
// error-free FP32 products and sums.
static void split_pair(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// uvw [n][3] (metres) -> pairs [n][8] = (u hi, u lo, v hi, v lo, w hi, w lo, 0, 0)
__global__ void split_uvw_kernel(const double *__restrict__ uvw, float4 *__restrict__ out, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[3], l[3];
    for (int j = 0; j < 3; ++j) {
        const double x = uvw[3 * i + j];
        h[j] = __double2float_rn(x);
        l[j] = __double2float_rn(x - (double)h[j]);
    }
    out[2 * i] = make_float4(h[0], l[0], h[1], l[1]);
    out[2 * i + 1] = make_float4(h[2], l[2], 0.0f, 0.0f);
}

// The separable kernels (L = 32, 24) write the phasor of visibility k at pixel (x, y) as
// exp(i (a X + c s(x))) exp(i (b Y + c t(y))) exp(i c r(x, y)) and keep the last
// factor to first order, 1 + i c r; the dropped terms are at most theta^2 / 2 in
// relative terms, theta = max |c| max |r|.  Below this bound that is <= 2^-20
// (9.5e-7), the order of the rounding of the FP16 split sums themselves.
constexpr double kSepThetaMax = 1.38e-3;

// Pieces of subgrid s (outside the remainder bound with any single w_s): the
// smallest grid of kt x kc equal blocks of its timesteps and channels (kt kc pieces,
// most even cut first) whose blocks each meet the bound with w_s = the middle of the
// block's own w range.  A piece costs the separable kernels' fixed cost per subgrid
// (transform, A-terms, adder: about F_L visibilities' worth) and saves the direct
// kernels' extra cost per visibility, so a subgrid of K_p visibilities is split only
// into at most (rho_L - 1) K_p / F_L pieces, rho_L the measured ratio of the direct to
// the separable kernels' time per visibility (L = 32: 3.8, 24: 2.7; at L = 16 the direct
// kernels come within 20 % and pieces measured slower, so 1: none) and
// F_L = 200 (L / 32)^2 visibilities.
static void split_pieces(idg_plan *p, int64_t s, double r_max, const double *uvw, const double *freqs_hz,
                         double *c_max) {
    const int32_t *d = &p->desc[s * kDescFields];
    const int t0 = d[IDG_DESC_T0], nt = d[IDG_DESC_NT], c0 = d[IDG_DESC_C0], nc = d[IDG_DESC_NC];
    const int64_t kp = d[IDG_DESC_KP];
    const double rho = p->L == 32 ? 3.8 : p->L == 24 ? 2.7 : 1.0;
    const double F = 200.0 * (p->L / 32.0) * (p->L / 32.0);
    const int64_t max_pieces = std::min<int64_t>((int64_t)((rho - 1.0) * (double)kp / F), (int64_t)nt * nc);
    // w range (wavelengths) of the block [ta, tb) x [ca, cb): w_t f is linear in f, so the
    // channel ends bound it
    // (every block has at least one timestep and one channel: kt <= nt, kc <= nc)
    auto range = [&](int ta, int tb, int ca, int cb, double *lo, double *hi) {
        const double fa = freqs_hz[ca] / kSpeedOfLight, fb = freqs_hz[cb - 1] / kSpeedOfLight;
        *lo = INFINITY;
        *hi = -INFINITY;
        for (int t = ta; t < tb; ++t) {
            const double w = uvw[((size_t)d[IDG_DESC_BASELINE] * p->n_t + t) * 3 + 2];
            *lo = std::min(*lo, std::min(w * fa, w * fb));
            *hi = std::max(*hi, std::max(w * fa, w * fb));
        }
    };
    auto meets = [&](double lo, double hi) { return kTwoPi * 0.5 * (hi - lo) * r_max <= kSepThetaMax; };
    for (int64_t prod = 2; prod <= max_pieces; ++prod)
        for (int kt = 1; kt <= nt && kt <= prod; ++kt) {
            if (prod % kt) continue;
            const int64_t kc = prod / kt;
            if (kc > nc) continue;
            bool ok = true;
            for (int i = 0; i < kt && ok; ++i)
                for (int j = 0; j < kc && ok; ++j) {
                    double lo, hi;
                    range(t0 + (int)((int64_t)i * nt / kt), t0 + (int)((int64_t)(i + 1) * nt / kt),
                          c0 + (int)((int64_t)j * nc / kc), c0 + (int)((int64_t)(j + 1) * nc / kc), &lo, &hi);
                    ok = meets(lo, hi);
                }
            if (!ok) continue;
            for (int i = 0; i < kt; ++i)
                for (int j = 0; j < kc; ++j) {
                    idg_plan::Piece pc;
                    pc.parent = (int32_t)s;
                    pc.t0 = t0 + (int)((int64_t)i * nt / kt);
                    pc.nt = t0 + (int)((int64_t)(i + 1) * nt / kt) - pc.t0;
                    pc.c0 = c0 + (int)((int64_t)j * nc / kc);
                    pc.nc = c0 + (int)((int64_t)(j + 1) * nc / kc) - pc.c0;
                    double lo, hi;
                    range(pc.t0, pc.t0 + pc.nt, pc.c0, pc.c0 + pc.nc, &lo, &hi);
                    pc.ws = 0.5 * (lo + hi);
                    *c_max = std::max(*c_max, kTwoPi * 0.5 * (hi - lo));
                    p->pieces.push_back(pc);
                }
            p->split_sub[s] = 1;
            return;
        }
}

idg::Geometry idg_plan::geometry() const {
    Geometry g;
    g.L = L;
    g.N = N;
    g.n_t = n_t;
    g.n_chan = n_chan;
    g.n_stations = n_stations;
    g.S = S;
    g.k_uv = 6.283185307179586476925286766559 * S / (double)L;
    g.sub = d_sub;
    g.order = d_order;
    g.uvw = d_uvw;
    g.scale = d_scale;
    g.uvw_f2 = d_uvw_f2;
    g.scale_f2 = d_scale_f2;
    g.nprime = d_nprime;
    g.sep = d_nprime + (size_t)L * L;
    g.separable = stats.separable;
    g.c_scale = c_scale;
    g.r_scale = r_scale;
    g.ds = ds;
    g.recurrence = opts.precision_mode == IDG_PHASOR_RECURRENCE ? 1 : 0;
    g.anchor = 8;
    return g;
}

int idg_plan::kernel_variant(int kernel) const {
    if (kernel < 0 || kernel >= IDG_KERNEL_COUNT) return 0;
    const int v = variant[kernel].load(std::memory_order_relaxed);
    return v >= 0 ? v : idg::get_variant(kernel, L);
}

extern "C" {

void idg_plan_options_default(idg_plan_options *o) {
    if (!o) return;
    o->kernel_size = 7.0;
    o->max_timesteps_per_subgrid = 128;
    o->precision_mode = IDG_PHASOR_SINCOS;
    o->fft_mode = IDG_FFT_FP32;
    o->adder_mode = IDG_ADDER_ATOMIC;
    o->n_host_threads = 0;
}

const char *idg_status_string(idg_status s) {
    switch (s) {
    case IDG_OK: return "ok";
    case IDG_ERR_INVALID_ARG: return "invalid argument";
    case IDG_ERR_NO_MEMORY: return "out of memory";
    case IDG_ERR_CUDA: return "CUDA error";
    case IDG_ERR_TIMEOUT: return "device wait timed out";
    case IDG_ERR_DEVICE_CHECK: return "device consistency check failed";
    case IDG_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *idg_last_error(void) { return g_last_error.c_str(); }

idg_status idg_device_errors(idg_stream stream) {
    int code = 0;
    idg_status st = read_device_errors(&code, stream);
    if (st != IDG_OK) return st;
    if (code & 1) return fail(IDG_ERR_TIMEOUT, "a bounded wait of a tensor-core kernel gave up; its outputs are invalid");
    if (code & 2)
        return fail(IDG_ERR_DEVICE_CHECK, "a device-side consistency check failed (classical gridder: a support "
                                          "outside its subgrid's tile was skipped)");
    return IDG_OK;
}

void idg_profile_enable(int on) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_on = on != 0;
}

idg_status idg_profile_read(int64_t *launches, double *ms, double *work, int reset) {
    std::vector<ProfRec> pend;
    {
        std::lock_guard<std::mutex> lock(g_prof_mu);
        pend.swap(g_prof_pending);
    }
    idg_status st = IDG_OK;
    for (auto &r : pend) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && st == IDG_OK) st = cuda_fail(e, "reading kernel timing events");
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        std::lock_guard<std::mutex> lock(g_prof_mu);
        g_prof_launches[r.kernel] += 1;
        g_prof_ms[r.kernel] += t;
        g_prof_work[r.kernel] += r.work;
    }
    std::lock_guard<std::mutex> lock(g_prof_mu);
    for (int k = 0; k < IDG_KERNEL_COUNT; ++k) {
        if (launches) launches[k] = g_prof_launches[k];
        if (ms) ms[k] = g_prof_ms[k];
        if (work) work[k] = g_prof_work[k];
        if (reset) {
            g_prof_launches[k] = 0;
            g_prof_ms[k] = 0.0;
            g_prof_work[k] = 0.0;
        }
    }
    return st;
}

int idg_supported_subgrid_sizes(int32_t *sizes, int cap) {
    static const int32_t all[] = {8, 16, 24, 32, 48, 64};
    int n = 0;
    for (int32_t L : all)
        if (gridder_supported(L)) {
            if (sizes && n < cap) sizes[n] = L;
            ++n;
        }
    return n;
}

void idg_plan_destroy(idg_plan *p) {
    if (!p) return;
    if (p->device < 0) {
        delete p;
        return;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (p->device >= 0) cudaSetDevice(p->device);
    cudaFree(p->d_sub);
    cudaFree(p->d_order);
    cudaFree(p->d_span_order);
    cudaFree(p->d_fused_order);
    cudaFree(p->d_fused_span);
    cudaFree(p->d_tile_ids);
    cudaFree(p->d_tile_first);
    cudaFree(p->d_tile_sub);
    cudaFree(p->d_uvw);
    cudaFree(p->d_scale);
    cudaFree(p->d_uvw_f2);
    cudaFree(p->d_scale_f2);
    cudaFree(p->d_nprime);
    cudaFree(p->d_taper);
    cudaFree(p->d_ones);
    if (prev >= 0) cudaSetDevice(prev);
    delete p;
}

idg_status idg_plan_create(const double *uvw_m, const double *freqs_hz, const int32_t *baselines,
                           const int32_t *aterm_offsets, int n_bl, int n_t, int n_chan, int n_stations,
                           int n_slots, int L, int N, double cell, double w_step,
                           const idg_plan_options *opts, idg_plan **out) {
    if (!out) return fail(IDG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    idg_plan_options o;
    idg_plan_options_default(&o);
    if (opts) o = *opts;
    if (!uvw_m || !freqs_hz || !baselines || !aterm_offsets)
        return fail(IDG_ERR_INVALID_ARG, "uvw, freqs, baselines and aterm_offsets are required");
    if (n_bl < 1 || n_t < 1 || n_chan < 1 || n_stations < 1 || n_slots < 1)
        return fail(IDG_ERR_INVALID_ARG, "n_bl, n_t, n_chan, n_stations and n_slots must be >= 1");
    if (!(o.kernel_size >= 1.0) || !std::isfinite(o.kernel_size))
        return fail(IDG_ERR_INVALID_ARG, "kernel_size must be a finite number >= 1");
    if (L < 2 || L % 2 != 0) return fail(IDG_ERR_INVALID_ARG, "subgrid_size must be even and >= 2");
    if ((double)L < o.kernel_size + 1.0)
        return fail(IDG_ERR_INVALID_ARG, "subgrid_size must be >= kernel_size + 1");
    if (N < L || N % 2 != 0) return fail(IDG_ERR_INVALID_ARG, "grid_size must be even and >= subgrid_size");
    if (!(cell > 0.0) || !std::isfinite(cell)) return fail(IDG_ERR_INVALID_ARG, "cell_size must be > 0");
    if (!((double)N * cell < 2.0))
        return fail(IDG_ERR_INVALID_ARG, "image size N * cell must be < 2 (direction cosines)");
    if (!(w_step >= 0.0) || !std::isfinite(w_step)) return fail(IDG_ERR_INVALID_ARG, "w_step must be >= 0");
    if (o.max_timesteps_per_subgrid < 1) return fail(IDG_ERR_INVALID_ARG, "max_timesteps_per_subgrid must be >= 1");
    if (o.precision_mode != IDG_PHASOR_SINCOS && o.precision_mode != IDG_PHASOR_RECURRENCE)
        return fail(IDG_ERR_INVALID_ARG, "unknown precision_mode");
    if (o.fft_mode != IDG_FFT_FP32 && o.fft_mode != IDG_FFT_TC_SPLIT)
        return fail(IDG_ERR_INVALID_ARG, "unknown fft_mode");
    if (o.fft_mode == IDG_FFT_TC_SPLIT && !dft_tc_supported(L))
        return fail(IDG_ERR_UNSUPPORTED, "the tensor-core subgrid transform is built for subgrid size 32");
    if (o.adder_mode != IDG_ADDER_ATOMIC && o.adder_mode != IDG_ADDER_COMPENSATED && o.adder_mode != IDG_ADDER_SORTED)
        return fail(IDG_ERR_INVALID_ARG, "unknown adder_mode");
    if (aterm_offsets[0] != 0 || aterm_offsets[n_slots] != n_t)
        return fail(IDG_ERR_INVALID_ARG, "aterm_offsets must start at 0 and end at n_t");
    for (int a = 0; a < n_slots; ++a)
        if (aterm_offsets[a + 1] <= aterm_offsets[a])
            return fail(IDG_ERR_INVALID_ARG, "aterm_offsets must be strictly increasing");
    for (int b = 0; b < n_bl; ++b)
        for (int k = 0; k < 2; ++k)
            if (baselines[2 * b + k] < 0 || baselines[2 * b + k] >= n_stations)
                return fail(IDG_ERR_INVALID_ARG, "baseline " + std::to_string(b) + " names a station out of range");
    for (int c = 0; c < n_chan; ++c)
        if (!(freqs_hz[c] > 0.0) || !std::isfinite(freqs_hz[c]))
            return fail(IDG_ERR_INVALID_ARG, "frequencies must be finite and > 0");
    // the channel recurrence needs uniformly spaced channels
    double ds = 0.0;
    if (n_chan > 1) {
        ds = (freqs_hz[n_chan - 1] - freqs_hz[0]) / (double)(n_chan - 1) / kSpeedOfLight;
        for (int c = 0; c < n_chan; ++c) {
            const double want = freqs_hz[0] / kSpeedOfLight + (double)c * ds;
            if (std::fabs(freqs_hz[c] / kSpeedOfLight - want) > 1e-9 * freqs_hz[0] / kSpeedOfLight) {
                ds = 0.0;
                break;
            }
        }
    }
    if (o.precision_mode == IDG_PHASOR_RECURRENCE && n_chan > 1 && ds == 0.0)
        return fail(IDG_ERR_INVALID_ARG, "precision_mode IDG_PHASOR_RECURRENCE needs uniformly spaced channels");
    const size_t n_uvw = (size_t)n_bl * n_t * 3;
    for (size_t i = 0; i < n_uvw; ++i)
        if (!std::isfinite(uvw_m[i])) return fail(IDG_ERR_INVALID_ARG, "uvw must be finite");

    idg_plan *p = new (std::nothrow) idg_plan();
    if (!p) return fail(IDG_ERR_NO_MEMORY, "host allocation of the plan failed");
    p->opts = o;
    p->n_bl = n_bl; p->n_t = n_t; p->n_chan = n_chan; p->n_stations = n_stations; p->n_slots = n_slots;
    p->L = L; p->N = N; p->cell = cell; p->w_step = w_step;
    p->S = (double)N * cell;
    p->ds = ds;
    p->baselines.assign(baselines, baselines + 2 * (size_t)n_bl);

    PlanParams pp{uvw_m, freqs_hz, aterm_offsets, n_bl, n_t, n_chan, n_slots, L, N, cell, w_step,
                  o.kernel_size, o.max_timesteps_per_subgrid, o.n_host_threads};
    PlanResult pr;
    try {
        pr = make_plan(pp);
    } catch (const std::bad_alloc &) {
        delete p;
        return fail(IDG_ERR_NO_MEMORY, "host allocation in the planner failed");
    }
    const int64_t n_sub = (int64_t)(pr.desc.size() / kDescFields);
    if (n_sub > INT32_MAX) {              // work orders, spans and tile lists hold int32 indices
        delete p;
        return fail(IDG_ERR_INVALID_ARG, "the plan has more subgrids than 32-bit subgrid indices hold");
    }
    p->desc = std::move(pr.desc);
    memset(&p->stats, 0, sizeof p->stats);
    p->stats.n_subgrids = n_sub;
    p->stats.n_vis_dropped = pr.n_dropped;
    p->stats.n_w_layers = pr.n_w;
    p->stats.w_layer_min = pr.k_min;
    p->stats.subgrid_size = L;
    p->stats.grid_size = N;
    p->stats.n_bl = n_bl; p->stats.n_t = n_t; p->stats.n_chan = n_chan;
    p->stats.n_stations = n_stations; p->stats.n_slots = n_slots;
    int64_t planned = 0, max_kp = 0;
    for (int64_t s = 0; s < n_sub; ++s) {
        const int64_t kp = p->desc[s * kDescFields + IDG_DESC_KP];
        planned += kp;
        max_kp = std::max(max_kp, kp);
    }
    p->stats.n_vis_planned = planned;
    p->kp_prefix_plan.assign((size_t)n_sub + 1, 0);
    p->kp_plan.assign((size_t)n_sub, 0);
    for (int64_t s = 0; s < n_sub; ++s) {
        p->kp_plan[s] = p->desc[s * kDescFields + IDG_DESC_KP];
        p->kp_prefix_plan[s + 1] = p->kp_prefix_plan[s] + p->kp_plan[s];
    }
    p->stats.max_kp = max_kp;
    p->any_dropped = pr.n_dropped > 0;

    // bound on the phase of the separable remainder: max |c_k| max |r(x, y)| with
    // c_k = 2 pi (w_k - w_s) and r = n'(x, y) - n'(x, j0) - n'(j0, y) + n'(j0, j0); per
    // subgrid the ends of its channel range bound the linear dependence on f.  Each
    // subgrid takes w_s = its w offset w0 when that meets the bound, else the middle
    // of its own w range (the separable kernels apply the rest, exp(+-2 pi i (w_s - w0)
    // n'(x, y)), to the subgrid image); the subgrids that meet the bound with it go to
    // the separable kernels, the others to the direct ones
    {
        auto n1 = [&](int x, int y) {
            const double l = ((double)x - 0.5 * L) * p->S / L;
            const double m = ((double)y - 0.5 * L) * p->S / L;
            return std::sqrt(1.0 - l * l - m * m) - 1.0;
        };
        // the reference row and column j0 of the split: r is about -(l^2 - l0^2)(m^2 - l0^2) / 4,
        // smallest in the largest |r| near l0^2 = half the largest l^2 (3 to 4 times smaller than
        // through the centre); the best j0 on the diagonal (n' is symmetric in l and m)
        double r_max = 0.0;
        p->sep_j0 = L / 2;
        for (int j = 0; j < L; ++j) {
            double rm = 0.0;
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) rm = std::max(rm, std::fabs(n1(x, y) - n1(x, j) - n1(j, y) + n1(j, j)));
            if (j == 0 || rm < r_max) {
                r_max = rm;
                p->sep_j0 = j;
            }
        }
        // (the separable degridder stages visibility indices in 31 bits)
        const bool fits = (int64_t)n_bl * n_t * n_chan < 0x7FFFFFFFll;
        const bool sized = separable_size(L) && fits;
        p->w_sep.assign((size_t)n_sub, 0.0);
        p->sep_sub.assign((size_t)n_sub, 0);
        p->split_sub.assign((size_t)n_sub, 0);
        p->pieces.clear();
        double theta = 0.0, c_max = 0.0;
        int64_t n_sep = 0, kp_sep = 0;
        for (int64_t s = 0; s < n_sub; ++s) {
            const int32_t *d = &p->desc[s * kDescFields];
            const double w0 = w_step > 0.0 ? (double)(d[IDG_DESC_LAYER] + pr.k_min) * w_step : 0.0;
            const int c0 = d[IDG_DESC_C0], c1 = d[IDG_DESC_C0] + d[IDG_DESC_NC] - 1;
            double lo = 0.0, hi = 0.0;
            for (int t = d[IDG_DESC_T0]; t < d[IDG_DESC_T0] + d[IDG_DESC_NT]; ++t) {
                const double w = uvw_m[((size_t)d[IDG_DESC_BASELINE] * n_t + t) * 3 + 2];
                const double wa = w * freqs_hz[c0] / kSpeedOfLight, wb = w * freqs_hz[c1] / kSpeedOfLight;
                if (t == d[IDG_DESC_T0]) lo = hi = wa;
                lo = std::min(lo, std::min(wa, wb));
                hi = std::max(hi, std::max(wa, wb));
            }
            const double cw0 = kTwoPi * std::max(std::fabs(lo - w0), std::fabs(hi - w0));
            const bool mid = cw0 * r_max > kSepThetaMax;
            const double cs = mid ? kTwoPi * 0.5 * (hi - lo) : cw0;
            p->w_sep[s] = mid ? 0.5 * (lo + hi) : w0;
            theta = std::max(theta, cs * r_max);
            if (sized && cs * r_max <= kSepThetaMax) {
                p->sep_sub[s] = 1;
                c_max = std::max(c_max, cs);
                ++n_sep;
                kp_sep += d[IDG_DESC_KP];
            } else if (sized) {
                split_pieces(p, s, r_max, uvw_m, freqs_hz, &c_max);
            }
        }
        p->sep_theta = theta;
        p->c_scale = 1.0f;
        if (c_max > 1.0) p->c_scale = (float)std::ldexp(1.0, -(int)std::ceil(std::log2(c_max)));
        p->r_scale = r_max > 0.0 ? (float)std::ldexp(1.0, std::min(100, (int)std::floor(std::log2(1.0 / r_max)))) : 1.0f;
        p->stats.separable = (sized && n_sep == n_sub) ? 1 : 0;
        p->stats.sep_phase = p->sep_theta;
        p->stats.n_sep_subgrids = n_sep;
        p->stats.n_vis_sep = kp_sep;
        p->stats.n_pieces = (int64_t)p->pieces.size();
        p->stats.n_split_subgrids = 0;
        p->stats.n_vis_split = 0;
        for (int64_t s = 0; s < n_sub; ++s)
            if (p->split_sub[s]) {
                ++p->stats.n_split_subgrids;
                p->stats.n_vis_split += p->desc[s * kDescFields + IDG_DESC_KP];
            }
    }

    // device metadata; without any CUDA device the plan stays host-only
    // (info and export work, device calls are rejected)
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || n_dev == 0) {
        cudaGetLastError();
        p->device = -1;
        p->stats.device = -1;
        *out = p;
        return IDG_OK;
    }
    e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
    p->stats.device = p->device;

    const double k_uv = kTwoPi * p->S / (double)L;      // as Geometry::k_uv
    std::vector<DevSubgrid> hsub((size_t)std::max<int64_t>(n_sub, 1));
    for (int64_t s = 0; s < n_sub; ++s) {
        const int32_t *d = &p->desc[s * kDescFields];
        DevSubgrid &g = hsub[s];
        g.bl = d[IDG_DESC_BASELINE]; g.slot = d[IDG_DESC_SLOT]; g.t0 = d[IDG_DESC_T0]; g.nt = d[IDG_DESC_NT];
        g.c0 = d[IDG_DESC_C0]; g.nc = d[IDG_DESC_NC]; g.q0 = d[IDG_DESC_Q0]; g.r0 = d[IDG_DESC_R0];
        g.layer = d[IDG_DESC_LAYER]; g.kp = d[IDG_DESC_KP];
        g.st_p = baselines[2 * g.bl]; g.st_q = baselines[2 * g.bl + 1];
        g.u0 = ((double)g.q0 + 0.5 * L - 0.5 * N) / p->S;
        g.v0 = ((double)g.r0 + 0.5 * L - 0.5 * N) / p->S;
        g.w0 = w_step > 0.0 ? (double)(g.layer + pr.k_min) * w_step : 0.0;
        split_pair(g.u0 * k_uv, g.a0h, g.a0l);
        split_pair(g.v0 * k_uv, g.b0h, g.b0l);
        split_pair(g.w0 * kTwoPi, g.c0h, g.c0l);
        const double ws = p->w_sep[s];
        split_pair(ws * kTwoPi, g.csh, g.csl);
        g.dws = (float)(2.0 * (ws - g.w0));
    }
    const int64_t n_pc = (int64_t)p->pieces.size();
    if (n_sub + n_pc > INT32_MAX) {
        delete p;
        return fail(IDG_ERR_INVALID_ARG, "the plan's subgrids and pieces exceed 32-bit work indices");
    }
    if (n_pc > 0) hsub.resize((size_t)(n_sub + n_pc));
    for (int64_t i = 0; i < n_pc; ++i) {
        const idg_plan::Piece &pc = p->pieces[i];
        DevSubgrid &g = hsub[n_sub + i];
        g = hsub[pc.parent];
        g.t0 = pc.t0; g.nt = pc.nt; g.c0 = pc.c0; g.nc = pc.nc; g.kp = pc.nt * pc.nc;
        split_pair(pc.ws * kTwoPi, g.csh, g.csl);
        g.dws = (float)(2.0 * (pc.ws - g.w0));
    }
    p->kp_all.assign((size_t)(n_sub + n_pc), 0);
    for (int64_t s = 0; s < n_sub + n_pc; ++s) p->kp_all[s] = hsub[s].kp;
    std::vector<int32_t> span_order;
    // device work order: the separable subgrids, then the others (one launch each),
    // each part with most visibilities first (longest-processing-time first for the
    // block scheduler), ties by A-term slot, then in plan order: the CTAs in flight then
    // share their slot's A-terms in L2 (a plan with A-terms every few timesteps has more
    // of them than L2 holds, and plan order is baseline-major)
    const auto work_first = [&](int32_t a, int32_t b) {
        if (p->sep_sub[a] != p->sep_sub[b]) return p->sep_sub[a] > p->sep_sub[b];
        if (hsub[a].kp != hsub[b].kp) return hsub[a].kp > hsub[b].kp;
        return hsub[a].slot < hsub[b].slot;
    };
    std::vector<int32_t> order((size_t)std::max<int64_t>(n_sub, 1));
    std::iota(order.begin(), order.begin() + n_sub, 0);
    std::stable_sort(order.begin(), order.begin() + n_sub, work_first);
    p->order.assign(order.begin(), order.begin() + n_sub);
    p->kp_prefix_order.assign((size_t)n_sub + 1, 0);
    p->kp_order.assign((size_t)n_sub, 0);
    p->sep_prefix_order.assign((size_t)n_sub + 1, 0);
    p->sep_prefix_plan.assign((size_t)n_sub + 1, 0);
    for (int64_t s = 0; s < n_sub; ++s) {
        p->kp_order[s] = hsub[order[s]].kp;
        p->kp_prefix_order[s + 1] = p->kp_prefix_order[s] + p->kp_order[s];
        p->sep_prefix_order[s + 1] = p->sep_prefix_order[s] + p->sep_sub[order[s]];
        p->sep_prefix_plan[s + 1] = p->sep_prefix_plan[s] + p->sep_sub[s];
    }
    // spans of whole baselines for the host-buffer calls (about 256 MB of
    // visibilities each, at least 4; the first and last cut to a quarter so the
    // copy pipeline fills and drains sooner), each span's subgrids by K_p descending
    {
        const int64_t vis_bytes = (int64_t)n_bl * n_t * n_chan * 32;
        int nk = (int)std::min<int64_t>(16, std::max<int64_t>(4, vis_bytes / (256ll << 20)));
        std::vector<double> frac;
        for (int k = 0; k <= nk; ++k) frac.push_back((double)k / nk);
        frac.insert(frac.begin() + 1, 0.25 / nk);
        frac.insert(frac.end() - 1, 1.0 - 0.25 / nk);
        bool sorted_bl = true;                   // the planner emits baseline-major order; otherwise one span
        for (int64_t s = 1; s < n_sub; ++s)
            if (hsub[s].bl < hsub[s - 1].bl) sorted_bl = false;
        if (!sorted_bl) frac = {0.0, 1.0};
        int64_t i = 0;
        int32_t last_b = -1;
        for (size_t k = 0; k < frac.size(); ++k) {
            const int32_t b = (int32_t)std::llround(frac[k] * n_bl);
            if (b == last_b) continue;           // spans of at least one baseline
            while (i < n_sub && hsub[i].bl < b) ++i;
            p->span_first.push_back(k + 1 == frac.size() ? n_sub : i);
            p->span_bl.push_back(b);
            last_b = b;
        }
        std::vector<int32_t> so((size_t)std::max<int64_t>(n_sub, 1));
        std::iota(so.begin(), so.begin() + n_sub, 0);
        for (size_t k = 0; k + 1 < p->span_first.size(); ++k)
            std::stable_sort(so.begin() + p->span_first[k], so.begin() + p->span_first[k + 1], work_first);
        p->kp_span_order.assign((size_t)n_sub, 0);
        p->kp_prefix_span.assign((size_t)n_sub + 1, 0);
        p->sep_prefix_span.assign((size_t)n_sub + 1, 0);
        for (int64_t s = 0; s < n_sub; ++s) {
            p->kp_span_order[s] = hsub[so[s]].kp;
            p->kp_prefix_span[s + 1] = p->kp_prefix_span[s] + p->kp_span_order[s];
            p->sep_prefix_span[s + 1] = p->sep_prefix_span[s] + p->sep_sub[so[s]];
        }
        span_order.swap(so);
    }
    // the composite calls' lists when some subgrids go in pieces: d_sub entries of the
    // separable subgrids and the pieces first, then the direct subgrids left, each part by
    // K_p descending; for the whole plan and per span
    std::vector<int32_t> fused_order, fused_span;
    if (n_pc > 0) {
        std::vector<int64_t> piece_first((size_t)n_sub + 1, 0);
        for (const auto &pc : p->pieces) ++piece_first[pc.parent + 1];
        for (int64_t s = 0; s < n_sub; ++s) piece_first[s + 1] += piece_first[s];
        auto sep_kind = [&](int32_t e) { return e >= n_sub || p->sep_sub[e]; };
        auto fused_first = [&](int32_t a, int32_t b) {
            if (sep_kind(a) != sep_kind(b)) return sep_kind(a);
            if (hsub[a].kp != hsub[b].kp) return hsub[a].kp > hsub[b].kp;
            return hsub[a].slot < hsub[b].slot;
        };
        // entries of plan subgrids [a, b): each subgrid itself, or its pieces
        auto entries = [&](int64_t a, int64_t b, std::vector<int32_t> &out) {
            for (int64_t s = a; s < b; ++s) {
                if (!p->split_sub[s]) out.push_back((int32_t)s);
                for (int64_t i = piece_first[s]; i < piece_first[s + 1]; ++i) out.push_back((int32_t)(n_sub + i));
            }
        };
        entries(0, n_sub, fused_order);
        std::stable_sort(fused_order.begin(), fused_order.end(), fused_first);
        p->fspan_first.assign(1, 0);
        for (size_t k = 0; k + 1 < p->span_first.size(); ++k) {
            const size_t a = fused_span.size();
            entries(p->span_first[k], p->span_first[k + 1], fused_span);
            std::stable_sort(fused_span.begin() + a, fused_span.end(), fused_first);
            p->fspan_first.push_back((int64_t)fused_span.size());
        }
        auto lists = [&](const std::vector<int32_t> &ord, std::vector<int32_t> &kp, std::vector<int64_t> &kpre,
                         std::vector<int64_t> &spre) {
            const size_t n = ord.size();
            kp.assign(n, 0);
            kpre.assign(n + 1, 0);
            spre.assign(n + 1, 0);
            for (size_t i = 0; i < n; ++i) {
                kp[i] = hsub[ord[i]].kp;
                kpre[i + 1] = kpre[i] + kp[i];
                spre[i + 1] = spre[i] + (sep_kind(ord[i]) ? 1 : 0);
            }
        };
        lists(fused_order, p->kp_fused_order, p->kp_prefix_fused, p->sep_prefix_fused);
        lists(fused_span, p->kp_fused_span, p->kp_prefix_fspan, p->sep_prefix_fspan);
    }
    std::vector<double> scale(n_chan);
    std::vector<float> scale_f2((size_t)4 * n_chan);
    for (int c = 0; c < n_chan; ++c) {
        scale[c] = freqs_hz[c] / kSpeedOfLight;
        split_pair(scale[c] * k_uv, scale_f2[4 * c], scale_f2[4 * c + 1]);
        split_pair(scale[c] * kTwoPi, scale_f2[4 * c + 2], scale_f2[4 * c + 3]);
    }
    // n' table, then the separable split n' = s(x) + t(y) + r(x, y) with s(x) = n'(x, j0)
    // and t(y) = n'(j0, y) - n'(j0, j0), j0 the plan's reference row and column
    std::vector<float> nprime((size_t)2 * L * L + 2 * L);
    auto n1 = [&](int x, int y) {
        const double l = ((double)x - 0.5 * L) * p->S / L;
        const double m = ((double)y - 0.5 * L) * p->S / L;
        return std::sqrt(1.0 - l * l - m * m) - 1.0;
    };
    const int j0 = p->sep_j0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            nprime[(size_t)y * L + x] = (float)n1(x, y);
            nprime[(size_t)L * L + 2 * L + (size_t)y * L + x] =
                (float)(n1(x, y) - n1(x, j0) - n1(j0, y) + n1(j0, j0));
        }
    for (int i = 0; i < L; ++i) {
        nprime[(size_t)L * L + i] = (float)n1(i, j0);
        nprime[(size_t)L * L + L + i] = (float)(n1(j0, i) - n1(j0, j0));
    }

    // the default taper (calls with a NULL taper): c[y][x] = a_y a_x with a the PSWF
    // window of the plan's beta (Sect. 4.1), as idg_taper_window gives it
    std::vector<float> taper_def;
    {
        std::vector<double> a((size_t)L);
        const std::string saved = g_last_error;
        if (idg_taper_window(L, o.kernel_size, IDG_TAPER_PSWF, a.data(), nullptr) == IDG_OK) {
            taper_def.resize((size_t)L * L);
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) taper_def[(size_t)y * L + x] = (float)(a[y] * a[x]);
        }
        g_last_error = saved;
    }

    const std::vector<float> ones((size_t)L * L, 1.0f);

    // IDG_ADDER_SORTED: for every grid tile that subgrids overlap, those subgrids in plan order
    std::vector<int32_t> tile_ids, tile_first, tile_sub;
    if (o.adder_mode == IDG_ADDER_SORTED && n_sub > 0) {
        const int ntx = (N + kTile - 1) / kTile;
        const int64_t per_layer = (int64_t)ntx * ntx, n_tiles = per_layer * p->stats.n_w_layers;
        std::vector<int32_t> count((size_t)n_tiles + 1, 0);
        auto each_tile = [&](int64_t s, auto &&fn) {
            const DevSubgrid &g = hsub[s];
            for (int ty = g.r0 / kTile; ty <= (g.r0 + L - 1) / kTile; ++ty)
                for (int tx = g.q0 / kTile; tx <= (g.q0 + L - 1) / kTile; ++tx) fn(g.layer * per_layer + ty * ntx + tx);
        };
        std::vector<int64_t> total((size_t)n_tiles + 1, 0);
        for (int64_t s = 0; s < n_sub; ++s) each_tile(s, [&](int64_t t) { ++total[t + 1]; });
        for (int64_t t = 0; t < n_tiles; ++t) total[t + 1] += total[t];
        if (total[n_tiles] > INT32_MAX) {
            delete p;
            return fail(IDG_ERR_INVALID_ARG, "the sorted adder's tile lists exceed 32-bit offsets");
        }
        for (int64_t t = 0; t <= n_tiles; ++t) count[t] = (int32_t)total[t];
        std::vector<int32_t> entries((size_t)count[n_tiles]), fill(count.begin(), count.end() - 1);
        for (int64_t s = 0; s < n_sub; ++s) each_tile(s, [&](int64_t t) { entries[fill[t]++] = (int32_t)s; });
        // the tiles with short lists first, then those with long lists (one cluster each)
        for (int heavy = 0; heavy < 2; ++heavy)
            for (int64_t t = 0; t < n_tiles; ++t) {
                const int32_t len = count[t + 1] - count[t];
                if (len == 0 || (len > kHeavyEntries) != (heavy == 1)) continue;
                tile_ids.push_back((int32_t)t);
                tile_first.push_back((int32_t)tile_sub.size());
                tile_sub.insert(tile_sub.end(), entries.begin() + count[t], entries.begin() + count[t + 1]);
                p->n_heavy_sorted += heavy;
            }
        tile_first.push_back((int32_t)tile_sub.size());
        p->n_tiles_sorted = (int64_t)tile_ids.size();
    }

    struct Up { void **dst; const void *src; size_t bytes; const char *what; };
    Up ups[] = {
        {(void **)&p->d_sub, hsub.data(), sizeof(DevSubgrid) * hsub.size(), "subgrid descriptors"},
        {(void **)&p->d_order, order.data(), sizeof(int32_t) * order.size(), "work order"},
        {(void **)&p->d_span_order, span_order.data(), sizeof(int32_t) * span_order.size(), "span order"},
        {(void **)&p->d_fused_order, fused_order.data(), sizeof(int32_t) * fused_order.size(), "piece work order"},
        {(void **)&p->d_fused_span, fused_span.data(), sizeof(int32_t) * fused_span.size(), "piece span order"},
        {(void **)&p->d_tile_ids, tile_ids.data(), sizeof(int32_t) * tile_ids.size(), "sorted adder tiles"},
        {(void **)&p->d_tile_first, tile_first.data(), sizeof(int32_t) * tile_first.size(), "sorted adder tile lists"},
        {(void **)&p->d_tile_sub, tile_sub.data(), sizeof(int32_t) * tile_sub.size(), "sorted adder tile subgrids"},
        {(void **)&p->d_uvw, uvw_m, sizeof(double) * n_uvw, "uvw"},
        {(void **)&p->d_scale, scale.data(), sizeof(double) * scale.size(), "channel scales"},
        {(void **)&p->d_scale_f2, scale_f2.data(), sizeof(float) * scale_f2.size(), "channel scale pairs"},
        {(void **)&p->d_nprime, nprime.data(), sizeof(float) * nprime.size(), "n' table"},
        {(void **)&p->d_taper, taper_def.data(), sizeof(float) * taper_def.size(), "default taper"},
        {(void **)&p->d_ones, ones.data(), sizeof(float) * ones.size(), "unit taper"},
    };
    // The uploads and the pair kernel run on a private non-blocking stream that only this
    // call waits for: plans are made on host threads while other threads run (and record
    // graphs of) their own work, and a device-wide synchronisation would wait on those
    // streams and invalidate a graph capture in progress.
    cudaStream_t ps = nullptr;
    e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        idg_plan_destroy(p);
        return cuda_fail(e, "plan upload stream");
    }
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    } guard{ps};
    for (auto &u : ups) {
        if (u.bytes == 0) continue;
        e = cudaMalloc(u.dst, u.bytes);
        if (e != cudaSuccess) {
            idg_status st = cuda_fail(e, (std::string("cudaMalloc(") + u.what + ")").c_str());
            cudaStreamSynchronize(ps);
            idg_plan_destroy(p);
            return st;
        }
        // (from pageable memory: the call returns once the source has been staged)
        e = cudaMemcpyAsync(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, ps);
        if (e != cudaSuccess) {
            idg_status st = cuda_fail(e, (std::string("cudaMemcpyAsync(") + u.what + ")").c_str());
            cudaStreamSynchronize(ps);
            idg_plan_destroy(p);
            return st;
        }
    }
    {
        const size_t n_bt = (size_t)n_bl * n_t;
        e = cudaMalloc((void **)&p->d_uvw_f2, sizeof(float) * 8 * std::max<size_t>(n_bt, 1));
        if (e == cudaSuccess && n_bt > 0) {
            split_uvw_kernel<<<(unsigned)((n_bt + 255) / 256), 256, 0, ps>>>(p->d_uvw, (float4 *)p->d_uvw_f2, n_bt);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
        if (e != cudaSuccess) {
            idg_status st = cuda_fail(e, "uvw pairs");
            cudaStreamSynchronize(ps);
            idg_plan_destroy(p);
            return st;
        }
    }
    *out = p;
    return IDG_OK;
}

idg_status idg_plan_info(const idg_plan *p, idg_plan_stats *out) {
    if (!p || !out) return fail(IDG_ERR_INVALID_ARG, "plan and out are required");
    *out = p->stats;
    return IDG_OK;
}

idg_status idg_plan_export(const idg_plan *p, int32_t *desc, int64_t cap) {
    if (!p || !desc) return fail(IDG_ERR_INVALID_ARG, "plan and desc are required");
    if (cap < p->stats.n_subgrids) return fail(IDG_ERR_INVALID_ARG, "desc capacity is smaller than n_subgrids");
    std::copy(p->desc.begin(), p->desc.end(), desc);
    return IDG_OK;
}

static idg_status no_default_taper() {
    return fail(IDG_ERR_INVALID_ARG, "the taper is NULL and the plan has no default taper");
}

static idg_status check_call(const idg_plan *p, const void *a, const char *an, const void *b, const char *bn) {
    if (!p) return fail(IDG_ERR_INVALID_ARG, "plan is NULL");
    if (!a) return fail(IDG_ERR_INVALID_ARG, std::string(an) + " is NULL");
    if (!b) return fail(IDG_ERR_INVALID_ARG, std::string(bn) + " is NULL");
    if (!gridder_supported(p->L))
        return fail(IDG_ERR_UNSUPPORTED, "subgrid size " + std::to_string(p->L) + " is not compiled in");
    return check_device(p);
}

// subgrid sets: [first, first + count) of the device work order or of plan order
static SubgridSet order_set(const idg_plan *p, int64_t first, int64_t count) {
    return SubgridSet{p->d_order + first, 0, count, p->kp_order.data() + first};
}
static SubgridSet plan_set(const idg_plan *p, int64_t first, int64_t count) {
    return SubgridSet{nullptr, first, count, p->kp_plan.data() + first};
}
static SubgridSet span_set(const idg_plan *p, int64_t first, int64_t count) {
    return SubgridSet{p->d_span_order + first, 0, count, p->kp_span_order.data() + first};
}

// positions of a launch: in the work order, in plan order, in the span order, or in the
// composite calls' lists with pieces (whole plan or per span)
enum class Order { Work, Plan, Span, Fused, FusedSpan };

static SubgridSet order_of(const idg_plan *p, Order o, int64_t first, int64_t count) {
    switch (o) {
    case Order::Work: return order_set(p, first, count);
    case Order::Plan: return plan_set(p, first, count);
    case Order::Span: return span_set(p, first, count);
    case Order::Fused: return SubgridSet{p->d_fused_order + first, 0, count, p->kp_fused_order.data() + first};
    default: return SubgridSet{p->d_fused_span + first, 0, count, p->kp_fused_span.data() + first};
    }
}

static const std::vector<int64_t> &kp_prefix(const idg_plan *p, Order o) {
    switch (o) {
    case Order::Work: return p->kp_prefix_order;
    case Order::Plan: return p->kp_prefix_plan;
    case Order::Span: return p->kp_prefix_span;
    case Order::Fused: return p->kp_prefix_fused;
    default: return p->kp_prefix_fspan;
    }
}

// algorithmic work of a launch over positions [first, first + count)
static double vispix(const idg_plan *p, int64_t first, int64_t count, Order o) {
    const auto &pre = kp_prefix(p, o);
    return (double)(pre[first + count] - pre[first]) * p->L * p->L;
}
static double pixels(const idg_plan *p, int64_t count) { return (double)count * p->L * p->L; }

static idg_status check_range(const idg_plan *p, int64_t first, int64_t count) {
    if (first < 0 || count < 0 || first + count > p->stats.n_subgrids)
        return fail(IDG_ERR_INVALID_ARG, "subgrid range out of the plan");
    return IDG_OK;
}

// The fused tensor-core kernels (L = 32) take the whole sequence of Algorithm 1
// (2) for a subgrid in one CTA, with the transform in shared memory; they serve
// the default kernel choice with the FP32 transform, direct phasors and the
// plain adder.  The degridder takes them when most visibilities of the launch
// lie in subgrids of at least kTcwFusedKpMin (direct) or kSepFusedKpMin
// (separable), as the default per-call choice does.
// the fused composite kernels: the direct tensor-core ones at L = 32, the separable ones at
// L = 32, 24 and 16 for subgrids that meet the remainder bound (the process-default kernel
// choice only); sep: the launch's subgrids take the separable kernels
static bool fused_size(const idg_plan *p, bool sep) { return p->L == 32 || (separable_size(p->L) && sep); }
static bool fused_grid(const idg_plan *p, bool sep) {
    return fused_size(p, sep) && p->opts.fft_mode == IDG_FFT_FP32 && p->opts.precision_mode == IDG_PHASOR_SINCOS &&
           p->opts.adder_mode == IDG_ADDER_ATOMIC && p->kernel_variant(IDG_KERNEL_GRIDDER) == 0;
}
static bool fused_degrid(const idg_plan *p, const SubgridSet &set, bool sep) {
    if (!(fused_size(p, sep) && p->opts.fft_mode == IDG_FFT_FP32 && p->opts.precision_mode == IDG_PHASOR_SINCOS &&
          p->kernel_variant(IDG_KERNEL_DEGRIDDER) == 0))
        return false;
    const int32_t kmin = sep ? kSepFusedKpMin : kTcwFusedKpMin;
    int64_t small = 0, all = 0;
    for (int64_t i = 0; i < set.count; ++i) {
        all += set.kp_host[i];
        if (set.kp_host[i] < kmin) small += set.kp_host[i];
    }
    return 2 * small <= all;
}

// Number of leading positions of [first, first + count) of order o that take the
// separable kernels: the separable subgrids when they come first in the range (the
// work order and every span list them first), else 0 and the direct kernels take
// the whole range (they serve every subgrid).
static int64_t sep_head(const idg_plan *p, Order o, int64_t first, int64_t count) {
    if (p->stats.separable) return count;
    const auto &pre = o == Order::Work    ? p->sep_prefix_order
                      : o == Order::Plan  ? p->sep_prefix_plan
                      : o == Order::Span  ? p->sep_prefix_span
                      : o == Order::Fused ? p->sep_prefix_fused
                                          : p->sep_prefix_fspan;
    if (pre.empty()) return 0;
    const int64_t ns = pre[first + count] - pre[first];
    return pre[first + ns] - pre[first] == ns ? ns : 0;
}

// the adder's per-call device buffer: the compensation grid (IDG_ADDER_COMPENSATED); none
// for the atomic and the sorted adder
static size_t adder_buffer_bytes(const idg_plan *p) {
    if (p->opts.adder_mode == IDG_ADDER_COMPENSATED) return (size_t)p->stats.n_w_layers * p->N * p->N * 32;
    return 0;
}
static SortedTiles sorted_tiles(const idg_plan *p) {
    return SortedTiles{p->d_tile_ids, p->d_tile_first, p->d_tile_sub, p->n_tiles_sorted, p->n_heavy_sorted};
}

// the composite calls need the subgrid scratch for a part that runs unfused
static bool grid_needs_scratch(const idg_plan *p, Order o, int64_t first, int64_t count) {
    const int64_t ns = sep_head(p, o, first, count);
    return p->opts.adder_mode != IDG_ADDER_ATOMIC || (ns > 0 && !fused_grid(p, true)) ||
           (ns < count && !fused_grid(p, false));
}
static bool degrid_needs_scratch(const idg_plan *p, Order o, int64_t first, int64_t count) {
    const int64_t ns = sep_head(p, o, first, count);
    return (ns > 0 && !fused_degrid(p, order_of(p, o, first, ns), true)) ||
           (ns < count && !fused_degrid(p, order_of(p, o, first + ns, count - ns), false));
}
// Whole-plan composite calls and the host-buffer calls' spans run over the lists with
// pieces when the plan has pieces and the separable kernels take them fused; else over
// the plan's subgrids (work order, span order).
static bool use_pieces(const idg_plan *p, bool grid) {
    if (p->pieces.empty()) return false;
    if (grid) return fused_grid(p, true);
    return fused_degrid(p, order_of(p, Order::Fused, 0, p->sep_prefix_fused.back()), true);
}
struct Lists {
    Order whole, span;
    int64_t n;                              // entries of the whole-plan list
    const std::vector<int64_t> *span_first; // span k at [(*span_first)[k], (*span_first)[k + 1])
};
static Lists lists_for(const idg_plan *p, bool grid) {
    // the sorted adder takes its subgrids in chunks of consecutive plan indices
    if (grid && p->opts.adder_mode == IDG_ADDER_SORTED)
        return Lists{Order::Plan, Order::Plan, p->stats.n_subgrids, &p->span_first};
    if (use_pieces(p, grid))
        return Lists{Order::Fused, Order::FusedSpan, (int64_t)p->kp_fused_order.size(), &p->fspan_first};
    return Lists{Order::Work, Order::Span, p->stats.n_subgrids, &p->span_first};
}

// the same over every span of the host-buffer calls
static bool spans_need_scratch(const idg_plan *p, bool grid) {
    const Lists ls = lists_for(p, grid);
    const auto &sf = *ls.span_first;
    for (size_t k = 0; k + 1 < sf.size(); ++k)
        if (sf[k + 1] > sf[k] && (grid ? grid_needs_scratch(p, ls.span, sf[k], sf[k + 1] - sf[k])
                                       : degrid_needs_scratch(p, ls.span, sf[k], sf[k + 1] - sf[k])))
            return true;
    return false;
}

// Grid the subgrids at positions [first, first + count) of the order o, all of one
// kind (g.separable), in pieces of at most `chunk` subgrids that pass through the
// subgrid scratch (gridder -> transform -> adder), or in one fused launch (no scratch).
static idg_status grid_part(const idg_plan *p, const Geometry &g, Order o, int64_t first, int64_t count,
                            void *scratch, int64_t chunk, const void *vis, const uint8_t *flags, const void *aterms,
                            const float *taper, void *grid, void *cbuf, cudaStream_t s) {
    if (!cbuf && fused_grid(p, g.separable != 0)) {
        ProfileScope ps(IDG_KERNEL_GRIDDER, s, vispix(p, first, count, o));
        const SubgridSet set = order_of(p, o, first, count);
        return g.separable ? launch_gridder_sep_fused(g, set, vis, flags, aterms, taper, grid, s)
                           : launch_gridder_tcw_fused(g, set, vis, flags, aterms, taper, grid, s);
    }
    idg_status st = IDG_OK;
    for (int64_t f = first; f < first + count && st == IDG_OK; f += chunk) {
        const int64_t cnt = std::min(chunk, first + count - f);
        const SubgridSet set = order_of(p, o, f, cnt);
        {
            ProfileScope ps(IDG_KERNEL_GRIDDER, s, vispix(p, f, cnt, o));
            st = launch_gridder(g, set, p->kernel_variant(IDG_KERNEL_GRIDDER), vis, flags, aterms, taper, scratch, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_FFT, s, (double)cnt);
            st = launch_subgrid_fft(p, cnt, -1, scratch, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_ADDER, s, 96.0 * pixels(p, cnt));
            st = p->opts.adder_mode == IDG_ADDER_SORTED ? launch_adder_sorted(g, set, scratch, grid, sorted_tiles(p), s)
                 : cbuf                                 ? launch_adder_compensated(g, set, scratch, grid, cbuf, s)
                                                        : launch_adder(g, set, scratch, grid, s);
        }
    }
    return st;
}

// Degrid the subgrids [first, first + count), all of one kind (splitter -> transform
// -> degridder), or in one fused launch.
static idg_status degrid_part(const idg_plan *p, const Geometry &g, Order o, int64_t first, int64_t count,
                              void *scratch, int64_t chunk, const void *grid, const uint8_t *flags, const void *aterms,
                              const float *taper, void *vis_out, cudaStream_t s) {
    const SubgridSet all = order_of(p, o, first, count);
    if (fused_degrid(p, all, g.separable != 0)) {
        ProfileScope ps(IDG_KERNEL_DEGRIDDER, s, vispix(p, first, count, o));
        return g.separable ? launch_degridder_sep_fused(g, all, grid, flags, aterms, taper, vis_out, s)
                           : launch_degridder_tcw_fused(g, all, grid, flags, aterms, taper, vis_out, s);
    }
    idg_status st = IDG_OK;
    for (int64_t f = first; f < first + count && st == IDG_OK; f += chunk) {
        const int64_t cnt = std::min(chunk, first + count - f);
        const SubgridSet set = order_of(p, o, f, cnt);
        {
            ProfileScope ps(IDG_KERNEL_SPLITTER, s, 64.0 * pixels(p, cnt));
            st = launch_splitter(g, set, grid, scratch, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_FFT, s, (double)cnt);
            st = launch_subgrid_fft(p, cnt, +1, scratch, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_DEGRIDDER, s, vispix(p, f, cnt, o));
            st = launch_degridder(g, set, p->kernel_variant(IDG_KERNEL_DEGRIDDER), scratch, flags, aterms, taper, vis_out, s);
        }
    }
    return st;
}

// A range of positions: its separable head by the separable kernels, the rest by the
// direct ones (g: the plan's geometry).
static idg_status grid_span(const idg_plan *p, const Geometry &g, Order o, int64_t first, int64_t count,
                            void *scratch, int64_t chunk, const void *vis, const uint8_t *flags, const void *aterms,
                            const float *taper, void *grid, void *cbuf, cudaStream_t s) {
    const int64_t ns = sep_head(p, o, first, count);
    Geometry gp = g;
    idg_status st = IDG_OK;
    if (ns > 0) {
        gp.separable = 1;
        st = grid_part(p, gp, o, first, ns, scratch, chunk, vis, flags, aterms, taper, grid, cbuf, s);
    }
    if (st == IDG_OK && ns < count) {
        gp.separable = 0;
        st = grid_part(p, gp, o, first + ns, count - ns, scratch, chunk, vis, flags, aterms, taper, grid, cbuf, s);
    }
    return st;
}

static idg_status degrid_span(const idg_plan *p, const Geometry &g, Order o, int64_t first, int64_t count,
                              void *scratch, int64_t chunk, const void *grid, const uint8_t *flags, const void *aterms,
                              const float *taper, void *vis_out, cudaStream_t s) {
    const int64_t ns = sep_head(p, o, first, count);
    Geometry gp = g;
    idg_status st = IDG_OK;
    if (ns > 0) {
        gp.separable = 1;
        st = degrid_part(p, gp, o, first, ns, scratch, chunk, grid, flags, aterms, taper, vis_out, s);
    }
    if (st == IDG_OK && ns < count) {
        gp.separable = 0;
        st = degrid_part(p, gp, o, first + ns, count - ns, scratch, chunk, grid, flags, aterms, taper, vis_out, s);
    }
    return st;
}

// The composite calls over the positions [first, first + count) of order o
// (the whole plan in work order for idg_grid / idg_degrid, a plan-order range
// for the range calls).
static idg_status grid_call(const idg_plan *p, Order o, int64_t first, int64_t count, const void *vis,
                            const uint8_t *flags, const void *aterms, const float *taper, void *grid,
                            cudaStream_t s) {
    if (count == 0) return IDG_OK;
    idg_status st = IDG_OK;
    const int64_t chunk = std::min(chunk_subgrids(p), count);
    const bool comp = p->opts.adder_mode == IDG_ADDER_COMPENSATED;
    void *scratch = nullptr;     // the subgrid scratch, unless fused launches take the call
    if (grid_needs_scratch(p, o, first, count))
        st = scratch_alloc(p->device, (size_t)chunk * p->L * p->L * 32, s, &scratch);
    if (st != IDG_OK) return st;
    const Geometry g = p->geometry();
    const size_t grid_f4 = (size_t)p->stats.n_w_layers * p->N * p->N * 2;
    const size_t abytes = adder_buffer_bytes(p);
    void *cbuf = nullptr;      // the compensation grid or the sorted adder's marks, zeroed
    if (abytes) {
        st = scratch_alloc(p->device, abytes, s, &cbuf);
        if (st == IDG_OK) {
            cudaError_t e0 = cudaMemsetAsync(cbuf, 0, abytes, s);
            if (e0 != cudaSuccess) st = cuda_fail(e0, "cudaMemsetAsync(adder buffer)");
        }
    }
    if (st == IDG_OK) st = grid_span(p, g, o, first, count, scratch, chunk, vis, flags, aterms, taper, grid, cbuf, s);
    if (cbuf) {
        if (st == IDG_OK && comp) st = launch_fold_compensation(grid, cbuf, grid_f4, s);
        cudaFreeAsync(cbuf, s);
    }
    cudaError_t e = scratch ? cudaFreeAsync(scratch, s) : cudaSuccess;
    if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaFreeAsync(scratch)");
    return st;
}

static idg_status degrid_call(const idg_plan *p, Order o, int64_t first, int64_t count, const void *grid,
                              const uint8_t *flags, const void *aterms, const float *taper, void *vis_out,
                              cudaStream_t s) {
    if (count == 0) return IDG_OK;
    idg_status st = IDG_OK;
    const int64_t chunk = std::min(chunk_subgrids(p), count);
    void *scratch = nullptr;
    if (degrid_needs_scratch(p, o, first, count))
        st = scratch_alloc(p->device, (size_t)chunk * p->L * p->L * 32, s, &scratch);
    if (st != IDG_OK) return st;
    st = degrid_span(p, p->geometry(), o, first, count, scratch, chunk, grid, flags, aterms, taper, vis_out, s);
    cudaError_t e = scratch ? cudaFreeAsync(scratch, s) : cudaSuccess;
    if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaFreeAsync(scratch)");
    return st;
}

idg_status idg_aterm_gradient(const idg_plan *p, const void *grid, const void *vis, const uint8_t *flags,
                              const void *aterms, const float *taper, void *residual, void *gradient, double *cost,
                              idg_stream stream) {
    idg_status st = check_call(p, grid, "d_grid", vis, "d_vis");
    if (st != IDG_OK) return st;
    if (!residual) return fail(IDG_ERR_INVALID_ARG, "d_residual is NULL");
    if (!gradient) return fail(IDG_ERR_INVALID_ARG, "d_gradient is NULL");
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = p->stats.n_subgrids;
    if (p->any_dropped || n == 0) {
        cudaError_t e = cudaMemsetAsync(residual, 0, (size_t)p->n_bl * p->n_t * p->n_chan * 32, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(residual)");
    }
    if (n == 0) return IDG_OK;
    // two scratch areas of `chunk` subgrid images: the model's P and the residuals' R
    const int64_t chunk = std::max<int64_t>(1, chunk_subgrids(p) / 2);
    const size_t img = (size_t)p->L * p->L * 32;
    void *scratch = nullptr;
    if ((st = scratch_alloc(p->device, 2 * (size_t)chunk * img, s, &scratch)) != IDG_OK) return st;
    void *P = scratch, *R = (char *)scratch + (size_t)chunk * img;
    const Geometry g = p->geometry();
    const int vd = p->kernel_variant(IDG_KERNEL_DEGRIDDER), vg = p->kernel_variant(IDG_KERNEL_GRIDDER);
    for (int64_t f = 0; f < n && st == IDG_OK; f += chunk) {
        const int64_t cnt = std::min(chunk, n - f);
        const SubgridSet set = order_set(p, f, cnt);
        {
            ProfileScope ps(IDG_KERNEL_SPLITTER, s, 64.0 * pixels(p, cnt));
            st = launch_splitter(g, set, grid, P, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_FFT, s, (double)cnt);
            st = launch_subgrid_fft(p, cnt, +1, P, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_DEGRIDDER, s, vispix(p, f, cnt, Order::Work));
            st = launch_degridder(g, set, vd, P, flags, aterms, taper, residual, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_CALIB_RESIDUAL, s,
                            96.0 * (double)(p->kp_prefix_order[f + cnt] - p->kp_prefix_order[f]));
            st = launch_calib_residual(g, set, vis, flags, residual, cost, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_GRIDDER, s, vispix(p, f, cnt, Order::Work));
            st = launch_gridder(g, set, vg, residual, flags, nullptr, p->d_ones, R, s);
        }
        if (st == IDG_OK) {
            ProfileScope ps(IDG_KERNEL_CALIB_GRADIENT, s, 256.0 * pixels(p, cnt));
            st = launch_calib_gradient(g, set, R, P, aterms, taper, gradient, s);
        }
    }
    cudaError_t e = cudaFreeAsync(scratch, s);
    if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaFreeAsync(scratch)");
    return st;
}

idg_status idg_grid(const idg_plan *p, const void *vis, const uint8_t *flags, const void *aterms,
                    const float *taper, void *grid, idg_stream stream) {
    idg_status st = check_call(p, vis, "d_vis", grid, "d_grid");
    if (st != IDG_OK) return st;
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    const Lists ls = lists_for(p, true);
    return grid_call(p, ls.whole, 0, ls.n, vis, flags, aterms, taper, grid, (cudaStream_t)stream);
}

idg_status idg_degrid(const idg_plan *p, const void *grid, const uint8_t *flags, const void *aterms,
                      const float *taper, void *vis_out, idg_stream stream) {
    idg_status st = check_call(p, grid, "d_grid", vis_out, "d_vis_out");
    if (st != IDG_OK) return st;
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = p->stats.n_subgrids;
    if (p->any_dropped || n == 0) {
        cudaError_t e = cudaMemsetAsync(vis_out, 0, (size_t)p->n_bl * p->n_t * p->n_chan * 32, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(vis_out)");
    }
    const Lists ls = lists_for(p, false);
    return degrid_call(p, ls.whole, 0, ls.n, grid, flags, aterms, taper, vis_out, s);
}

idg_status idg_grid_range(const idg_plan *p, int64_t first, int64_t count, const void *vis, const uint8_t *flags,
                          const void *aterms, const float *taper, void *grid, idg_stream stream) {
    idg_status st = check_call(p, vis, "d_vis", grid, "d_grid");
    if (st != IDG_OK) return st;
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    if ((st = check_range(p, first, count)) != IDG_OK) return st;
    return grid_call(p, Order::Plan, first, count, vis, flags, aterms, taper, grid, (cudaStream_t)stream);
}

idg_status idg_degrid_range(const idg_plan *p, int64_t first, int64_t count, const void *grid, const uint8_t *flags,
                            const void *aterms, const float *taper, void *vis_out, idg_stream stream) {
    idg_status st = check_call(p, grid, "d_grid", vis_out, "d_vis_out");
    if (st != IDG_OK) return st;
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    if ((st = check_range(p, first, count)) != IDG_OK) return st;
    return degrid_call(p, Order::Plan, first, count, grid, flags, aterms, taper, vis_out, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// host-buffer variants
//
// Visibilities are stored baseline-major and the plan orders subgrids by
// baseline, so the call is cut into spans of whole baselines whose
// visibilities are one contiguous range.  A private copy stream moves span k
// while the caller's stream computes span k - 1 (gridding) or k + 1
// (degridding); events order the two streams.  The grid itself moves before
// (degridding) or after (gridding) the spans.

namespace {
struct DevBufs {
    void *ptr[7] = {};
    cudaStream_t s;
    explicit DevBufs(cudaStream_t st) : s(st) {}
    ~DevBufs() {
        for (void *p : ptr)
            if (p) cudaFreeAsync(p, s);
    }
};

// On an early return of a host-buffer call: the compute stream waits for the copy
// stream's work and the call returns only after both ended, so that no copy still
// reads the caller's host memory, or writes a buffer freed on the compute stream.
struct CopyJoin {
    cudaStream_t s, cs;
    bool done = false;
    CopyJoin(cudaStream_t st, cudaStream_t cst) : s(st), cs(cst) {}
    ~CopyJoin() {
        if (done) return;
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
            if (cudaEventRecord(e, cs) == cudaSuccess) cudaStreamWaitEvent(s, e, 0);
            cudaEventDestroy(e);
        }
        cudaStreamSynchronize(s);
    }
};

struct Events {
    std::vector<cudaEvent_t> ev;
    ~Events() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    cudaError_t add(cudaEvent_t *out) {
        cudaError_t e = cudaEventCreateWithFlags(out, cudaEventDisableTiming);
        if (e == cudaSuccess) ev.push_back(*out);
        return e;
    }
};

std::mutex g_copy_mu;
cudaStream_t g_copy_stream[64] = {};

idg_status copy_stream(int dev, cudaStream_t *out) {
    if (dev < 0 || dev >= 64) return fail(IDG_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_copy_mu);
    if (!g_copy_stream[dev]) {
        cudaError_t e = cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "creating the copy stream");
    }
    *out = g_copy_stream[dev];
    return IDG_OK;
}

idg_status h2d(void *d, const void *h, size_t bytes, cudaStream_t cs, const char *what) {
    if (!h || !bytes) return IDG_OK;
    cudaError_t e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, cs);
    return e == cudaSuccess ? IDG_OK : cuda_fail(e, what);
}
}  // namespace

idg_status idg_grid_host(const idg_plan *p, const void *h_vis, const uint8_t *h_flags, const void *h_aterms,
                         const float *h_taper, void *h_grid, idg_stream stream) {
    idg_status st = check_call(p, h_vis, "h_vis", h_grid, "h_grid");
    if (st != IDG_OK) return st;
    if (!h_taper && !p->d_taper) return no_default_taper();
    cudaStream_t s = (cudaStream_t)stream, cs = nullptr;
    if ((st = copy_stream(p->device, &cs)) != IDG_OK) return st;
    const size_t per_bl = (size_t)p->n_t * p->n_chan;      // visibilities per baseline
    const size_t nvis = (size_t)p->n_bl * per_bl;
    const size_t grid_bytes = (size_t)p->stats.n_w_layers * p->N * p->N * 32;
    const size_t at_bytes = h_aterms ? (size_t)p->n_slots * p->n_stations * p->L * p->L * 32 : 0;
    const int64_t chunk = chunk_subgrids(p);
    DevBufs b(s);
    CopyJoin join(s, cs);
    const bool comp = p->opts.adder_mode == IDG_ADDER_COMPENSATED;
    const size_t sizes[6] = {nvis * 32, h_flags ? nvis : 0, at_bytes, h_taper ? (size_t)p->L * p->L * 4 : 0, grid_bytes,
                             spans_need_scratch(p, true) ? (size_t)chunk * p->L * p->L * 32 : 0};
    for (int k = 0; k < 6 && st == IDG_OK; ++k)
        if (sizes[k]) st = scratch_alloc(p->device, sizes[k], s, &b.ptr[k]);
    const size_t grid_f4 = grid_bytes / 16;
    const size_t abytes = adder_buffer_bytes(p);
    if (st == IDG_OK && abytes) st = scratch_alloc(p->device, abytes, s, &b.ptr[6]);
    if (st != IDG_OK) return st;
    Events ev;
    cudaEvent_t e_alloc, e_end;
    cudaError_t e = ev.add(&e_alloc);
    if (e == cudaSuccess) e = ev.add(&e_end);
    if (e == cudaSuccess) e = cudaEventRecord(e_alloc, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, e_alloc, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.ptr[4], 0, grid_bytes, s);
    if (e == cudaSuccess && abytes) e = cudaMemsetAsync(b.ptr[6], 0, abytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "grid_host setup");
    if ((st = h2d(b.ptr[2], h_aterms, at_bytes, cs, "copy of A-terms")) != IDG_OK) return st;
    if ((st = h2d(b.ptr[3], h_taper, sizes[3], cs, "copy of taper")) != IDG_OK) return st;
    const Lists ls = lists_for(p, true);
    const auto &sf = *ls.span_first;
    const auto &sb = p->span_bl;
    const Geometry g = p->geometry();
    for (size_t k = 0; k + 1 < sf.size() && st == IDG_OK; ++k) {
        const size_t v0 = (size_t)sb[k] * per_bl, nv = (size_t)(sb[k + 1] - sb[k]) * per_bl;
        st = h2d((char *)b.ptr[0] + v0 * 32, (const char *)h_vis + v0 * 32, nv * 32, cs, "copy of visibilities");
        if (st == IDG_OK && h_flags)
            st = h2d((char *)b.ptr[1] + v0, h_flags + v0, nv, cs, "copy of flags");
        cudaEvent_t e_up;
        if (st == IDG_OK && (e = ev.add(&e_up)) == cudaSuccess && (e = cudaEventRecord(e_up, cs)) == cudaSuccess)
            e = cudaStreamWaitEvent(s, e_up, 0);
        if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "ordering the copy and compute streams");
        if (st == IDG_OK && sf[k + 1] > sf[k])
            st = grid_span(p, g, ls.span, sf[k], sf[k + 1] - sf[k], b.ptr[5], chunk, b.ptr[0],
                           (const uint8_t *)b.ptr[1], b.ptr[2], h_taper ? (const float *)b.ptr[3] : p->d_taper, b.ptr[4],
                           b.ptr[6], s);
    }
    if (st == IDG_OK && comp) st = launch_fold_compensation(b.ptr[4], b.ptr[6], grid_f4, s);
    // the copy stream's work ends before the buffers are released on s
    e = cudaEventRecord(e_end, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e_end, 0);
    if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "ordering the copy and compute streams");
    if (st != IDG_OK) return st;
    e = cudaMemcpyAsync(h_grid, b.ptr[4], grid_bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the grid to the host");
    e = cudaStreamSynchronize(s);
    join.done = true;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return IDG_OK;
}

idg_status idg_degrid_host(const idg_plan *p, const void *h_grid, const uint8_t *h_flags, const void *h_aterms,
                           const float *h_taper, void *h_vis_out, idg_stream stream) {
    idg_status st = check_call(p, h_grid, "h_grid", h_vis_out, "h_vis_out");
    if (st != IDG_OK) return st;
    if (!h_taper && !p->d_taper) return no_default_taper();
    cudaStream_t s = (cudaStream_t)stream, cs = nullptr;
    if ((st = copy_stream(p->device, &cs)) != IDG_OK) return st;
    const size_t per_bl = (size_t)p->n_t * p->n_chan;
    const size_t nvis = (size_t)p->n_bl * per_bl;
    const size_t grid_bytes = (size_t)p->stats.n_w_layers * p->N * p->N * 32;
    const size_t at_bytes = h_aterms ? (size_t)p->n_slots * p->n_stations * p->L * p->L * 32 : 0;
    const int64_t chunk = chunk_subgrids(p);
    DevBufs b(s);
    CopyJoin join(s, cs);
    const size_t sizes[6] = {grid_bytes, h_flags ? nvis : 0, at_bytes, h_taper ? (size_t)p->L * p->L * 4 : 0, nvis * 32,
                             (size_t)chunk * p->L * p->L * 32};
    for (int k = 0; k < 6 && st == IDG_OK; ++k)
        if (sizes[k]) st = scratch_alloc(p->device, sizes[k], s, &b.ptr[k]);
    if (st != IDG_OK) return st;
    Events ev;
    cudaEvent_t e_alloc, e_in, e_end;
    cudaError_t e = ev.add(&e_alloc);
    if (e == cudaSuccess) e = ev.add(&e_in);
    if (e == cudaSuccess) e = ev.add(&e_end);
    if (e == cudaSuccess) e = cudaEventRecord(e_alloc, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, e_alloc, 0);
    if (e != cudaSuccess) return cuda_fail(e, "degrid_host setup");
    if ((st = h2d(b.ptr[0], h_grid, grid_bytes, cs, "copy of the grid")) != IDG_OK) return st;
    if ((st = h2d(b.ptr[1], h_flags, sizes[1], cs, "copy of flags")) != IDG_OK) return st;
    if ((st = h2d(b.ptr[2], h_aterms, at_bytes, cs, "copy of A-terms")) != IDG_OK) return st;
    if ((st = h2d(b.ptr[3], h_taper, sizes[3], cs, "copy of taper")) != IDG_OK) return st;
    e = cudaEventRecord(e_in, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e_in, 0);
    if (e == cudaSuccess && p->any_dropped) e = cudaMemsetAsync(b.ptr[4], 0, nvis * 32, s);
    if (e != cudaSuccess) return cuda_fail(e, "degrid_host inputs");
    const Lists ls = lists_for(p, false);
    const auto &sf = *ls.span_first;
    const auto &sb = p->span_bl;
    const Geometry g = p->geometry();
    for (size_t k = 0; k + 1 < sf.size() && st == IDG_OK; ++k) {
        if (sf[k + 1] > sf[k])
            st = degrid_span(p, g, ls.span, sf[k], sf[k + 1] - sf[k], b.ptr[5], chunk, b.ptr[0],
                             (const uint8_t *)b.ptr[1], b.ptr[2], h_taper ? (const float *)b.ptr[3] : p->d_taper,
                             b.ptr[4], s);
        cudaEvent_t e_done;
        if (st == IDG_OK && (e = ev.add(&e_done)) == cudaSuccess && (e = cudaEventRecord(e_done, s)) == cudaSuccess)
            e = cudaStreamWaitEvent(cs, e_done, 0);
        if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "ordering the copy and compute streams");
        if (st == IDG_OK) {
            const size_t v0 = (size_t)sb[k] * per_bl, nv = (size_t)(sb[k + 1] - sb[k]) * per_bl;
            e = cudaMemcpyAsync((char *)h_vis_out + v0 * 32, (const char *)b.ptr[4] + v0 * 32, nv * 32,
                                cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) st = cuda_fail(e, "copy of the visibilities to the host");
        }
    }
    e = cudaEventRecord(e_end, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e_end, 0);
    if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "ordering the copy and compute streams");
    if (st != IDG_OK) return st;
    e = cudaStreamSynchronize(s);
    join.done = true;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return IDG_OK;
}

// Both directions in one call: the visibilities gridded into h_grid and the model grid
// degridded into h_vis_out.  One copy stream carries, in order, the shared inputs, the
// visibility spans (each released to the compute stream as it lands), the model grid
// (which lands while the gridding still runs), then -- once the gridding is done -- the
// gridded grid back to the host while the degridding runs, and the model visibilities
// span by span behind the degridding.
idg_status idg_grid_degrid_host(const idg_plan *p, const void *h_vis, const void *h_model, const uint8_t *h_flags,
                                const void *h_aterms, const float *h_taper, void *h_grid, void *h_vis_out,
                                idg_stream stream) {
    idg_status st = check_call(p, h_vis, "h_vis", h_grid, "h_grid");
    if (st != IDG_OK) return st;
    if (!h_model) return fail(IDG_ERR_INVALID_ARG, "h_model is NULL");
    if (!h_vis_out) return fail(IDG_ERR_INVALID_ARG, "h_vis_out is NULL");
    if (!h_taper && !p->d_taper) return no_default_taper();
    cudaStream_t s = (cudaStream_t)stream, cs = nullptr;
    if ((st = copy_stream(p->device, &cs)) != IDG_OK) return st;
    const size_t per_bl = (size_t)p->n_t * p->n_chan;
    const size_t nvis = (size_t)p->n_bl * per_bl;
    const size_t grid_bytes = (size_t)p->stats.n_w_layers * p->N * p->N * 32;
    const size_t at_bytes = h_aterms ? (size_t)p->n_slots * p->n_stations * p->L * p->L * 32 : 0;
    const int64_t chunk = chunk_subgrids(p);
    const bool comp = p->opts.adder_mode == IDG_ADDER_COMPENSATED;
    DevBufs b(s);
    // 0 vis, 1 flags, 2 A-terms, 3 taper, 4 grid out, 5 scratch, 6 compensation; model grid and
    // model visibilities in a second set
    DevBufs b2(s);
    CopyJoin join(s, cs);
    const size_t sizes[6] = {nvis * 32, h_flags ? nvis : 0, at_bytes, h_taper ? (size_t)p->L * p->L * 4 : 0,
                             grid_bytes, (size_t)chunk * p->L * p->L * 32};
    for (int k = 0; k < 6 && st == IDG_OK; ++k)
        if (sizes[k]) st = scratch_alloc(p->device, sizes[k], s, &b.ptr[k]);
    const size_t grid_f4 = grid_bytes / 16;
    const size_t abytes = adder_buffer_bytes(p);
    if (st == IDG_OK && abytes) st = scratch_alloc(p->device, abytes, s, &b.ptr[6]);
    if (st == IDG_OK) st = scratch_alloc(p->device, grid_bytes, s, &b2.ptr[0]);       // model grid
    if (st == IDG_OK) st = scratch_alloc(p->device, nvis * 32, s, &b2.ptr[1]);        // model visibilities
    if (st != IDG_OK) return st;
    const float *taper = h_taper ? (const float *)b.ptr[3] : p->d_taper;
    Events ev;
    cudaEvent_t e_alloc, e_model, e_grid_done, e_end;
    cudaError_t e = ev.add(&e_alloc);
    if (e == cudaSuccess) e = ev.add(&e_model);
    if (e == cudaSuccess) e = ev.add(&e_grid_done);
    if (e == cudaSuccess) e = ev.add(&e_end);
    if (e == cudaSuccess) e = cudaEventRecord(e_alloc, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, e_alloc, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.ptr[4], 0, grid_bytes, s);
    if (e == cudaSuccess && abytes) e = cudaMemsetAsync(b.ptr[6], 0, abytes, s);
    if (e == cudaSuccess && p->any_dropped) e = cudaMemsetAsync(b2.ptr[1], 0, nvis * 32, s);
    if (e != cudaSuccess) return cuda_fail(e, "grid_degrid_host setup");
    if ((st = h2d(b.ptr[2], h_aterms, at_bytes, cs, "copy of A-terms")) != IDG_OK) return st;
    if ((st = h2d(b.ptr[3], h_taper, sizes[3], cs, "copy of taper")) != IDG_OK) return st;
    if ((st = h2d(b.ptr[1], h_flags, sizes[1], cs, "copy of flags")) != IDG_OK) return st;
    const Lists lg = lists_for(p, true), ld = lists_for(p, false);
    const auto &sf = p->span_first;                // spans of baselines (the same k in every list)
    const auto &sb = p->span_bl;
    const Geometry g = p->geometry();
    // gridding, span by span behind the visibility copies
    for (size_t k = 0; k + 1 < sf.size() && st == IDG_OK; ++k) {
        const size_t v0 = (size_t)sb[k] * per_bl, nv = (size_t)(sb[k + 1] - sb[k]) * per_bl;
        st = h2d((char *)b.ptr[0] + v0 * 32, (const char *)h_vis + v0 * 32, nv * 32, cs, "copy of visibilities");
        cudaEvent_t e_up;
        if (st == IDG_OK && (e = ev.add(&e_up)) == cudaSuccess && (e = cudaEventRecord(e_up, cs)) == cudaSuccess)
            e = cudaStreamWaitEvent(s, e_up, 0);
        if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "ordering the copy and compute streams");
        if (st == IDG_OK && sf[k + 1] > sf[k])
            st = grid_span(p, g, lg.span, (*lg.span_first)[k], (*lg.span_first)[k + 1] - (*lg.span_first)[k],
                           b.ptr[5], chunk, b.ptr[0],
                           (const uint8_t *)b.ptr[1], b.ptr[2], taper, b.ptr[4], b.ptr[6], s);
    }
    // the model grid lands while the gridding runs
    if (st == IDG_OK) st = h2d(b2.ptr[0], h_model, grid_bytes, cs, "copy of the model grid");
    if (st == IDG_OK && (e = cudaEventRecord(e_model, cs)) != cudaSuccess) st = cuda_fail(e, "model event");
    if (st == IDG_OK && comp) st = launch_fold_compensation(b.ptr[4], b.ptr[6], grid_f4, s);
    if (st == IDG_OK && (e = cudaEventRecord(e_grid_done, s)) != cudaSuccess) st = cuda_fail(e, "grid event");
    // the gridded grid goes back while the degridding runs
    if (st == IDG_OK && (e = cudaStreamWaitEvent(cs, e_grid_done, 0)) == cudaSuccess)
        e = cudaMemcpyAsync(h_grid, b.ptr[4], grid_bytes, cudaMemcpyDeviceToHost, cs);
    if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "copy of the grid to the host");
    if (st == IDG_OK && (e = cudaStreamWaitEvent(s, e_model, 0)) != cudaSuccess) st = cuda_fail(e, "model wait");
    // degridding, span by span ahead of the visibility copies back
    for (size_t k = 0; k + 1 < sf.size() && st == IDG_OK; ++k) {
        if (sf[k + 1] > sf[k])
            st = degrid_span(p, g, ld.span, (*ld.span_first)[k], (*ld.span_first)[k + 1] - (*ld.span_first)[k],
                             b.ptr[5], chunk, b2.ptr[0],
                             (const uint8_t *)b.ptr[1], b.ptr[2], taper, b2.ptr[1], s);
        cudaEvent_t e_done;
        if (st == IDG_OK && (e = ev.add(&e_done)) == cudaSuccess && (e = cudaEventRecord(e_done, s)) == cudaSuccess)
            e = cudaStreamWaitEvent(cs, e_done, 0);
        if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "ordering the copy and compute streams");
        if (st == IDG_OK) {
            const size_t v0 = (size_t)sb[k] * per_bl, nv = (size_t)(sb[k + 1] - sb[k]) * per_bl;
            e = cudaMemcpyAsync((char *)h_vis_out + v0 * 32, (const char *)b2.ptr[1] + v0 * 32, nv * 32,
                                cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) st = cuda_fail(e, "copy of the visibilities to the host");
        }
    }
    // the copy stream's work ends before the buffers are released on s
    e = cudaEventRecord(e_end, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e_end, 0);
    if (st == IDG_OK && e != cudaSuccess) st = cuda_fail(e, "ordering the copy and compute streams");
    if (st != IDG_OK) return st;
    e = cudaStreamSynchronize(s);
    join.done = true;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return IDG_OK;
}

// ---------------------------------------------------------------------------
// stage entry points

idg_status idg_grid_subgrids(const idg_plan *p, int64_t first, int64_t count, const void *vis,
                             const uint8_t *flags, const void *aterms, const float *taper, void *sub,
                             idg_stream stream) {
    idg_status st = check_call(p, vis, "d_vis", sub, "d_subgrids");
    if (st != IDG_OK) return st;
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    if ((st = check_range(p, first, count)) != IDG_OK || count == 0) return st;
    ProfileScope ps(IDG_KERNEL_GRIDDER, stream, vispix(p, first, count, Order::Plan));
    return launch_gridder(p->geometry(), plan_set(p, first, count), p->kernel_variant(IDG_KERNEL_GRIDDER), vis,
                          flags, aterms, taper, sub, stream);
}

idg_status idg_fft_subgrids(const idg_plan *p, int64_t count, int direction, void *sub, idg_stream stream) {
    idg_status st = check_call(p, sub, "d_subgrids", sub, "d_subgrids");
    if (st != IDG_OK) return st;
    if (direction != -1 && direction != 1) return fail(IDG_ERR_INVALID_ARG, "direction must be -1 or +1");
    if (count < 0) return fail(IDG_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return IDG_OK;
    ProfileScope ps(IDG_KERNEL_FFT, stream, (double)count);
    return launch_subgrid_fft(p, count, direction, sub, stream);
}

idg_status idg_add_subgrids(const idg_plan *p, int64_t first, int64_t count, const void *sub, void *grid,
                            idg_stream stream) {
    idg_status st = check_call(p, sub, "d_subgrids", grid, "d_grid");
    if (st != IDG_OK) return st;
    if ((st = check_range(p, first, count)) != IDG_OK || count == 0) return st;
    ProfileScope ps(IDG_KERNEL_ADDER, stream, 96.0 * pixels(p, count));
    if (p->opts.adder_mode == IDG_ADDER_SORTED)   // (a plan-order range is what the sorted adder takes)
        return launch_adder_sorted(p->geometry(), plan_set(p, first, count), sub, grid, sorted_tiles(p), stream);
    return launch_adder(p->geometry(), plan_set(p, first, count), sub, grid, stream);
}

idg_status idg_split_subgrids(const idg_plan *p, int64_t first, int64_t count, const void *grid, void *sub,
                              idg_stream stream) {
    idg_status st = check_call(p, grid, "d_grid", sub, "d_subgrids");
    if (st != IDG_OK) return st;
    if ((st = check_range(p, first, count)) != IDG_OK || count == 0) return st;
    ProfileScope ps(IDG_KERNEL_SPLITTER, stream, 64.0 * pixels(p, count));
    return launch_splitter(p->geometry(), plan_set(p, first, count), grid, sub, stream);
}

idg_status idg_degrid_subgrids(const idg_plan *p, int64_t first, int64_t count, const void *sub,
                               const uint8_t *flags, const void *aterms, const float *taper, void *vis_out,
                               idg_stream stream) {
    idg_status st = check_call(p, sub, "d_subgrids", vis_out, "d_vis_out");
    if (st != IDG_OK) return st;
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    if ((st = check_range(p, first, count)) != IDG_OK || count == 0) return st;
    ProfileScope ps(IDG_KERNEL_DEGRIDDER, stream, vispix(p, first, count, Order::Plan));
    return launch_degridder(p->geometry(), plan_set(p, first, count), p->kernel_variant(IDG_KERNEL_DEGRIDDER), sub,
                            flags, aterms, taper, vis_out, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// kernel variants and the autotuner

namespace idg {
namespace {
std::atomic<int> g_variant[IDG_KERNEL_COUNT][65];
}

int get_variant(int kernel, int L) {
    if (kernel < 0 || kernel >= IDG_KERNEL_COUNT || L < 0 || L > 64) return 0;
    return g_variant[kernel][L].load(std::memory_order_relaxed);
}

void set_variant(int kernel, int L, int v) {
    if (kernel < 0 || kernel >= IDG_KERNEL_COUNT || L < 0 || L > 64) return;
    g_variant[kernel][L].store(v, std::memory_order_relaxed);
}
}  // namespace idg

extern "C" {

int idg_kernel_variant_count(int kernel, int L) {
    if (kernel == IDG_KERNEL_GRIDDER) return gridder_variant_count(L);
    if (kernel == IDG_KERNEL_DEGRIDDER) return degridder_variant_count(L);
    if (kernel == IDG_KERNEL_BATCH_GRID || kernel == IDG_KERNEL_BATCH_DEGRID) return batch_variant_count(kernel, L);
    if (kernel >= 0 && kernel < IDG_KERNEL_COUNT) return gridder_supported(L) ? 1 : 0;
    return 0;
}

const char *idg_kernel_variant_name(int kernel, int L, int v) {
    if (kernel == IDG_KERNEL_GRIDDER) return gridder_variant_name(L, v);
    if (kernel == IDG_KERNEL_DEGRIDDER) return degridder_variant_name(L, v);
    if (kernel == IDG_KERNEL_BATCH_GRID || kernel == IDG_KERNEL_BATCH_DEGRID) return batch_variant_name(kernel, L, v);
    if (kernel >= 0 && kernel < IDG_KERNEL_COUNT && v == 0 && gridder_supported(L)) return "default";
    return nullptr;
}

idg_status idg_set_kernel_variant(int kernel, int L, int v) {
    const int n = idg_kernel_variant_count(kernel, L);
    if (n == 0) return fail(IDG_ERR_INVALID_ARG, "no such kernel or subgrid size");
    if (v < 0 || v >= n) return fail(IDG_ERR_INVALID_ARG, "variant out of range");
    set_variant(kernel, L, v);
    return IDG_OK;
}

int idg_get_kernel_variant(int kernel, int L) { return get_variant(kernel, L); }

idg_status idg_plan_set_kernel_variant(idg_plan *p, int kernel, int v) {
    if (!p) return fail(IDG_ERR_INVALID_ARG, "plan is NULL");
    if (kernel != IDG_KERNEL_GRIDDER && kernel != IDG_KERNEL_DEGRIDDER)
        return fail(IDG_ERR_INVALID_ARG, "a plan holds a choice for the gridder and the degridder only");
    const int n = idg_kernel_variant_count(kernel, p->L);
    if (n == 0) return fail(IDG_ERR_INVALID_ARG, "no such kernel for the plan's subgrid size");
    if (v < -1 || v >= n) return fail(IDG_ERR_INVALID_ARG, "variant out of range");
    p->variant[kernel].store(v, std::memory_order_relaxed);
    return IDG_OK;
}

int idg_plan_get_kernel_variant(const idg_plan *p, int kernel) {
    if (!p || kernel < 0 || kernel >= IDG_KERNEL_COUNT) return -1;
    return p->kernel_variant(kernel);
}

idg_status idg_autotune(const idg_plan *p, const void *vis, const uint8_t *flags, const void *aterms,
                        const float *taper, void *vis_scratch, int64_t max_subgrids, double *gridder_ms,
                        double *degridder_ms, int cap, idg_stream stream) {
    idg_status st = check_call(p, vis, "d_vis", vis, "d_vis");
    if (st != IDG_OK) return st;
    if (!(taper = p->taper_or_default(taper))) return no_default_taper();
    const int64_t n = p->stats.n_subgrids;
    if (n == 0) return IDG_OK;
    const int64_t m = std::min<int64_t>(n, max_subgrids > 0 ? max_subgrids : 4096);
    cudaStream_t s = (cudaStream_t)stream;
    // strided sample of the work order: it stays sorted by K_p
    std::vector<int32_t> hidx((size_t)m), hkp((size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        const int64_t pos = i * n / m;
        hidx[i] = p->order[pos];
        hkp[i] = p->kp_order[pos];
    }
    void *d_idx = nullptr, *scratch = nullptr;
    if ((st = scratch_alloc(p->device, sizeof(int32_t) * (size_t)m, s, &d_idx)) != IDG_OK) return st;
    if ((st = scratch_alloc(p->device, (size_t)m * p->L * p->L * 32, s, &scratch)) != IDG_OK) {
        cudaFreeAsync(d_idx, s);
        return st;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t ce = cudaMemcpyAsync(d_idx, hidx.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) st = cuda_fail(ce, "autotune index upload");
    const Geometry g = p->geometry();
    const SubgridSet set{(const int32_t *)d_idx, 0, m, hkp.data()};
    constexpr int kReps = 3;
    auto time_variants = [&](int kernel, int nvar, double *out_ms, auto &&launch) -> int {
        int best = 0;
        double best_ms = 1e300;
        for (int v = 0; v < nvar && st == IDG_OK; ++v) {
            st = launch(v);   // warm-up
            if (st != IDG_OK) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < kReps && st == IDG_OK; ++r) st = launch(v);
            cudaEventRecord(e1, s);
            ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) { st = cuda_fail(ce, "autotune timing"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double t = ms / kReps;
            if (out_ms && v < cap) out_ms[v] = t;
            if (t < best_ms) { best_ms = t; best = v; }
        }
        if (st == IDG_OK) p->variant[kernel].store(best, std::memory_order_relaxed);
        return best;
    };
    if (st == IDG_OK)
        time_variants(IDG_KERNEL_GRIDDER, gridder_variant_count(p->L), gridder_ms, [&](int v) {
            return launch_gridder(g, set, v, vis, flags, aterms, taper, scratch, s);
        });
    if (st == IDG_OK && vis_scratch)
        time_variants(IDG_KERNEL_DEGRIDDER, degridder_variant_count(p->L), degridder_ms, [&](int v) {
            return launch_degridder(g, set, v, scratch, flags, aterms, taper, vis_scratch, s);
        });
    cudaFreeAsync(scratch, s);
    cudaFreeAsync(d_idx, s);
    ce = cudaStreamSynchronize(s);
    if (st == IDG_OK && ce != cudaSuccess) st = cuda_fail(ce, "autotune synchronize");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // extern "C"
