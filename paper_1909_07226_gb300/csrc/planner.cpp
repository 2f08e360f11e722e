// Host planner: partition of the visibilities into subgrids (Sect. 3.2, Fig. 2).
//
// Baselines are planned independently on a pool of host threads; the results
// are concatenated in baseline order, so the plan does not depend on the
// thread count.  Every floating-point step is written so that it rounds the
// same way on every IEEE-754 host: compile with -ffp-contract=off.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "idg_internal.h"

namespace idg {
namespace {

struct Box {
    double umin, umax, vmin, vmax, wmin, wmax;
    void reset() {
        umin = vmin = wmin = INFINITY;
        umax = vmax = wmax = -INFINITY;
    }
    void take(double u, double v, double w) {
        umin = std::min(umin, u); umax = std::max(umax, u);
        vmin = std::min(vmin, v); vmax = std::max(vmax, v);
        wmin = std::min(wmin, w); wmax = std::max(wmax, w);
    }
    void merge(const Box &o) {
        umin = std::min(umin, o.umin); umax = std::max(umax, o.umax);
        vmin = std::min(vmin, o.vmin); vmax = std::max(vmax, o.vmax);
        wmin = std::min(wmin, o.wmin); wmax = std::max(wmax, o.wmax);
    }
};

// Central pixel of an extent: its midpoint rounded half up.
inline double centre_of(double lo, double hi) { return std::floor((lo + hi) * 0.5 + 0.5); }

struct Rules {
    double smax;      // (L - beta + 1) / 2, allowed shift from the centre (Sect. 4.3)
    double half_L;
    double N;
    double w_step;

    bool size_ok(const Box &b) const {
        const double cu = centre_of(b.umin, b.umax), cv = centre_of(b.vmin, b.vmax);
        if (cu - b.umin > smax || b.umax - cu > smax) return false;
        if (cv - b.vmin > smax || b.vmax - cv > smax) return false;
        if (w_step > 0.0 && b.wmax - b.wmin > w_step) return false;
        return true;
    }
    bool ok(const Box &b) const {
        if (!size_ok(b)) return false;
        const double cu = centre_of(b.umin, b.umax), cv = centre_of(b.vmin, b.vmax);
        return cu - half_L >= 0.0 && cu + half_L <= N && cv - half_L >= 0.0 && cv + half_L <= N;
    }
};

struct Emitted {
    int32_t f[kDescFields];
    int64_t k;   // absolute w-layer
};

struct BaselinePlan {
    std::vector<Emitted> out;
    int64_t dropped = 0;
};

void plan_baseline(const PlanParams &p, const Rules &R, const std::vector<double> &scale, int b,
                   std::vector<double> &pu, std::vector<double> &pv, std::vector<double> &pw,
                   BaselinePlan &res) {
    const int nt = p.n_t, nc = p.n_chan;
    const double S = (double)p.N * p.cell;
    const double halfN = 0.5 * p.N;
    // grid-pixel coordinates of every (t, c) sample of this baseline
    for (int t = 0; t < nt; ++t) {
        const double *x = p.uvw + ((size_t)b * nt + t) * 3;
        for (int c = 0; c < nc; ++c) {
            const double sc = scale[c];
            pu[(size_t)t * nc + c] = (x[0] * sc) * S + halfN;
            pv[(size_t)t * nc + c] = (x[1] * sc) * S + halfN;
            pw[(size_t)t * nc + c] = x[2] * sc;
        }
    }
    auto box_of = [&](int t, int c0, int n) {
        Box bx;
        bx.reset();
        for (int c = c0; c < c0 + n; ++c) {
            const size_t i = (size_t)t * nc + c;
            bx.take(pu[i], pv[i], pw[i]);
        }
        return bx;
    };
    for (int a = 0; a < p.n_slots; ++a) {
        const int ts = p.aterm_offsets[a], te = p.aterm_offsets[a + 1];
        // fewest channel groups such that each single timestep of each group fits by size
        int G = 1;
        for (; G < nc; ++G) {
            bool all = true;
            const int base = nc / G, extra = nc % G;
            for (int t = ts; t < te && all; ++t) {
                int c0 = 0;
                for (int g = 0; g < G && all; ++g) {
                    const int n = base + (g < extra ? 1 : 0);
                    all = R.size_ok(box_of(t, c0, n));
                    c0 += n;
                }
            }
            if (all) break;
        }
        const int base = nc / G, extra = nc % G;
        int c0 = 0;
        for (int g = 0; g < G; ++g) {
            const int n = base + (g < extra ? 1 : 0);
            int t = ts;
            while (t < te) {
                Box blk = box_of(t, c0, n);
                if (!R.ok(blk)) {          // a single timestep whose box leaves the grid
                    res.dropped += n;
                    ++t;
                    continue;
                }
                const int t0 = t++;
                while (t < te && t - t0 < p.t_max) {
                    Box next = blk;
                    next.merge(box_of(t, c0, n));
                    if (!R.ok(next)) break;
                    blk = next;
                    ++t;
                }
                Emitted e;
                const double cu = centre_of(blk.umin, blk.umax);
                const double cv = centre_of(blk.vmin, blk.vmax);
                e.k = p.w_step > 0.0 ? (int64_t)std::floor((blk.wmin + blk.wmax) * 0.5 / p.w_step + 0.5) : 0;
                e.f[IDG_DESC_BASELINE] = b;
                e.f[IDG_DESC_SLOT] = a;
                e.f[IDG_DESC_T0] = t0;
                e.f[IDG_DESC_NT] = t - t0;
                e.f[IDG_DESC_C0] = c0;
                e.f[IDG_DESC_NC] = n;
                e.f[IDG_DESC_Q0] = (int32_t)cu - p.L / 2;
                e.f[IDG_DESC_R0] = (int32_t)cv - p.L / 2;
                e.f[IDG_DESC_LAYER] = 0;
                e.f[IDG_DESC_KP] = (t - t0) * n;
                res.out.push_back(e);
            }
            c0 += n;
        }
    }
}

}  // namespace

PlanResult make_plan(const PlanParams &p) {
    Rules R;
    R.smax = ((double)p.L - p.beta + 1.0) * 0.5;
    R.half_L = 0.5 * p.L;
    R.N = (double)p.N;
    R.w_step = p.w_step;
    std::vector<double> scale(p.n_chan);
    for (int c = 0; c < p.n_chan; ++c) scale[c] = p.freqs[c] / kSpeedOfLight;

    std::vector<BaselinePlan> per_bl(p.n_bl);
    int nthreads = p.n_threads > 0 ? p.n_threads : (int)std::thread::hardware_concurrency();
    nthreads = std::max(1, std::min(nthreads, p.n_bl));
    std::atomic<int> next{0};
    auto worker = [&]() {
        std::vector<double> pu((size_t)p.n_t * p.n_chan), pv(pu.size()), pw(pu.size());
        for (;;) {
            const int b = next.fetch_add(1);
            if (b >= p.n_bl) break;
            plan_baseline(p, R, scale, b, pu, pv, pw, per_bl[b]);
        }
    };
    if (nthreads == 1) {
        worker();
    } else {
        std::vector<std::thread> pool;
        for (int i = 0; i < nthreads; ++i) pool.emplace_back(worker);
        for (auto &th : pool) th.join();
    }

    PlanResult res;
    size_t total = 0;
    bool any = false;
    int64_t kmin = 0, kmax = 0;
    for (auto &bp : per_bl) {
        total += bp.out.size();
        res.n_dropped += bp.dropped;
        for (auto &e : bp.out) {
            if (!any || e.k < kmin) kmin = e.k;
            if (!any || e.k > kmax) kmax = e.k;
            any = true;
        }
    }
    res.desc.resize(total * kDescFields);
    size_t i = 0;
    for (auto &bp : per_bl) {
        for (auto &e : bp.out) {
            e.f[IDG_DESC_LAYER] = (int32_t)(e.k - kmin);
            std::copy(e.f, e.f + kDescFields, res.desc.begin() + i * kDescFields);
            ++i;
        }
    }
    res.k_min = (int32_t)kmin;
    res.n_w = any ? (int32_t)(kmax - kmin + 1) : 1;
    return res;
}

}  // namespace idg
