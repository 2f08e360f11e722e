// Anti-aliasing windows for image domain gridding (Sect. 4.1-4.3, appendix), host FP64.
//
// The taper c[i][j] = a_i a_j is an input of the gridder and degridder.  Two 1D windows
// of L samples are offered, each with its aliasing level (Table 1):
//   - the zeroth prolate spheroidal wave function psi_0(c = pi beta / 2, eta = 2(x - L/2)/L)
//     (Sect. 4.1): the optimal window of classical gridding for kernel support beta; its
//     side-lobe energy is eps^2 = 1 - lambda_0(c) (the classical-gridding column);
//   - the optimal window of image domain gridding (Sect. 4.3): the minimiser of the mean
//     side-lobe energy of the effective window over the allowed sample positions,
//     eps^2 = a^T Rbar a / a^T a, Rbar = Qbar (Hadamard) Sbar (appendix), i.e. the
//     eigenvector of Rbar's smallest eigenvalue.
//
// Coordinates are in samples: sample k sits at x = k (k = 0 .. L-1) and the main lobe is
// [0, L), so sample L/2 is its centre.  A sample shifted by s pixels from the subgrid
// centre sees the phases exp(i 2 pi (k - l) s / L); s ranges over the allowed shifts
// |s| <= (L - beta + 1) / 2 (the reading of the allowed shift used by the planner).
//
// Qbar_kl = integral over x < 0 and x > L of sinc(x - k) sinc(x - l) (sinc(t) = sin(pi t) /
// (pi t)).  With sin(pi (x - k)) = (-1)^k sin(pi x) and partial fractions,
//   k != l:  Qbar_kl = (-1)^(k+l) / (pi^2 (k - l)) [G(k) - G(l) - G(L - k) + G(L - l)],
//            G(t) = (ln|t| - Ci(2 pi |t|)) / 2, an even antiderivative of sin^2(pi t) / t,
//            continuous at 0 with G(0) = -(gamma + ln 2 pi) / 2;
//   k == l:  Qbar_kk = 1 - (Si(2 pi k) + Si(2 pi (L - k))) / pi,
// from the antiderivative -sin^2(pi t) / (pi^2 t) + Si(2 pi t) / pi of sinc^2.  These are
// the closed forms the appendix builds on the cosine integral Ci.
// Sbar_kl = the mean of exp(i 2 pi (k - l) s / L) over |s| <= W / 2, W = L - beta + 1:
//   Sbar_kl = sinc((k - l) W / L).
#include <cmath>
#include <complex>
#include <vector>

#include "idg_internal.h"

namespace idg {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kEulerGamma = 0.57721566490153286060651209008240243;

// Si(x) and Ci(x), x > 0.  Small x: the power series
//   Si(x) = sum_k (-1)^k x^(2k+1) / ((2k+1) (2k+1)!),
//   Ci(x) = gamma + ln x + sum_{k>=1} (-1)^k x^(2k) / (2k (2k)!)   (Abramowitz & Stegun 5.2.14, 5.2.16);
// larger x: E1(ix) = -Ci(x) + i (Si(x) - pi/2) from the continued fraction
//   E1(z) = e^-z / (z + 1 - 1^2 / (z + 3 - 2^2 / (z + 5 - ...)))   (A&S 5.1.22),
// evaluated by the modified Lentz method.
void sici(double x, double &si, double &ci) {
    if (x <= 2.0) {
        const double x2 = x * x;
        double term = x, s = x;                 // k = 0 term of Si
        for (int k = 1; k < 60; ++k) {
            term *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
            const double add = term / (2.0 * k + 1.0);
            s += add;
            if (std::fabs(add) < 1e-18 * std::fabs(s)) break;
        }
        double tc = 1.0, c = 0.0;
        for (int k = 1; k < 60; ++k) {
            tc *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
            const double add = tc / (2.0 * k);
            c += add;
            if (std::fabs(add) < 1e-18 * (std::fabs(c) + 1e-300)) break;
        }
        si = s;
        ci = kEulerGamma + std::log(x) + c;
        return;
    }
    using cd = std::complex<double>;
    const cd z(0.0, x);
    const double tiny = 1e-300;
    cd b = z + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 1000; ++i) {
        const double an = -(double)i * (double)i;
        b += 2.0;
        d = 1.0 / (an * d + b);
        c = b + an / c;
        const cd del = c * d;
        h *= del;
        if (std::fabs(del.real() - 1.0) + std::fabs(del.imag()) < 1e-16) break;
    }
    const cd e1 = h * cd(std::cos(x), -std::sin(x));    // e^{-ix} times the fraction
    ci = -e1.real();
    si = kPi / 2.0 + e1.imag();
}

double sinc(double t) { return t == 0.0 ? 1.0 : std::sin(kPi * t) / (kPi * t); }

// G(t) = (ln|t| - Ci(2 pi |t|)) / 2, continuous at 0
double G(double t) {
    t = std::fabs(t);
    if (t == 0.0) return -(kEulerGamma + std::log(2.0 * kPi)) / 2.0;
    double si, ci;
    sici(2.0 * kPi * t, si, ci);
    return (std::log(t) - ci) / 2.0;
}

// Rbar = Qbar (Hadamard) Sbar, row-major L x L
std::vector<double> rbar(int L, double beta) {
    std::vector<double> g(L + 1), si(L + 1);
    for (int t = 0; t <= L; ++t) {
        g[t] = G((double)t);
        double s = 0.0, c = 0.0;
        if (t > 0) sici(2.0 * kPi * t, s, c);
        si[t] = s;
    }
    const double W = (double)L - beta + 1.0;
    std::vector<double> R((size_t)L * L);
    for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l) {
            double q;
            if (k == l) {
                q = 1.0 - (si[k] + si[L - k]) / kPi;
            } else {
                const double sgn = ((k + l) & 1) ? -1.0 : 1.0;
                q = sgn / (kPi * kPi * (double)(k - l)) * (g[k] - g[l] - g[L - k] + g[L - l]);
            }
            R[(size_t)k * L + l] = q * sinc((double)(k - l) * W / (double)L);
        }
    return R;
}

// Eigenpairs of a symmetric matrix A (n x n, row-major, overwritten) by cyclic Jacobi
// rotations (Golub & Van Loan, Sect. 8.5): eigenvalues in w, eigenvectors in the columns of V.
void jacobi_eigh(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, total = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                const double a = A[(size_t)p * n + q] * A[(size_t)p * n + q];
                total += a;
                if (p != q) off += a;
            }
        if (off <= 1e-32 * total || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// psi_0(c, .) in the normalised even Legendre polynomials sqrt(m + 1/2) P_m (m = 2j): the
// eigenvector of the smallest eigenvalue of the prolate operator's symmetric tridiagonal
// matrix in that basis (Bouwkamp; Xiao, Rokhlin & Yarvin 2001).  Sign: d_0 > 0.
std::vector<double> pswf_coeffs(double c, int n_terms) {
    std::vector<double> M((size_t)n_terms * n_terms, 0.0);
    for (int j = 0; j < n_terms; ++j) {
        const double m = 2.0 * j;
        M[(size_t)j * n_terms + j] = m * (m + 1.0) + c * c * (2.0 * m * (m + 1.0) - 1.0) / ((2.0 * m + 3.0) * (2.0 * m - 1.0));
        if (j + 1 < n_terms) {
            const double o = c * c * (m + 2.0) * (m + 1.0) / ((2.0 * m + 3.0) * std::sqrt((2.0 * m + 1.0) * (2.0 * m + 5.0)));
            M[(size_t)j * n_terms + j + 1] = o;
            M[(size_t)(j + 1) * n_terms + j] = o;
        }
    }
    std::vector<double> w, V;
    jacobi_eigh(n_terms, M, w, V);
    int imin = 0;
    for (int i = 1; i < n_terms; ++i)
        if (w[i] < w[imin]) imin = i;
    std::vector<double> d(n_terms);
    for (int j = 0; j < n_terms; ++j) d[j] = V[(size_t)j * n_terms + imin];
    if (d[0] < 0.0)
        for (double &v : d) v = -v;
    return d;
}

// sum_j d_j sqrt(2j + 1/2) P_2j(x), P_n by the three-term recurrence
double legendre_even_series(const std::vector<double> &d, double x) {
    double p_prev = 1.0, p_cur = x, sum = d[0] * std::sqrt(0.5);
    int n = 1;
    for (size_t j = 1; j < d.size(); ++j) {
        while (n < 2 * (int)j) {
            const double p_next = ((2.0 * n + 1.0) * x * p_cur - n * p_prev) / (n + 1.0);
            p_prev = p_cur;
            p_cur = p_next;
            ++n;
        }
        sum += d[j] * std::sqrt(2.0 * j + 0.5) * p_cur;
    }
    return sum;
}

idg_status check_args(int L, double beta) {
    if (L < 2 || L > 512 || (L & 1))
        return fail(IDG_ERR_INVALID_ARG, "the window length must be even, 2 .. 512");
    if (!(beta > 0.0) || !(beta < (double)L + 1.0) || !std::isfinite(beta))
        return fail(IDG_ERR_INVALID_ARG, "beta must lie in (0, L + 1)");
    return IDG_OK;
}

}  // namespace
}  // namespace idg

using namespace idg;

extern "C" {

idg_status idg_taper_window(int L, double beta, int kind, double *a_out, double *eps_out) {
    idg_status st = check_args(L, beta);
    if (st != IDG_OK) return st;
    if (!a_out && !eps_out) return fail(IDG_ERR_INVALID_ARG, "a_out and eps_out are both NULL");
    if (kind == IDG_TAPER_PSWF) {
        const double c = kPi * beta / 2.0;
        const std::vector<double> d = pswf_coeffs(c, 64);
        const double psi0 = legendre_even_series(d, 0.0);
        if (a_out)
            for (int x = 0; x < L; ++x) a_out[x] = legendre_even_series(d, 2.0 * ((double)x - L / 2) / (double)L) / psi0;
        if (eps_out) {
            // F psi = int_{-1}^{1} e^{i c x t} psi(t) dt has psi_0 as eigenfunction with
            // mu_0 = (int psi_0) / psi_0(0) = sqrt(2) d_0 / psi_0(0); the time-frequency
            // limiting operator is (c / 2 pi) F*F, so lambda_0 = c mu_0^2 / (2 pi)
            const double mu0 = std::sqrt(2.0) * d[0] / psi0;
            const double lam0 = c * mu0 * mu0 / (2.0 * kPi);
            *eps_out = std::sqrt(std::fmax(1.0 - lam0, 0.0));
        }
        return IDG_OK;
    }
    if (kind == IDG_TAPER_IDG_OPTIMAL) {
        std::vector<double> R = rbar(L, beta), w, V;
        jacobi_eigh(L, R, w, V);
        int imin = 0;
        double wmax = 0.0;
        for (int i = 0; i < L; ++i) {
            if (w[i] < w[imin]) imin = i;
            wmax = std::fmax(wmax, std::fabs(w[i]));
        }
        // below this the smallest eigenvalue, and so the window, is not determined in FP64
        // (eps below about 1e-7 of the largest eigenvalue's square root; beta >~ 12)
        if (!(w[imin] >= 1e-14 * wmax))
            return fail(IDG_ERR_UNSUPPORTED, "the optimal window is below FP64 resolution for this beta (eps < ~1e-7)");
        if (a_out) {
            const double centre = V[(size_t)(L / 2) * L + imin];
            if (centre == 0.0) return fail(IDG_ERR_INVALID_ARG, "degenerate window (zero at the centre)");
            for (int x = 0; x < L; ++x) a_out[x] = V[(size_t)x * L + imin] / centre;
        }
        if (eps_out) *eps_out = std::sqrt(std::fmax(w[imin], 0.0));
        return IDG_OK;
    }
    return fail(IDG_ERR_INVALID_ARG, "unknown window kind");
}

idg_status idg_taper_aliasing(int L, double beta, const double *a, double *eps_out) {
    idg_status st = check_args(L, beta);
    if (st != IDG_OK) return st;
    if (!a || !eps_out) return fail(IDG_ERR_INVALID_ARG, "a and eps_out are required");
    const std::vector<double> R = rbar(L, beta);
    double num = 0.0, den = 0.0;
    for (int k = 0; k < L; ++k) {
        den += a[k] * a[k];
        for (int l = 0; l < L; ++l) num += a[k] * R[(size_t)k * L + l] * a[l];
    }
    if (!(den > 0.0)) return fail(IDG_ERR_INVALID_ARG, "the window is zero");
    *eps_out = std::sqrt(std::fmax(num / den, 0.0));
    return IDG_OK;
}

}  // extern "C"
