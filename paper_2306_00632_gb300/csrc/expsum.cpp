// Best exponential sums for 1/lambda on [1, M] (Prop. 1, eq. estimate_approx_diag) and the preconditioner
// rank R_P = min{R : E_R(M_P) <= eps_prec / M_P} of eq. estimate_prec_rel, on the host.
//
// The paper reads omega_j, alpha_j from published tables. Here they are computed:
//  - the best R-term sum in the maximum norm is unique and its error equioscillates at 2R + 1 points
//    (alternation theorem for exponential sums, Braess, Nonlinear Approximation Theory, 1986);
//  - Remez exchange: the levelled equations 1/x_i - s(x_i) = sign_i E at 2R + 1 trial points are solved by
//    Newton's method in (log alpha, log omega, E), and the trial points move to the alternating extrema of
//    the new error until the largest error equals |E|;
//  - the start: a weighted least-squares fit on a log grid, reweighted towards the maximum norm (Lawson),
//    solved by Levenberg-Marquardt with Householder QR of the damped system (the Jacobians of exponential
//    sums are too ill-conditioned for normal equations); R - 1 -> R by stretching the log alpha / log omega
//    profile over the term index.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tpcg.h"
#include "setup.h"

namespace tpcg {

void set_error(const std::string& msg);

namespace {

using Vec = std::vector<double>;

// min ||A x - b|| for a column-major m x n A (m >= n), by Householder QR; A and b are overwritten
bool lstsq_qr(Vec& A, Vec& b, int m, int n, Vec& x) {
    for (int k = 0; k < n; ++k) {
        double* a = &A[(size_t)k * m];
        double nrm = 0;
        for (int i = k; i < m; ++i) nrm += a[i] * a[i];
        nrm = sqrt(nrm);
        if (nrm == 0.0) return false;
        const double alpha = a[k] > 0 ? -nrm : nrm;
        a[k] -= alpha;   // v = a_k.. - alpha e_k, stored in place
        double vv = 0;
        for (int i = k; i < m; ++i) vv += a[i] * a[i];
        if (vv == 0.0) return false;
        for (int j = k + 1; j < n; ++j) {
            double* c = &A[(size_t)j * m];
            double d = 0;
            for (int i = k; i < m; ++i) d += a[i] * c[i];
            d = 2.0 * d / vv;
            for (int i = k; i < m; ++i) c[i] -= d * a[i];
        }
        double d = 0;
        for (int i = k; i < m; ++i) d += a[i] * b[i];
        d = 2.0 * d / vv;
        for (int i = k; i < m; ++i) b[i] -= d * a[i];
        a[k] = alpha;    // R_kk; the rest of column k below the diagonal is no longer needed
    }
    x.assign(n, 0.0);
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[(size_t)j * m + k] * x[j];
        const double rkk = A[(size_t)k * m + k];
        if (rkk == 0.0 || !std::isfinite(rkk)) return false;
        x[k] = s / rkk;
    }
    for (double v : x)
        if (!std::isfinite(v)) return false;
    return true;
}

double err_at(double x, const Vec& om, const Vec& al) {
    double s = 0;
    for (size_t j = 0; j < al.size(); ++j) s += om[j] * exp(-al[j] * x);
    return 1.0 / x - s;
}

Vec log_grid(double M, int npts) {
    Vec x(npts);
    const double L = log(M);
    for (int i = 0; i < npts; ++i) x[i] = exp(L * i / (npts - 1));
    return x;
}

// alternating extrema of the error on a fine log grid (same-sign neighbours merged into the larger);
// returns the largest |error| on the grid
double alternants(double M, const Vec& om, const Vec& al, Vec& pts, Vec& ev, int npts = 60000) {
    const Vec x = log_grid(M, npts);
    Vec e(npts);
    double emax = 0;
    for (int i = 0; i < npts; ++i) {
        e[i] = err_at(x[i], om, al);
        emax = std::max(emax, fabs(e[i]));
    }
    std::vector<int> keep;
    auto push = [&](int i) {
        if (!keep.empty() && ((e[i] > 0) == (e[keep.back()] > 0))) {
            if (fabs(e[i]) > fabs(e[keep.back()])) keep.back() = i;
        } else {
            keep.push_back(i);
        }
    };
    push(0);
    for (int i = 1; i < npts - 1; ++i)
        if ((e[i] - e[i - 1]) * (e[i + 1] - e[i]) <= 0) push(i);
    push(npts - 1);
    pts.clear();
    ev.clear();
    for (int i : keep) {
        pts.push_back(x[i]);
        ev.push_back(e[i]);
    }
    return emax;
}

// Newton's method for 1/x_i - s(x_i) = sign_i E in (log alpha, log omega, E), step halving on the residual
void solve_levelled(const Vec& pts, Vec& om, Vec& al, double& E) {
    const int R = (int)al.size(), n = 2 * R + 1;
    Vec sign(n);
    const double s0 = err_at(pts[0], om, al) >= 0 ? 1.0 : -1.0;
    for (int i = 0; i < n; ++i) sign[i] = (i % 2 ? -s0 : s0);
    Vec u(n);
    for (int j = 0; j < R; ++j) { u[j] = log(al[j]); u[R + j] = log(om[j]); }
    u[2 * R] = fabs(E);
    auto resid = [&](const Vec& v, Vec& f) {
        f.resize(n);
        double nrm = 0;
        for (int i = 0; i < n; ++i) {
            double s = 0;
            for (int j = 0; j < R; ++j) s += exp(v[R + j] - exp(v[j]) * pts[i]);
            f[i] = 1.0 / pts[i] - s - sign[i] * v[2 * R];
            nrm += f[i] * f[i];
        }
        return sqrt(nrm);
    };
    Vec f, f2, J((size_t)n * n), du, v(n);
    for (int it = 0; it < 80; ++it) {
        const double f0 = resid(u, f);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < R; ++j) {
                const double a = exp(u[j]), t = exp(u[R + j] - a * pts[i]);   // omega_j exp(-alpha_j x_i)
                J[(size_t)j * n + i] = t * a * pts[i];
                J[(size_t)(R + j) * n + i] = -t;
            }
            J[(size_t)(2 * R) * n + i] = -sign[i];
        }
        Vec rhs(n);
        for (int i = 0; i < n; ++i) rhs[i] = -f[i];
        Vec Jc = J;
        if (!lstsq_qr(Jc, rhs, n, n, du)) break;
        double step = 1.0;
        while (step > 1e-6) {
            for (int i = 0; i < n; ++i) v[i] = u[i] + step * du[i];
            const double f1 = resid(v, f2);
            if (f1 < f0 && std::isfinite(f1)) break;
            step *= 0.5;
        }
        double dn = 0, un = 0;
        for (int i = 0; i < n; ++i) {
            u[i] += step * du[i];
            dn += step * step * du[i] * du[i];
            un += u[i] * u[i];
        }
        if (sqrt(dn) < 1e-14 * (1.0 + sqrt(un))) break;
    }
    for (int j = 0; j < R; ++j) { al[j] = exp(u[j]); om[j] = exp(u[R + j]); }
    E = u[2 * R];
}

// Remez exchange; returns the largest error on the grid and whether it equals the levelled |E|
double remez(double M, Vec& om, Vec& al, bool* ok) {
    const int R = (int)al.size();
    Vec pts, ev;
    double E = -1, emax = 1e300;
    *ok = false;
    for (int it = 0; it < 60; ++it) {
        emax = alternants(M, om, al, pts, ev);
        if ((int)pts.size() < 2 * R + 1) return emax;
        int lo = 0, hi = (int)pts.size();
        while (hi - lo > 2 * R + 1) {
            if (fabs(ev[lo]) < fabs(ev[hi - 1])) ++lo; else --hi;
        }
        Vec p(pts.begin() + lo, pts.begin() + hi);
        if (E < 0) {
            E = 0;
            for (int i = lo; i < hi; ++i) E += fabs(ev[i]);
            E /= (hi - lo);
        }
        solve_levelled(p, om, al, E);
        emax = alternants(M, om, al, pts, ev);
        if (emax <= fabs(E) * (1.0 + 1e-8)) {
            *ok = true;
            return emax;
        }
    }
    return emax;
}

// weighted least squares on a log grid, Lawson reweighting, Levenberg-Marquardt with QR and box clipping
void least_squares_start(double M, Vec& om, Vec& al, int npts = 800, int lawson = 2) {
    const int R = (int)al.size(), n = 2 * R;
    const Vec x = log_grid(M, npts);
    Vec w(npts, 1.0), u(n), lo(n), hi(n);
    for (int j = 0; j < R; ++j) {
        lo[j] = log(0.01 / M); hi[j] = log(200.0);
        lo[R + j] = -40.0; hi[R + j] = 10.0;
        u[j] = std::min(std::max(log(al[j]), lo[j] + 1e-9), hi[j] - 1e-9);
        u[R + j] = std::min(std::max(log(om[j]), lo[R + j] + 1e-9), hi[R + j] - 1e-9);
    }
    auto resid = [&](const Vec& v, Vec& r) {
        r.resize(npts);
        double s2 = 0;
        for (int i = 0; i < npts; ++i) {
            double s = 0;
            for (int j = 0; j < R; ++j) s += exp(v[R + j] - exp(v[j]) * x[i]);
            r[i] = w[i] * (1.0 / x[i] - s);
            s2 += r[i] * r[i];
        }
        return s2;
    };
    Vec r, r2, v(n), A, b, d;
    for (int round = 0; round <= lawson; ++round) {
        double lam = 1e-3;
        double c0 = resid(u, r);
        for (int it = 0; it < 300; ++it) {
            const int m = npts + n;
            A.assign((size_t)m * n, 0.0);
            b.assign(m, 0.0);
            for (int i = 0; i < npts; ++i) {
                for (int j = 0; j < R; ++j) {
                    const double a = exp(u[j]), t = exp(u[R + j] - a * x[i]);
                    A[(size_t)j * m + i] = w[i] * t * a * x[i];
                    A[(size_t)(R + j) * m + i] = -w[i] * t;
                }
                b[i] = -r[i];
            }
            const double sl = sqrt(lam);
            for (int j = 0; j < n; ++j) A[(size_t)j * m + npts + j] = sl;
            bool accepted = false;
            if (lstsq_qr(A, b, m, n, d)) {
                for (int j = 0; j < n; ++j) v[j] = std::min(std::max(u[j] + d[j], lo[j]), hi[j]);
                const double c1 = resid(v, r2);
                if (c1 < c0 && std::isfinite(c1)) {
                    const double rel = (c0 - c1) / c0;
                    u = v;
                    r = r2;
                    c0 = c1;
                    lam = std::max(lam / 3.0, 1e-12);
                    accepted = true;
                    if (rel < 1e-12) break;
                }
            }
            if (!accepted) {
                lam *= 4.0;
                if (lam > 1e12) break;
            }
        }
        // reweight towards the maximum norm: w <- w sqrt|e|, normalised, floored
        double wm = 0;
        for (int i = 0; i < npts; ++i) {
            const double e = r[i] / w[i];
            w[i] *= sqrt(fabs(e));
            wm = std::max(wm, w[i]);
        }
        for (int i = 0; i < npts; ++i) w[i] = std::max(w[i] / wm, 1e-3);
        c0 = resid(u, r);
    }
    for (int j = 0; j < R; ++j) { al[j] = exp(u[j]); om[j] = exp(u[R + j]); }
}

// R -> R + 1 terms: log alpha and log omega, sorted by alpha, interpolated over the term index
void stretch(Vec& om, Vec& al) {
    const int R = (int)al.size();
    std::vector<int> o(R);
    for (int j = 0; j < R; ++j) o[j] = j;
    std::sort(o.begin(), o.end(), [&](int a, int b) { return al[a] < al[b]; });
    Vec la(R), lw(R);
    for (int j = 0; j < R; ++j) { la[j] = log(al[o[j]]); lw[j] = log(om[o[j]]); }
    Vec na(R + 1), nw(R + 1);
    for (int k = 0; k <= R; ++k) {
        const double t = (R == 1) ? 0.0 : (double)k * (R - 1) / R;
        const int i0 = std::min((int)t, R - 1), i1 = std::min(i0 + 1, R - 1);
        const double f = t - i0;
        na[k] = exp(la[i0] + f * (la[i1] - la[i0]));
        nw[k] = exp(lw[i0] + f * (lw[i1] - lw[i0]));
    }
    al = na;
    om = nw;
}

}  // namespace

static int expsum_best_compute(double M, double eps_prec, int rmax, std::vector<double>* omega,
                               std::vector<double>* alpha, double* E_out) {
    if (!(M >= 1.0) || !(eps_prec > 0.0) || rmax < 1) return -1;
    Vec om{0.5}, al{0.5};
    for (int R = 1; R <= rmax; ++R) {
        if (R > 1) stretch(om, al);
        least_squares_start(M, om, al);
        bool ok = false;
        const double E = remez(M, om, al, &ok);   // E is the largest error on the grid either way
        if (E <= eps_prec / M) {
            *omega = om;
            *alpha = al;
            if (E_out) *E_out = E;
            return R;
        }
    }
    return -1;
}

// M_P depends only on n, p and the direction weights, not on the geometry, so many setups share it: results
// are kept per (M, eps_prec, rmax) for the life of the process (at most 256 entries)
int expsum_best(double M, double eps_prec, int rmax, std::vector<double>* omega, std::vector<double>* alpha,
                double* E_out) {
    using Key = std::tuple<double, double, int>;
    struct Entry {
        int R;
        Vec om, al;
        double E;
    };
    static std::mutex mu;
    static std::map<Key, Entry> cache;
    const Key key{M, eps_prec, rmax};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *omega = it->second.om;
            *alpha = it->second.al;
            if (E_out) *E_out = it->second.E;
            return it->second.R;
        }
    }
    double E = 0;
    const int R = expsum_best_compute(M, eps_prec, rmax, omega, alpha, &E);
    if (E_out) *E_out = E;
    if (R > 0) {
        std::lock_guard<std::mutex> lock(mu);
        if (cache.size() >= 256) cache.clear();
        cache[key] = Entry{R, *omega, *alpha, E};
    }
    return R;
}

}  // namespace tpcg

extern "C" int tpcg_expsum_best(double M, double eps_prec, int rmax, double* omega, double* alpha, int* R_out,
                                double* E_out) {
    if (!omega || !alpha || !R_out || rmax < 1) {
        tpcg::set_error("tpcg_expsum_best: null output or rmax < 1");
        return TPCG_E_INVALID;
    }
    std::vector<double> om, al;
    double E = 0;
    const int R = tpcg::expsum_best(M, eps_prec, rmax, &om, &al, &E);
    if (R < 1) {
        tpcg::set_error("tpcg_expsum_best: no best sum with R <= rmax meets E_R(M) <= eps_prec / M (or M < 1)");
        return TPCG_E_INVALID;
    }
    for (int j = 0; j < R; ++j) { omega[j] = om[j]; alpha[j] = al[j]; }
    *R_out = R;
    if (E_out) *E_out = E;
    return TPCG_OK;
}
