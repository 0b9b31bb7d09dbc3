// Host FP64 setup (untimed): B-spline matrices (Sec. 2.1-2.2), low-rank Chebyshev approximation of the
// parametric coefficients folded into a Kronecker sum (App. A), Tucker rhs (App. A), approximate
// eigenpairs of the univariate pencils (App. B), exponential sums and R_P (Prop. 1, eq. estimate_prec_rel).
#include "setup.h"

#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/tpcg.h"

namespace tpcg {

void set_error(const std::string& msg);

namespace {

using Vec = std::vector<double>;

// ---------------------------------------------------------------------------------------------- dense helpers
// column-major n x m matrices
struct Mat {
    int r = 0, c = 0;
    Vec a;
    Mat() = default;
    Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, 0.0) {}
    double& operator()(int i, int j) { return a[i + (size_t)j * r]; }
    double operator()(int i, int j) const { return a[i + (size_t)j * r]; }
};

Mat matmul(const Mat& A, const Mat& B, bool ta = false, bool tb = false) {
    const int m = ta ? A.c : A.r, k = ta ? A.r : A.c, nn = tb ? B.r : B.c;
    Mat C(m, nn);
    for (int j = 0; j < nn; ++j)
        for (int q = 0; q < k; ++q) {
            const double b = tb ? B(j, q) : B(q, j);
            if (b == 0.0) continue;
            for (int i = 0; i < m; ++i) C(i, j) += (ta ? A(q, i) : A(i, q)) * b;
        }
    return C;
}

// solve A X = B by LU with partial pivoting (A square, overwritten copy)
bool lu_solve(Mat A, Mat& B) {
    const int n = A.r;
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int pk = k;
        double mx = fabs(A(k, k));
        for (int i = k + 1; i < n; ++i)
            if (fabs(A(i, k)) > mx) { mx = fabs(A(i, k)); pk = i; }
        if (mx == 0.0) return false;
        piv[k] = pk;
        if (pk != k) {
            for (int j = 0; j < n; ++j) std::swap(A(k, j), A(pk, j));
            for (int j = 0; j < B.c; ++j) std::swap(B(k, j), B(pk, j));
        }
        for (int i = k + 1; i < n; ++i) {
            const double l = A(i, k) / A(k, k);
            A(i, k) = l;
            if (l == 0.0) continue;
            for (int j = k + 1; j < n; ++j) A(i, j) -= l * A(k, j);
            for (int j = 0; j < B.c; ++j) B(i, j) -= l * B(k, j);
        }
    }
    for (int j = 0; j < B.c; ++j)
        for (int i = n - 1; i >= 0; --i) {
            double s = B(i, j);
            for (int q = i + 1; q < n; ++q) s -= A(i, q) * B(q, j);
            B(i, j) = s / A(i, i);
        }
    return true;
}

// cyclic Jacobi for a symmetric matrix: A = V diag(d) V^T, eigenvalues ascending
void sym_eig(Mat A, Vec* d, Mat* V) {
    const int n = A.r;
    Mat v(n, n);
    for (int i = 0; i < n; ++i) v(i, i) = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                tot += A(i, j) * A(i, j);
                if (i != j) off += A(i, j) * A(i, j);
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A(p, q);
                if (apq == 0.0) continue;
                const double th = (A(q, q) - A(p, p)) / (2 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1));
                const double c = 1 / sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A(k, p), akq = A(k, q);
                    A(k, p) = c * akp - s * akq;
                    A(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A(p, k), aqk = A(q, k);
                    A(p, k) = c * apk - s * aqk;
                    A(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v(k, p), vkq = v(k, q);
                    v(k, p) = c * vkp - s * vkq;
                    v(k, q) = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A(a, a) < A(b, b); });
    d->assign(n, 0.0);
    *V = Mat(n, n);
    for (int j = 0; j < n; ++j) {
        (*d)[j] = A(idx[j], idx[j]);
        for (int i = 0; i < n; ++i) (*V)(i, j) = v(i, idx[j]);
    }
}

// one-sided Jacobi on the rows of A (m x N): A = U diag(s) V^T; returns U (m x m) and s sorted descending
void left_svd(Mat A, Vec* s, Mat* U) {
    const int m = A.r, N = A.c;
    Mat J(m, m);
    for (int i = 0; i < m; ++i) J(i, i) = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        bool rotated = false;
        for (int i = 0; i < m - 1; ++i)
            for (int j = i + 1; j < m; ++j) {
                double a = 0, b = 0, g = 0;
                for (int q = 0; q < N; ++q) {
                    a += A(i, q) * A(i, q);
                    b += A(j, q) * A(j, q);
                    g += A(i, q) * A(j, q);
                }
                if (fabs(g) <= 1e-15 * sqrt(a * b) || g == 0.0) continue;
                rotated = true;
                const double zeta = (b - a) / (2 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1 + zeta * zeta));
                const double c = 1 / sqrt(1 + t * t), sn = c * t;
                for (int q = 0; q < N; ++q) {
                    const double x = A(i, q), y = A(j, q);
                    A(i, q) = c * x - sn * y;
                    A(j, q) = sn * x + c * y;
                }
                for (int q = 0; q < m; ++q) {
                    const double x = J(q, i), y = J(q, j);
                    J(q, i) = c * x - sn * y;
                    J(q, j) = sn * x + c * y;
                }
            }
        if (!rotated) break;
    }
    Vec nr(m);
    for (int i = 0; i < m; ++i) {
        double a = 0;
        for (int q = 0; q < N; ++q) a += A(i, q) * A(i, q);
        nr[i] = sqrt(a);
    }
    std::vector<int> idx(m);
    for (int i = 0; i < m; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return nr[a] > nr[b]; });
    s->assign(m, 0.0);
    *U = Mat(m, m);
    for (int j = 0; j < m; ++j) {
        (*s)[j] = nr[idx[j]];
        for (int q = 0; q < m; ++q) (*U)(q, j) = J(q, idx[j]);
    }
}

// ---------------------------------------------------------------------------------------------- tensors
struct Ten {
    int d[3] = {0, 0, 0};
    Vec a;
    double& at(int i, int j, int k) { return a[i + (size_t)d[0] * (j + (size_t)d[1] * k)]; }
    double at(int i, int j, int k) const { return a[i + (size_t)d[0] * (j + (size_t)d[1] * k)]; }
};

Mat unfold(const Ten& T, int m) {
    const int o1 = (m + 1) % 3, o2 = (m + 2) % 3;
    Mat U(T.d[m], T.d[o1] * T.d[o2]);
    for (int k = 0; k < T.d[2]; ++k)
        for (int j = 0; j < T.d[1]; ++j)
            for (int i = 0; i < T.d[0]; ++i) {
                int id[3] = {i, j, k};
                U(id[m], id[o1] + T.d[o1] * id[o2]) = T.at(i, j, k);
            }
    return U;
}

// T x_m A^T with A (d_m x s): result dim m becomes s
Ten project(const Ten& T, int m, const Mat& A) {
    Ten R;
    for (int t = 0; t < 3; ++t) R.d[t] = T.d[t];
    R.d[m] = A.c;
    R.a.assign((size_t)R.d[0] * R.d[1] * R.d[2], 0.0);
    for (int k = 0; k < T.d[2]; ++k)
        for (int j = 0; j < T.d[1]; ++j)
            for (int i = 0; i < T.d[0]; ++i) {
                int id[3] = {i, j, k};
                const double v = T.at(i, j, k);
                for (int c = 0; c < A.c; ++c) {
                    int od[3] = {i, j, k};
                    od[m] = c;
                    R.at(od[0], od[1], od[2]) += A(id[m], c) * v;
                }
            }
    return R;
}

// ST-HOSVD with the per-mode budget eps^2 ||T||^2 / 3
void sthosvd(Ten T, double eps, Ten* core, Mat S[3]) {
    double nrm2 = 0;
    for (double v : T.a) nrm2 += v * v;
    const double budget = eps * eps * nrm2 / 3.0;
    for (int m = 0; m < 3; ++m) {
        Vec s;
        Mat U;
        left_svd(unfold(T, m), &s, &U);
        const int dm = T.d[m];
        double tail = 0;
        int keep = dm;
        for (int i = dm - 1; i >= 0; --i) {
            if (tail + s[i] * s[i] <= budget) { tail += s[i] * s[i]; keep = i; } else break;
        }
        if (keep == 0 && nrm2 > 0) keep = 1;
        Mat Sm(dm, keep);
        for (int c = 0; c < keep; ++c)
            for (int i = 0; i < dm; ++i) Sm(i, c) = U(i, c);
        S[m] = Sm;
        T = project(T, m, Sm);
    }
    *core = T;
}

// ---------------------------------------------------------------------------------------------- B-splines
struct Spline {
    int p, n_el, m;   // degree, spans, basis size (m = n_el + p)
    Vec knots;
    Spline(int p_, int ne) : p(p_), n_el(ne), m(ne + p_) {
        knots.assign(p + 1, 0.0);
        for (int i = 1; i < n_el; ++i) knots.push_back((double)i / n_el);
        for (int i = 0; i <= p; ++i) knots.push_back(1.0);
    }
    int span(double x) const {
        int s = p + (int)floor(x * n_el);
        if (s > p + n_el - 1) s = p + n_el - 1;
        if (s < p) s = p;
        return s;
    }
    // derivatives 0..nd of the p+1 non-zero functions N_{s-p..s} at x (de Boor's triangular table)
    void ders(int s, double x, int nd, std::vector<Vec>* out) const {
        const Vec& U = knots;
        std::vector<Vec> ndu(p + 1, Vec(p + 1, 0.0));
        Vec left(p + 1), right(p + 1);
        ndu[0][0] = 1.0;
        for (int j = 1; j <= p; ++j) {
            left[j] = x - U[s + 1 - j];
            right[j] = U[s + j] - x;
            double saved = 0.0;
            for (int r = 0; r < j; ++r) {
                ndu[j][r] = right[r + 1] + left[j - r];
                const double tmp = ndu[r][j - 1] / ndu[j][r];
                ndu[r][j] = saved + right[r + 1] * tmp;
                saved = left[j - r] * tmp;
            }
            ndu[j][j] = saved;
        }
        out->assign(nd + 1, Vec(p + 1, 0.0));
        for (int j = 0; j <= p; ++j) (*out)[0][j] = ndu[j][p];
        std::vector<Vec> a(2, Vec(p + 1, 0.0));
        for (int r = 0; r <= p; ++r) {
            int s1 = 0, s2 = 1;
            a[0][0] = 1.0;
            for (int k = 1; k <= nd; ++k) {
                double d = 0.0;
                const int rk = r - k, pk = p - k;
                if (pk < 0) { (*out)[k][r] = 0.0; continue; }
                if (r >= k) {
                    a[s2][0] = a[s1][0] / ndu[pk + 1][rk];
                    d = a[s2][0] * ndu[rk][pk];
                }
                const int j1 = (rk >= -1) ? 1 : -rk;
                const int j2 = (r - 1 <= pk) ? k - 1 : p - r;
                for (int j = j1; j <= j2; ++j) {
                    a[s2][j] = (a[s1][j] - a[s1][j - 1]) / ndu[pk + 1][rk + j];
                    d += a[s2][j] * ndu[rk + j][pk];
                }
                if (r <= pk) {
                    a[s2][k] = -a[s1][k - 1] / ndu[pk + 1][r];
                    d += a[s2][k] * ndu[r][pk];
                }
                (*out)[k][r] = d;
                std::swap(s1, s2);
            }
        }
        double f = p;
        for (int k = 1; k <= nd; ++k) {
            for (int j = 0; j <= p; ++j) (*out)[k][j] *= f;
            f *= (p - k);
        }
    }
};

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_q
void gauss_legendre(int q, Vec* x, Vec* w) {
    x->assign(q, 0.0);
    w->assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double z = cos(M_PI * (i + 0.75) / (q + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) { p1 = z; p0 = 1.0; }
            dp = q * (z * p1 - p0) / (z * z - 1);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= q; ++k) {
            const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1);
        (*x)[q - 1 - i] = z;
        (*w)[q - 1 - i] = 2.0 / ((1 - z * z) * dp * dp);
    }
}

// quadrature on all spans: points, weights, and the p+1 non-zero values/derivatives.  The space drops the end
// function of every Dirichlet end (k = 0) and keeps that of every Neumann end (k = 1): n = m - 2 + k0 + k1.
struct Quad {
    int q = 0, n_el = 0, p = 0, n = 0, k0 = 0, k1 = 0;
    Vec x, w;                     // n_el * q
    std::vector<int> first;       // reduced index of the first local function (may be -1)
    std::vector<Vec> val, der;    // [pt][0..p]
};

Quad make_quad(const Spline& sp, int k0 = 0, int k1 = 0) {
    Quad Q;
    Q.p = sp.p;
    Q.n_el = sp.n_el;
    Q.k0 = k0;
    Q.k1 = k1;
    Q.n = sp.m - 2 + k0 + k1;
    Q.q = sp.p + 3;
    Vec gx, gw;
    gauss_legendre(Q.q, &gx, &gw);
    const double h = 1.0 / sp.n_el;
    for (int e = 0; e < sp.n_el; ++e)
        for (int k = 0; k < Q.q; ++k) {
            const double xx = (e + 0.5 * (gx[k] + 1.0)) * h;
            Q.x.push_back(xx);
            Q.w.push_back(0.5 * h * gw[k]);
            const int s = sp.p + e;
            std::vector<Vec> d;
            sp.ders(s, xx, 1, &d);
            Q.val.push_back(d[0]);
            Q.der.push_back(d[1]);
            Q.first.push_back(s - sp.p - 1 + k0);
        }
    return Q;
}

// banded C[i, j] = int delta_i(b_i) delta_j(b_j) g  -> band[d*n + i] = C[i, i + d - p]
void weighted_band(const Quad& Q, bool di, bool dj, const Vec& g, double* band) {
    const int n = Q.n, p = Q.p;
    std::fill(band, band + (size_t)(2 * p + 1) * n, 0.0);
    for (size_t k = 0; k < Q.x.size(); ++k) {
        const double wg = Q.w[k] * (g.empty() ? 1.0 : g[k]);
        const Vec& vi = di ? Q.der[k] : Q.val[k];
        const Vec& vj = dj ? Q.der[k] : Q.val[k];
        for (int a = 0; a <= p; ++a) {
            const int i = Q.first[k] + a;
            if (i < 0 || i >= n) continue;
            for (int b = 0; b <= p; ++b) {
                const int j = Q.first[k] + b;
                if (j < 0 || j >= n) continue;
                band[(size_t)(j - i + p) * n + i] += wg * vi[a] * vj[b];
            }
        }
    }
}

Mat band_to_dense(const double* band, int n, int p) {
    Mat A(n, n);
    for (int d = 0; d <= 2 * p; ++d)
        for (int i = 0; i < n; ++i) {
            const int j = i + d - p;
            if (j >= 0 && j < n) A(i, j) = band[(size_t)d * n + i];
        }
    return A;
}

// ---------------------------------------------------------------------------------------------- geometry
const double CENTROID = 28.0 / (9.0 * M_PI);

// G = J^-1 and det J of the map at a parametric point (J[a][b] = dF_a / d eta_b)
void inverse_jacobian(int kind, double amp, double e1, double e2, double e3, double Ji[3][3], double* detJ) {
    if (kind == TPCG_GEOM_CUBE) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Ji[a][b] = (a == b) ? 1.0 : 0.0;
        *detJ = 1.0;
        return;
    }
    const double rho = 1 + e1, th = 0.5 * M_PI * e2;
    const double tau = amp * sin(M_PI * e3), dtau = amp * M_PI * cos(M_PI * e3);
    const double c = cos(tau), s = sin(tau);
    const double px = rho * cos(th) - CENTROID, py = rho * sin(th) - CENTROID;
    const double d1x = cos(th), d1y = sin(th);
    const double d2x = -0.5 * M_PI * rho * sin(th), d2y = 0.5 * M_PI * rho * cos(th);
    double J[3][3] = {{c * d1x - s * d1y, c * d2x - s * d2y, dtau * (-s * px - c * py)},
                      {s * d1x + c * d1y, s * d2x + c * d2y, dtau * (c * px - s * py)},
                      {0, 0, 1}};
    // inverse by cofactors
    double C[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            C[a][b] = J[a1][b1] * J[a2][b2] - J[a1][b2] * J[a2][b1];
        }
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Ji[a][b] = C[b][a] / det;
    *detJ = det;
}

// Poisson: Q = det J J^-1 J^-T and omega = det J f (App. A).  The cube's f makes u = s(x) s(y) s(z) the solution,
// s(t) = sin(w t + k0 pi/2), w = (1 - k0/2 - k1/2) pi (zero at Dirichlet faces, zero slope at Neumann faces).
void coefficients(int kind, double amp, double e1, double e2, double e3, double Q[3][3], double* om, int k0 = 0,
                  int k1 = 0) {
    double Ji[3][3], det;
    inverse_jacobian(kind, amp, e1, e2, e3, Ji, &det);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += Ji[a][k] * Ji[b][k];
            Q[a][b] = det * v;
        }
    if (kind == TPCG_GEOM_CUBE) {
        const double w = (1.0 - 0.5 * (k0 + k1)) * M_PI, ph = 0.5 * M_PI * k0;
        *om = 3 * w * w * sin(w * e1 + ph) * sin(w * e2 + ph) * sin(w * e3 + ph);
    } else
        *om = det * 1.0;
}

// Elasticity (Sec. 5.3), trial phi e_j with derivative k, test psi e_i with derivative l:
// C[i][j][k][l] = det [mu delta_ij (G G^T)_kl + mu G_ki G_lj + lambda G_kj G_li], G = J^-1
void elast_coefficients(int kind, double amp, double lam, double mu, double e1, double e2, double e3,
                        double Cc[3][3][3][3], double* detJ) {
    double G[3][3], det;
    inverse_jacobian(kind, amp, e1, e2, e3, G, &det);
    double GGt[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0;
            for (int q = 0; q < 3; ++q) v += G[a][q] * G[b][q];
            GGt[a][b] = v;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    Cc[i][j][k][l] = det * (mu * (i == j ? 1.0 : 0.0) * GGt[k][l] + mu * G[k][i] * G[l][j] +
                                            lam * G[k][j] * G[l][i]);
    *detJ = det;
}

// ---------------------------------------------------------------------------------------------- Chebyshev
const int NCHEB = 33;

double cheb_pt(int k) { return 0.5 * (1.0 - cos(M_PI * k / (NCHEB - 1))); }

// barycentric interpolation (second-kind points) of the columns of F (NCHEB x c) at x
void cheb_interp(const Mat& F, const Vec& x, Mat* out) {
    *out = Mat((int)x.size(), F.c);
    Vec wb(NCHEB), xc(NCHEB);
    for (int k = 0; k < NCHEB; ++k) {
        xc[k] = cheb_pt(k);
        wb[k] = ((k % 2) ? -1.0 : 1.0) * ((k == 0 || k == NCHEB - 1) ? 0.5 : 1.0);
    }
    for (size_t q = 0; q < x.size(); ++q) {
        int hit = -1;
        for (int k = 0; k < NCHEB; ++k)
            if (x[q] == xc[k]) hit = k;
        for (int c = 0; c < F.c; ++c) {
            if (hit >= 0) { (*out)((int)q, c) = F(hit, c); continue; }
            double num = 0, den = 0;
            for (int k = 0; k < NCHEB; ++k) {
                const double t = wb[k] / (x[q] - xc[k]);
                num += t * F(k, c);
                den += t;
            }
            (*out)((int)q, c) = num / den;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------- exp sums
double expsum_error(const double* omega, const double* alpha, int R, double M, int npts) {
    double e = 0;
    for (int i = 0; i < npts; ++i) {
        const double lam = exp(log(M) * i / (npts - 1));
        double s = 0;
        for (int j = 0; j < R; ++j) s += omega[j] * exp(-alpha[j] * lam);
        e = std::max(e, fabs(1.0 / lam - s));
    }
    return e;
}

// Sinc-quadrature sums of 1/lambda = int exp(s - lambda e^s) ds, nodes s0 + k h: the smallest R (with a
// search over (h, s0)) whose error meets E_R(M) <= eps_prec / M on a log grid of [1, M].
int expsum_sinc(double M, double eps_prec, std::vector<double>* omega, std::vector<double>* alpha) {
    const double target = eps_prec / M;
    const double top0 = log(log(1.0 / target) + 2.0) + 0.5;
    std::vector<double> om, al;
    for (int R = 1; R <= 120; ++R) {
        double best = 1e300, bh = 0, bs = 0;
        for (int ih = 0; ih < 30; ++ih) {
            const double h = 0.15 + (1.6 - 0.15) * ih / 29.0;
            for (int is = 0; is < 13; ++is) {
                const double s0 = top0 - h * (R - 1) - 2.0 + 3.0 * is / 12.0;
                om.resize(R);
                al.resize(R);
                for (int k = 0; k < R; ++k) {
                    al[k] = exp(s0 + h * k);
                    om[k] = h * al[k];
                }
                const double e = expsum_error(om.data(), al.data(), R, M, 400);
                if (e < best) { best = e; bh = h; bs = s0; }
            }
        }
        if (best <= target) {
            om.resize(R);
            al.resize(R);
            for (int k = 0; k < R; ++k) {
                al[k] = exp(bs + bh * k);
                om[k] = bh * al[k];
            }
            if (expsum_error(om.data(), al.data(), R, M, 4000) <= target) {
                *omega = om;
                *alpha = al;
                return R;
            }
        }
    }
    return -1;
}

// ---------------------------------------------------------------------------------------------- setup
// Kronecker terms of sum_{k,l} int C_kl d_k phi d_l psi: per entry (k, l), ST-HOSVD of the Chebyshev samples,
// fold the largest-rank mode (App. A, eq. matrix_CP); appended to H.w / H.bands
static int terms_from_coeffs(Ten (&Tq)[3][3], double eps_geo, const Quad& Q, int n, int p, HostProblem& H) {
    const int bw = 2 * p + 1;
    double nmax = 0, nrm[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (double v : Tq[a][b].a) s += v * v;
            nrm[a][b] = sqrt(s);
            nmax = std::max(nmax, nrm[a][b]);
        }
    H.w.clear();
    H.bands.clear();
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            if (nrm[k][l] <= 1e-13 * nmax) continue;
            Ten core;
            Mat S[3];
            sthosvd(Tq[k][l], eps_geo, &core, S);
            Mat g[3];
            for (int t = 0; t < 3; ++t) cheb_interp(S[t], Q.x, &g[t]);
            const int Rk[3] = {core.d[0], core.d[1], core.d[2]};
            int ms = 0;
            for (int t = 1; t < 3; ++t)
                if (Rk[t] >= Rk[ms]) ms = t;
            const int o1 = (ms == 0) ? 1 : 0;
            const int o2 = (ms == 2) ? 1 : 2;
            for (int a = 0; a < Rk[o1]; ++a)
                for (int b = 0; b < Rk[o2]; ++b) {
                    Vec fn[3];
                    fn[o1].resize(Q.x.size());
                    fn[o2].resize(Q.x.size());
                    fn[ms].assign(Q.x.size(), 0.0);
                    for (size_t q = 0; q < Q.x.size(); ++q) {
                        fn[o1][q] = g[o1]((int)q, a);
                        fn[o2][q] = g[o2]((int)q, b);
                    }
                    for (int c = 0; c < Rk[ms]; ++c) {
                        int id[3];
                        id[o1] = a;
                        id[o2] = b;
                        id[ms] = c;
                        const double cv = core.at(id[0], id[1], id[2]);
                        for (size_t q = 0; q < Q.x.size(); ++q) fn[ms][q] += cv * g[ms]((int)q, c);
                    }
                    H.w.push_back(1.0);
                    const size_t off = H.bands.size();
                    H.bands.resize(off + (size_t)3 * bw * n);
                    for (int t = 0; t < 3; ++t)
                        weighted_band(Q, t == l, t == k, fn[t], &H.bands[off + (size_t)t * bw * n]);
                }
        }
    H.R = (int)H.w.size();
    if (H.R < 1 || H.R > TPCG_MAX_BLOCKS - 1) {
        set_error("tpcg_setup: operator has " + std::to_string(H.R) + " terms (need 1.." +
                  std::to_string(TPCG_MAX_BLOCKS - 1) + ")");
        return TPCG_E_INVALID;
    }

    return TPCG_OK;
}

// Tucker rhs (App. A): core of the samples' ST-HOSVD times `scale`, factors F_t[i, r] = int b_i u_{t,r}
static void rhs_from_samples(const Ten& Tw, double eps_geo, const Quad& Q, int n, int p, double scale, HostProblem& H) {
    {
        Ten core;
        Mat S[3];
        sthosvd(Tw, eps_geo, &core, S);
        for (int t = 0; t < 3; ++t) {
            Mat g;
            cheb_interp(S[t], Q.x, &g);
            H.rf[t] = core.d[t];
            H.f_U[t].assign((size_t)n * H.rf[t], 0.0);
            for (size_t q = 0; q < Q.x.size(); ++q)
                for (int a = 0; a <= p; ++a) {
                    const int i = Q.first[q] + a;
                    if (i < 0 || i >= n) continue;
                    for (int r = 0; r < H.rf[t]; ++r) H.f_U[t][i + (size_t)r * n] += Q.w[q] * Q.val[q][a] * g((int)q, r);
                }
        }
        H.f_core = core.a;
        for (double& v : H.f_core) v *= scale;
    }

}

// App. B eigenpairs (sparse sine factorization, V2 U2, Lambda~) and the exponential sum of Prop. 1.  The ends
// carry the conditions of Q (k = 0 Dirichlet, 1 Neumann): V_h,1 asks the even derivatives 2, 4, .. <= p - 1 to
// vanish at a Dirichlet end and the odd ones 1, 3, .. <= p - 1 at a Neumann end; an end with c conditions
// contributes the part of the span of its 2c end functions that meets them (c functions) to V1 and the rest
// (c functions) to null(V1^T).  The sinusoids are sin(omega_j x + k0 pi/2), omega_j = (j - k0/2 - k1/2) pi.
static int fd_tables(const Spline& sp, const Quad& Q, int n, int p, double eps_prec, HostProblem& H) {
    const int n_el = sp.n_el, k0 = Q.k0, k1 = Q.k1;
    const int bw = 2 * p + 1;
    int nord[2] = {0, 0}, ord[2][4];
    for (int end = 0; end < 2; ++end)
        for (int d = ((end == 0 ? k0 : k1) == 1 ? 1 : 2); d <= p - 1; d += 2) ord[end][nord[end]++] = d;
    const int c0 = nord[0], c1 = nord[1];
    const int blk[2] = {2 * c0, 2 * c1};   // end functions holding the conditions
    const int n1 = n - c0 - c1;
    const int n2 = c0 + c1;
    H.n1 = n1;
    H.n2 = n2;
    std::vector<double> Mb((size_t)bw * n), Kb((size_t)bw * n);
    weighted_band(Q, false, false, Vec(), Mb.data());
    weighted_band(Q, true, true, Vec(), Kb.data());
    Mat Md = band_to_dense(Mb.data(), n, p), Kd = band_to_dense(Kb.data(), n, p);
    // V1: Phi0 | Phi | Phi1
    Mat V1(n, n1);
    Mat Z[2] = {Mat(blk[0], c0), Mat(blk[1], c1)};
    for (int end = 0; end < 2; ++end) {
        const int c = nord[end], m = blk[end];
        if (c == 0) continue;
        const double xe = end == 0 ? 0.0 : 1.0;
        const int s = sp.span(xe);
        std::vector<Vec> d;
        sp.ders(s, xe, ord[end][c - 1], &d);
        // D (c x m): rows = the end's derivative orders, columns = its m end functions
        Mat D(c, m);
        const int base = end == 0 ? 0 : n - m;   // reduced index of the first end function
        for (int kk = 0; kk < c; ++kk) {
            double sc = 0;
            for (int a = 0; a <= p; ++a) {
                const int i = s - p - 1 + k0 + a;
                if (i >= base && i < base + m) D(kk, i - base) = d[ord[end][kk]][a];
                sc = std::max(sc, fabs(d[ord[end][kk]][a]));
            }
            for (int q = 0; q < m; ++q) D(kk, q) /= sc;
        }
        Vec ev;
        Mat EV;
        sym_eig(matmul(D, D, true, false), &ev, &EV);   // null space: the m - c smallest
        for (int q = 0; q < c; ++q)
            for (int i = 0; i < m; ++i) Z[end](i, q) = EV(i, q);
    }
    for (int q = 0; q < c0; ++q)
        for (int i = 0; i < blk[0]; ++i) V1(i, q) = Z[0](i, q);
    for (int i = blk[0]; i < n - blk[1]; ++i) V1(i, c0 + (i - blk[0])) = 1.0;
    for (int q = 0; q < c1; ++q)
        for (int i = 0; i < blk[1]; ++i) V1(n - blk[1] + i, n1 - c1 + q) = Z[1](i, q);
    // interpolation points (breakpoints without the Dirichlet ends, or span midpoints) and Cint[l, i] = v_i(x_l)
    Vec xi(n1);
    for (int l = 0; l < n1; ++l) xi[l] = (p % 2 == 1) ? (double)(l + 1 - k0) / n_el : (l + 0.5) / n_el;
    Mat E(n1, n);
    for (int l = 0; l < n1; ++l) {
        const int s = sp.span(xi[l]);
        std::vector<Vec> d;
        sp.ders(s, xi[l], 0, &d);
        for (int a = 0; a <= p; ++a) {
            const int i = s - p - 1 + k0 + a;
            if (i >= 0 && i < n) E(l, i) = d[0][a];
        }
    }
    Mat Cint = matmul(E, V1);
    Vec om(n1);
    for (int j = 0; j < n1; ++j) om[j] = (j + 1 - 0.5 * (k0 + k1)) * M_PI;
    Mat Udft(n1, n1);
    for (int l = 0; l < n1; ++l)
        for (int j = 0; j < n1; ++j) Udft(l, j) = sqrt(2.0) * sin(om[j] * xi[l] + 0.5 * M_PI * k0);
    Mat U1 = Udft;
    if (!lu_solve(Cint, U1)) {
        set_error("tpcg_setup: singular collocation matrix");
        return TPCG_E_INVALID;
    }
    Mat V1U1 = matmul(V1, U1);
    // mu_j: symbol of an interior B-spline sampled on the interpolation lattice
    {
        const int f0 = (p + n_el - 1) / 2;   // full index of an interior function: distinct local knots
        const int i0 = f0 - 1 + k0;          // its reduced index
        const double cen = 0.5 * (sp.knots[f0] + sp.knots[f0 + p + 1]);
        H.mu.assign(n1, 0.0);
        for (int l = 0; l < n1; ++l) {
            const double v = E(l, i0);
            if (v == 0.0) continue;
            const double off = xi[l] - cen;
            for (int j = 0; j < n1; ++j) H.mu[j] += v * cos(om[j] * off);
        }
    }
    // W = V1U1 diag(mu) U_dft^{-1}  (solve U_dft^T W^T = (V1U1 diag mu)^T), then keep its sparse pattern
    Mat RHS(n1, n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n1; ++j) RHS(j, i) = V1U1(i, j) * H.mu[j];
    Mat UdT(n1, n1);
    for (int a = 0; a < n1; ++a)
        for (int b = 0; b < n1; ++b) UdT(a, b) = Udft(b, a);
    if (!lu_solve(UdT, RHS)) {
        set_error("tpcg_setup: singular sine matrix");
        return TPCG_E_INVALID;
    }
    double wmax = 0;
    for (double v : RHS.a) wmax = std::max(wmax, fabs(v));
    H.w_rowptr.assign(n + 1, 0);
    H.w_col.clear();
    H.w_val.clear();
    for (int i = 0; i < n; ++i) {
        for (int l = 0; l < n1; ++l) {
            const double v = RHS(l, i);
            if (fabs(v) > 1e-11 * wmax) {
                H.w_col.push_back(l);
                H.w_val.push_back(v);
            }
        }
        H.w_rowptr[i + 1] = (int)H.w_col.size();
    }
    // V2 = M^{-1} N with N a basis of null(V1^T); U2, Lambda2 from the projected pencil
    H.lam.assign(n, 0.0);
    for (int j = 0; j < n1; ++j) H.lam[j] = om[j] * om[j];
    H.v2u2.clear();
    if (n2 > 0) {
        Mat N(n, n2);
        for (int end = 0; end < 2; ++end) {
            const int c = nord[end], m = blk[end];
            if (c == 0) continue;
            Vec ev;
            Mat EV;
            sym_eig(matmul(Z[end], Z[end], false, true), &ev, &EV);   // null(Z^T): eigenvalue-0 eigenvectors of Z Z^T
            for (int q = 0; q < m - c; ++q)
                for (int i = 0; i < m; ++i) N((end == 0 ? 0 : n - m) + i, end * c0 + q) = EV(i, q);
        }
        Mat V2 = N;
        if (!lu_solve(Md, V2)) {
            set_error("tpcg_setup: singular mass matrix");
            return TPCG_E_INVALID;
        }
        Mat A2 = matmul(V2, matmul(Kd, V2), true, false);
        Mat B2 = matmul(V2, matmul(Md, V2), true, false);
        // Cholesky B2 = L L^T, C = L^{-1} A2 L^{-T}
        Mat L(n2, n2);
        for (int j = 0; j < n2; ++j) {
            double s = B2(j, j);
            for (int q = 0; q < j; ++q) s -= L(j, q) * L(j, q);
            L(j, j) = sqrt(s);
            for (int i = j + 1; i < n2; ++i) {
                double t = B2(i, j);
                for (int q = 0; q < j; ++q) t -= L(i, q) * L(j, q);
                L(i, j) = t / L(j, j);
            }
        }
        Mat Li(n2, n2);   // L^{-1}
        for (int c = 0; c < n2; ++c)
            for (int i = 0; i < n2; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                for (int q = 0; q < i; ++q) s -= L(i, q) * Li(q, c);
                Li(i, c) = s / L(i, i);
            }
        Mat C = matmul(Li, matmul(A2, Li, false, true));
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < i; ++j) C(i, j) = C(j, i) = 0.5 * (C(i, j) + C(j, i));
        Vec lam2;
        Mat Y;
        sym_eig(C, &lam2, &Y);
        Mat U2 = matmul(Li, Y, true, false);   // L^{-T} Y
        Mat VU = matmul(V2, U2);
        H.v2u2 = VU.a;
        for (int j = 0; j < n2; ++j) H.lam[n1 + j] = lam2[j];
    }
    double lmin = 1e300, lmax = 0;
    for (double v : H.lam) { lmin = std::min(lmin, v); lmax = std::max(lmax, v); }
    H.lambda_min = 3.0 * lmin;
    H.lambda_max = 3.0 * lmax;
    const double MP = H.lambda_max / H.lambda_min;
    H.RP = expsum_kind() == 1 ? expsum_best(MP, eps_prec, 60, &H.omega, &H.alpha, nullptr)
                              : expsum_sinc(MP, eps_prec, &H.omega, &H.alpha);
    if (H.RP < 1) {
        set_error("tpcg_setup: no exponential sum found");
        return TPCG_E_INVALID;
    }
    return TPCG_OK;
}

int host_setup(const tpcg_geometry& geo, int p, int n, HostProblem* out) {
    const int k0 = geo.k0, k1 = geo.k1;
    if (k0 < 0 || k0 > 1 || k1 < 0 || k1 > 1 || (k0 == 1 && k1 == 1)) {
        set_error("tpcg_setup: boundary flags (k0, k1) must be (0,0), (0,1) or (1,0)");
        return TPCG_E_INVALID;
    }
    const int n_el = n - p + 2 - k0 - k1;
    if (p < 1 + (k0 | k1) || p > 5 || n_el <= p || n > 1024 ||
        (geo.kind != TPCG_GEOM_CUBE && geo.kind != TPCG_GEOM_TWIST)) {
        set_error("tpcg_setup: need 1 <= p <= 5 (2 <= p with a Neumann end), n - p + 2 - k0 - k1 > p, n <= 1024 and "
                  "a known geometry");
        return TPCG_E_INVALID;
    }
    const double eps_geo = geo.eps_geo > 0 ? geo.eps_geo : 1e-8;
    const double eps_prec = geo.eps_prec > 0 ? geo.eps_prec : 0.1;
    HostProblem& H = *out;
    H.k0 = k0;
    H.k1 = k1;
    Spline sp(p, n_el);
    Quad Q = make_quad(sp, k0, k1);

    // ---- coefficient samples on the Chebyshev grid
    Ten Tq[3][3], Tw;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Tq[a][b].d[0] = Tq[a][b].d[1] = Tq[a][b].d[2] = NCHEB;
            Tq[a][b].a.assign((size_t)NCHEB * NCHEB * NCHEB, 0.0);
        }
    Tw.d[0] = Tw.d[1] = Tw.d[2] = NCHEB;
    Tw.a.assign((size_t)NCHEB * NCHEB * NCHEB, 0.0);
    for (int k = 0; k < NCHEB; ++k)
        for (int j = 0; j < NCHEB; ++j)
            for (int i = 0; i < NCHEB; ++i) {
                double Qv[3][3], om;
                coefficients(geo.kind, geo.amp, cheb_pt(i), cheb_pt(j), cheb_pt(k), Qv, &om, k0, k1);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) Tq[a][b].at(i, j, k) = Qv[a][b];
                Tw.at(i, j, k) = om;
            }
    {
        const int st = terms_from_coeffs(Tq, eps_geo, Q, n, p, H);
        if (st != TPCG_OK) return st;
    }
    rhs_from_samples(Tw, eps_geo, Q, n, p, 1.0, H);
    return fd_tables(sp, Q, n, p, eps_prec, H);
}


// Elasticity (Sec. 5.3): out[3 i + j] holds block A_ij (Kronecker terms of C^{ij}_{kl}), the rhs component f_i
// (force_i times the load of a unit body force, det J) and the shared App. B / Prop. 1 tables.
int host_elast_setup(const tpcg_geometry& geo, int p, int n, double lam, double mu, const double force[3],
                     HostProblem out[9]) {
    const int k0 = geo.k0, k1 = geo.k1;
    if (k0 < 0 || k0 > 1 || k1 < 0 || k1 > 1 || (k0 == 1 && k1 == 1)) {
        set_error("tpcg_elast_setup: boundary flags (k0, k1) must be (0,0), (0,1) or (1,0)");
        return TPCG_E_INVALID;
    }
    const int n_el = n - p + 2 - k0 - k1;
    if (p < 1 + (k0 | k1) || p > 5 || n_el <= p || n > 1024 ||
        (geo.kind != TPCG_GEOM_CUBE && geo.kind != TPCG_GEOM_TWIST) || !(mu > 0) || !(lam >= 0)) {
        set_error("tpcg_elast_setup: need 1 <= p <= 5 (2 <= p with a traction-free face), n - p + 2 - k0 - k1 > p, "
                  "n <= 1024, a known geometry, mu > 0, lambda >= 0");
        return TPCG_E_INVALID;
    }
    const double eps_geo = geo.eps_geo > 0 ? geo.eps_geo : 1e-8;
    const double eps_prec = geo.eps_prec > 0 ? geo.eps_prec : 0.1;
    Spline sp(p, n_el);
    Quad Q = make_quad(sp, k0, k1);
    const size_t N3 = (size_t)NCHEB * NCHEB * NCHEB;
    std::vector<Ten> Tc(81);   // [((i*3 + j)*3 + k)*3 + l]
    for (Ten& T : Tc) {
        T.d[0] = T.d[1] = T.d[2] = NCHEB;
        T.a.assign(N3, 0.0);
    }
    Ten Tw;
    Tw.d[0] = Tw.d[1] = Tw.d[2] = NCHEB;
    Tw.a.assign(N3, 0.0);
    for (int k3 = 0; k3 < NCHEB; ++k3)
        for (int j3 = 0; j3 < NCHEB; ++j3)
            for (int i3 = 0; i3 < NCHEB; ++i3) {
                double C[3][3][3][3], det;
                elast_coefficients(geo.kind, geo.amp, lam, mu, cheb_pt(i3), cheb_pt(j3), cheb_pt(k3), C, &det);
                for (int q = 0; q < 81; ++q) Tc[q].at(i3, j3, k3) = C[q / 27][(q / 9) % 3][(q / 3) % 3][q % 3];
                Tw.at(i3, j3, k3) = det;
            }
    HostProblem fdh;
    fdh.k0 = k0;
    fdh.k1 = k1;
    {
        const int st = fd_tables(sp, Q, n, p, eps_prec, fdh);
        if (st != TPCG_OK) return st;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            HostProblem& H = out[3 * i + j];
            H = fdh;   // App. B tables and exponential sum
            Ten Tq[3][3];
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) Tq[k][l] = Tc[((i * 3 + j) * 3 + k) * 3 + l];
            const int st = terms_from_coeffs(Tq, eps_geo, Q, n, p, H);
            if (st != TPCG_OK) return st;
            rhs_from_samples(Tw, eps_geo, Q, n, p, force[i], H);
        }
    return TPCG_OK;
}

}  // namespace tpcg

// Host-only form of tpcg_setup: the same FP64 setup, its tables copied to caller-owned host buffers (no GPU call)
extern "C" int tpcg_setup_host(const tpcg_geometry* geo, int degree, int n, tpcg_problem_info* info, double* w,
                               double* bands, double* f_core, double* f_U0, double* f_U1, double* f_U2, double* lam,
                               double* mu, double* v2u2, double* omega, double* alpha, int* w_rowptr, int* w_col,
                               double* w_val) {
    if (!geo || !info) {
        tpcg::set_error("tpcg_setup_host: null geometry or info");
        return TPCG_E_INVALID;
    }
    tpcg::HostProblem H;
    const int s = tpcg::host_setup(*geo, degree, n, &H);
    if (s != TPCG_OK) return s;
    *info = tpcg_problem_info{};
    info->n = n;
    info->p = degree;
    info->R = H.R;
    info->RP = H.RP;
    info->n1 = H.n1;
    info->n2 = H.n2;
    for (int t = 0; t < 3; ++t) info->rf[t] = H.rf[t];
    info->lambda_min = H.lambda_min;
    info->lambda_max = H.lambda_max;
    info->MP = H.lambda_max / H.lambda_min;
    info->w_nnz = (int)H.w_val.size();
    info->k0 = H.k0;
    info->k1 = H.k1;
    auto cp = [](double* dst, const std::vector<double>& v) {
        if (dst && !v.empty()) std::copy(v.begin(), v.end(), dst);
    };
    cp(w, H.w);
    cp(bands, H.bands);
    cp(f_core, H.f_core);
    cp(f_U0, H.f_U[0]);
    cp(f_U1, H.f_U[1]);
    cp(f_U2, H.f_U[2]);
    cp(lam, H.lam);
    cp(mu, H.mu);
    cp(v2u2, H.v2u2);
    cp(omega, H.omega);
    cp(alpha, H.alpha);
    cp(w_val, H.w_val);
    if (w_rowptr) std::copy(H.w_rowptr.begin(), H.w_rowptr.end(), w_rowptr);
    if (w_col && !H.w_col.empty()) std::copy(H.w_col.begin(), H.w_col.end(), w_col);
    return TPCG_OK;
}
