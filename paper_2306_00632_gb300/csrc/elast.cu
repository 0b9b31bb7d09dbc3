// Compressible linear elasticity in Tucker format (Sec. 5.3): the 3 x 3 block operator A = [A_ij], block
// right-hand side, block-diagonal FD preconditioner, and Alg. 5 on block vectors.
//
// Every block A_ij is a Kronecker sum (its own tpcg_problem holding the bands and weights); the diagonal
// problems also hold the rhs component f_i and the App. B / Prop. 1 tables shared by all blocks.  A block
// vector is three Tucker tensors.  Products y_i = sum_j A_ij x_j append the R_ij blocks of every A_ij x_j
// to y_i's block list (apply_append_impl), so a block product is one unrounded Tucker tensor per component;
// scalar products are sums over components, truncations and sums act per component (Sec. 5.3).
// Preconditioner block i: fast diagonalization of mu (K M M + M K M + M M K) + (lambda + mu) (K in
// direction i), i.e. Alg. 4 with direction weights c_t = mu + (lambda + mu) delta_ti.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "kernels.cuh"
#include "setup.h"

struct tpcg_elast_s {
    int n, p, dtype;
    tpcg_problem blk[9];   // A_ij at 3 i + j; the diagonal ones carry f_i and the FD tables
    double c[3][3];        // direction weights of preconditioner block i
    double lame_lambda, lame_mu;
    double norm_f;         // ||[f_1; f_2; f_3]||
};

namespace tpcg {

__global__ void sum3_kernel(const double* a, double* out) { *out = a[0] + a[1] + a[2]; }

// an empty block list (rank 0, no blocks): the start of an appended block product
__global__ void set_empty_kernel(TuckerDesc* d) {
    d->nblk = 0;
    d->rank[0] = d->rank[1] = d->rank[2] = 0;
}

static int elast_check_block(tpcg_elast e, const tucker_t* x, const char* what) {
    for (int i = 0; i < 3; ++i) TPCG_TRY(check_tensor(&x[i], e->n, e->dtype, what));
    return TPCG_OK;
}

// y_i = (f_i if residual) -/+ sum_j A_ij x_j for i = 0, 1, 2 (unrounded; x_j may be block tensors).
// err: nine device ints, block (i, j) sets err[3 i + j] when its product does not fit y_i; the solver passes
// flags of its own context (null: the blocks' problem flags, for standalone calls)
template <typename T>
static int elast_apply_impl(tpcg_elast e, tucker_t* const* x, tucker_t* const* y, bool residual, int cap,
                            cudaStream_t st, int* err = nullptr) {
    for (int i = 0; i < 3; ++i) {
        if (residual)
            TPCG_TRY(copy_tensor_impl<T>(&e->blk[4 * i]->f, y[i], e->n, cap, st));
        else {
            set_empty_kernel<<<1, 1, 0, st>>>(static_cast<TuckerDesc*>(y[i]->desc));
            TPCG_CHECK_LAUNCH();
        }
        for (int j = 0; j < 3; ++j)
            TPCG_TRY(apply_append_impl<T>(e->blk[3 * i + j], x[j], y[i], residual ? -1.0 : 1.0, st,
                                          err ? err + 3 * i + j : nullptr));
    }
    return TPCG_OK;
}

// v_i = P~_i^-1 s_i (Alg. 4 with the direction weights of block i)
template <typename T>
static int elast_precond_impl(tpcg_elast e, tpcg_ctx c, tucker_t* const* s, tucker_t* const* v, cudaStream_t st) {
    for (int i = 0; i < 3; ++i) TPCG_TRY(fd_impl<T>(e->blk[4 * i], c, s[i], v[i], st, e->c[i]));
    return TPCG_OK;
}

// *out = sum_i <x_i, y_i> (x_i, y_i plain)
template <typename T>
static int elast_dot_impl(tpcg_ctx c, tucker_t* const* x, tucker_t* const* y, double* out, cudaStream_t st) {
    double* part = c->scal + 160;
    for (int i = 0; i < 3; ++i) TPCG_TRY(dot_cached<T>(c, x[i], y[i], part + i, st));
    sum3_kernel<<<1, 1, 0, st>>>(part, out);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

}  // namespace tpcg

using namespace tpcg;

namespace tpcg {

// Alg. 5 on block vectors (same steps and scalar updates as the scalar solver, block operations)
template <typename T>
static int elast_solve_impl(tpcg_elast e, tpcg_ctx c, const tpcg_params* prm, tucker_t* xout, tpcg_stats* st,
                            cudaStream_t s) {
    TPCG_TRY(ensure_tensors(c, 21));
    const int rc = (prm->rank_cap > 0 && prm->rank_cap < c->rank_cap) ? prm->rank_cap : c->rank_cap;
    const int n = c->n, cap = c->max_cols;
    double* sc = c->scal;
    double* dprm = c->scal + 100;
    double hp[P_COUNT] = {prm->tol, prm->eps0, prm->eps_min, prm->alpha, prm->delta, prm->beta_trunc};
    TPCG_CUDA(cudaMemcpyAsync(dprm, hp, sizeof(hp), cudaMemcpyHostToDevice, s));
    // block vectors: x, r, z, p, q, big, big2 (three tensors each)
    tucker_t* x[3];
    tucker_t* r[3];
    tucker_t* z[3];
    tucker_t* p[3];
    tucker_t* q[3];
    tucker_t* big[3];
    tucker_t* big2[3];
    tucker_t** all[7] = {x, r, z, p, q, big, big2};
    for (int v = 0; v < 7; ++v)
        for (int i = 0; i < 3; ++i) all[v][i] = &c->tens[3 * v + i];
    auto bswap = [](tucker_t** a, tucker_t** b) {
        for (int i = 0; i < 3; ++i) std::swap(a[i], b[i]);
    };
    auto bround = [&](tucker_t** y, const double* eps_dev) -> int {
        for (int i = 0; i < 3; ++i) TPCG_TRY(round_cached<T>(c, y[i], eps_dev, rc, s, prm->tol < 1e-8 ? -1 : 0));
        return TPCG_OK;
    };
    auto bcopy = [&](tucker_t** a, tucker_t** b) -> int {
        for (int i = 0; i < 3; ++i) TPCG_TRY(copy_tensor_impl<T>(a[i], b[i], n, cap, s));
        return TPCG_OK;
    };
    auto baxpby = [&](tucker_t** a, const double* bdev, tucker_t** b, tucker_t** out) -> int {
        for (int i = 0; i < 3; ++i) TPCG_TRY(axpby_impl<T>(1.0, nullptr, a[i], 0.0, bdev, b[i], out[i], nullptr, s));
        return TPCG_OK;
    };
    double* eta = sc + S_ETA;
    // capacity flags of the nine block products and of the preconditioner, read every iteration; they live in
    // this context, so solves that share the elasticity object never see each other's flags
    int* fd_err = reinterpret_cast<int*>(sc + 230);
    int* apply_err = reinterpret_cast<int*>(sc + 240);   // 9 ints
    TPCG_CUDA(cudaMemsetAsync(fd_err, 0, sizeof(int), s));
    TPCG_CUDA(cudaMemsetAsync(apply_err, 0, 9 * sizeof(int), s));
    // x_0 = 0, r_0 = f
    for (int i = 0; i < 3; ++i) TPCG_TRY(set_zero(x[i], s));
    for (int i = 0; i < 3; ++i) TPCG_TRY(copy_tensor_impl<T>(&e->blk[4 * i]->f, r[i], n, cap, s));
    TPCG_TRY(elast_dot_impl<T>(c, r, r, sc + S_RR, s));
    launch_scalar(OP_INIT, sc, dprm, s);
    // z_0 = T(P^-1 r_0, eta_0), p_0 = z_0, q_0 = T(A p_0, eta_0), xi_0 = p_0 . q_0
    TPCG_TRY(elast_precond_impl<T>(e, c, r, big, s));
    TPCG_TRY(bround(big, eta));
    bswap(z, big);
    TPCG_TRY(bcopy(z, p));
    TPCG_TRY(elast_apply_impl<T>(e, p, big, false, cap, s, apply_err));
    TPCG_TRY(bround(big, eta));
    bswap(q, big);
    TPCG_TRY(elast_dot_impl<T>(c, p, q, sc + S_XI, s));
    launch_scalar(OP_XI, sc, dprm, s);
    double host[S_COUNT];
    int k = 0, status = TPCG_OK, trials_total = 0;
    for (;;) {
        int flags[10] = {0};
        D2H rd[11] = {{host, sc, sizeof(host)}, {&flags[9], fd_err, sizeof(int)}};
        for (int q9 = 0; q9 < 9; ++q9) rd[2 + q9] = {&flags[q9], apply_err + q9, sizeof(int)};
        TPCG_TRY(fetch(c, s, rd, 11));
        bool over = false;
        for (int q9 = 0; q9 < 10; ++q9) over = over || flags[q9] != 0;
        if (over) {
            set_error("tpcg_elast_solve: an unrounded block product exceeded the context's max_cols or the block limit");
            status = TPCG_E_INVALID;
            break;
        }
        if (host[S_BAD] != 0.0) { status = TPCG_E_BREAKDOWN; break; }
        if (host[S_STOP] != 0.0) break;
        if (k >= prm->max_it) { status = TPCG_E_NOT_CONVERGED; break; }
        TPCG_TRY(elast_dot_impl<T>(c, r, p, sc + S_RP, s));
        launch_scalar(OP_OMEGA, sc, dprm, s);
        // dynamic truncation of x_k + omega_k p_k (Alg. 2 with block scalar products)
        TPCG_TRY(elast_dot_impl<T>(c, p, x, sc + S_PXK, s));
        TPCG_TRY(elast_dot_impl<T>(c, p, p, sc + S_PP, s));
        TPCG_TRY(baxpby(x, sc + S_OMEGA, p, big));
        for (int trial = 0;; ++trial) {
            TPCG_TRY(bcopy(big, big2));
            TPCG_TRY(bround(big2, sc + S_EPS));
            TPCG_TRY(elast_dot_impl<T>(c, p, big2, sc + S_PXN, s));
            launch_scalar(OP_DT, sc, dprm, s);
            ++trials_total;
            double done;
            TPCG_TRY(fetch(c, s, {{&done, sc + S_DONE, sizeof(double)}}));
            if (done != 0.0 || trial > 64) break;
        }
        bswap(x, big2);
        // r_{k+1} = T(f - A x_{k+1}, eta_k)
        TPCG_TRY(elast_apply_impl<T>(e, x, big, true, cap, s, apply_err));
        TPCG_TRY(bround(big, eta));
        bswap(r, big);
        TPCG_TRY(elast_dot_impl<T>(c, r, r, sc + S_RR, s));
        launch_scalar(OP_RES, sc, dprm, s);
        // z_{k+1} = T(P^-1 r_{k+1}, eta_{k+1}); beta_k = -z_{k+1} . q_k / xi_k
        TPCG_TRY(elast_precond_impl<T>(e, c, r, big, s));
        TPCG_TRY(bround(big, eta));
        bswap(z, big);
        TPCG_TRY(elast_dot_impl<T>(c, z, q, sc + S_ZQ, s));
        launch_scalar(OP_BETA, sc, dprm, s);
        // p_{k+1} = T(z_{k+1} + beta_k p_k, eta_{k+1})
        TPCG_TRY(baxpby(z, sc + S_BETA, p, big));
        TPCG_TRY(bround(big, eta));
        bswap(p, big);
        // q_{k+1} = T(A p_{k+1}, eta_{k+1}); xi_{k+1} = p_{k+1} . q_{k+1}
        TPCG_TRY(elast_apply_impl<T>(e, p, big, false, cap, s, apply_err));
        TPCG_TRY(bround(big, eta));
        bswap(q, big);
        TPCG_TRY(elast_dot_impl<T>(c, p, q, sc + S_XI, s));
        launch_scalar(OP_XI, sc, dprm, s);
        ++k;
    }
    for (int i = 0; i < 3; ++i) TPCG_TRY(copy_tensor_impl<T>(x[i], &xout[i], n, xout[i].cap, s));
    // true residual ||f - A x|| (Z formation per component, no truncation)
    TPCG_TRY(elast_apply_impl<T>(e, x, big, true, cap, s, apply_err));
    for (int i = 0; i < 3; ++i) TPCG_TRY(tensor_norm2<T>(c, big[i], sc + 170 + i, s));
    double nr2[3];
    TPCG_TRY(fetch(c, s, {{nr2, sc + 170, sizeof(nr2)}, {host, sc, sizeof(host)}}));
    int rk[3][3], nb = 0;
    for (int i = 0; i < 3; ++i) TPCG_TRY(tucker_get_ranks(&xout[i], rk[i], &nb, s));   // synchronises
    if (st) {
        st->iters = k;
        st->status = status;
        st->rel_res = host[S_NF] > 0 ? host[S_NR] / host[S_NF] : 0.0;
        double mem = 0.0;
        for (int t = 0; t < 3; ++t) st->rank[t] = std::max(rk[0][t], std::max(rk[1][t], rk[2][t]));
        for (int i = 0; i < 3; ++i)
            mem += (double)rk[i][0] * rk[i][1] * rk[i][2] + (double)n * (rk[i][0] + rk[i][1] + rk[i][2]);
        st->mem_compression = mem / (3.0 * n * (double)n * n) * 100.0;   // Sec. 5.3 definition
        st->dt_trials = trials_total;
        st->max_rank_seen = std::max(st->rank[0], std::max(st->rank[1], st->rank[2]));
        st->outer_iters = 0;
        const double t2 = std::max(nr2[0], 0.0) + std::max(nr2[1], 0.0) + std::max(nr2[2], 0.0);
        st->true_rel_res = host[S_NF] > 0 ? sqrt(t2) / host[S_NF] : 0.0;
    }
    return status;
}

}  // namespace tpcg

// ======================================================================================= C ABI
template <typename F>
static int elast_by_dtype(int dtype, F&& f) {
    if (dtype == TPCG_F64) return f(double());
    if (dtype == TPCG_F32) return f(float());
    set_error("elasticity: dtype must be TPCG_F64 or TPCG_F32");
    return TPCG_E_INVALID;
}

extern "C" void tpcg_elast_destroy(tpcg_elast e) {
    if (!e) return;
    for (int q = 0; q < 9; ++q)
        if (e->blk[q]) tpcg_problem_destroy(e->blk[q]);
    delete e;
}

extern "C" int tpcg_elast_create(const tpcg_problem_arrays* blocks, double lame_lambda, double lame_mu,
                                 tpcg_elast* out) {
    if (!blocks || !out || !(lame_mu > 0) || !(lame_lambda >= 0)) {
        set_error("tpcg_elast_create: need 9 block arrays, mu > 0 and lambda >= 0");
        return TPCG_E_INVALID;
    }
    for (int q = 0; q < 9; ++q)
        if (blocks[q].n != blocks[0].n || blocks[q].p != blocks[0].p || blocks[q].dtype != blocks[0].dtype) {
            set_error("tpcg_elast_create: blocks differ in n, p or dtype");
            return TPCG_E_INVALID;
        }
    if (blocks[0].dtype != TPCG_F64 && blocks[0].dtype != TPCG_F32) {
        set_error("tpcg_elast_create: dtype must be TPCG_F64 or TPCG_F32");
        return TPCG_E_INVALID;
    }
    tpcg_elast e = new tpcg_elast_s();
    for (int q = 0; q < 9; ++q) e->blk[q] = nullptr;
    e->n = blocks[0].n;
    e->p = blocks[0].p;
    e->dtype = blocks[0].dtype;
    e->lame_lambda = lame_lambda;
    e->lame_mu = lame_mu;
    for (int q = 0; q < 9; ++q) {
        const int s = tpcg_problem_create(&blocks[q], &e->blk[q]);
        if (s != TPCG_OK) {
            tpcg_elast_destroy(e);
            return s;
        }
    }
    double nf2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        nf2 += e->blk[4 * i]->norm_f * e->blk[4 * i]->norm_f;
        for (int t = 0; t < 3; ++t) e->c[i][t] = lame_mu + (t == i ? lame_lambda + lame_mu : 0.0);
    }
    e->norm_f = sqrt(nf2);
    *out = e;
    return TPCG_OK;
}

extern "C" int tpcg_elast_setup(const tpcg_geometry* geo, int degree, int n, double lame_lambda, double lame_mu,
                                const double* force, int dtype, tpcg_elast* out) {
    if (!geo || !force || !out) return TPCG_E_INVALID;
    HostProblem hp[9];
    TPCG_TRY(host_elast_setup(*geo, degree, n, lame_lambda, lame_mu, force, hp));
    tpcg_problem_arrays a[9];
    for (int q = 0; q < 9; ++q) {
        HostProblem& h = hp[q];
        a[q] = tpcg_problem_arrays{};
        a[q].n = n; a[q].p = degree; a[q].R = h.R; a[q].dtype = dtype;
        a[q].w = h.w.data();
        a[q].bands = h.bands.data();
        for (int t = 0; t < 3; ++t) { a[q].rf[t] = h.rf[t]; a[q].f_U[t] = h.f_U[t].data(); }
        a[q].f_core = h.f_core.data();
        a[q].n1 = h.n1; a[q].n2 = h.n2; a[q].RP = h.RP; a[q].w_nnz = (int)h.w_val.size();
        a[q].lam = h.lam.data(); a[q].mu = h.mu.data();
        a[q].w_rowptr = h.w_rowptr.data(); a[q].w_col = h.w_col.data(); a[q].w_val = h.w_val.data();
        a[q].v2u2 = h.v2u2.empty() ? nullptr : h.v2u2.data();
        a[q].omega = h.omega.data(); a[q].alpha = h.alpha.data(); a[q].lambda_min = h.lambda_min;
        a[q].k0 = h.k0; a[q].k1 = h.k1;
    }
    return tpcg_elast_create(a, lame_lambda, lame_mu, out);
}

extern "C" int tpcg_elast_get_info(tpcg_elast e, int* R, int* RP, double* norm_f) {
    if (!e) return TPCG_E_INVALID;
    if (R)
        for (int q = 0; q < 9; ++q) R[q] = e->blk[q]->R;
    if (RP) *RP = e->blk[0]->RP;
    if (norm_f) *norm_f = e->norm_f;
    return TPCG_OK;
}

extern "C" int tpcg_elast_apply(tpcg_elast e, const tucker_t* x, tucker_t* y, void* stream) {
    if (!e || !x || !y) return TPCG_E_INVALID;
    TPCG_TRY(elast_check_block(e, x, "tpcg_elast_apply x"));
    TPCG_TRY(elast_check_block(e, y, "tpcg_elast_apply y"));
    tucker_t* xp[3] = {const_cast<tucker_t*>(&x[0]), const_cast<tucker_t*>(&x[1]), const_cast<tucker_t*>(&x[2])};
    tucker_t* yp[3] = {&y[0], &y[1], &y[2]};
    return elast_by_dtype(e->dtype, [&](auto z) {
        return elast_apply_impl<decltype(z)>(e, xp, yp, false, y[0].cap, static_cast<cudaStream_t>(stream));
    });
}

extern "C" int tpcg_elast_residual(tpcg_elast e, const tucker_t* x, tucker_t* y, void* stream) {
    if (!e || !x || !y) return TPCG_E_INVALID;
    TPCG_TRY(elast_check_block(e, x, "tpcg_elast_residual x"));
    TPCG_TRY(elast_check_block(e, y, "tpcg_elast_residual y"));
    tucker_t* xp[3] = {const_cast<tucker_t*>(&x[0]), const_cast<tucker_t*>(&x[1]), const_cast<tucker_t*>(&x[2])};
    tucker_t* yp[3] = {&y[0], &y[1], &y[2]};
    return elast_by_dtype(e->dtype, [&](auto z) {
        return elast_apply_impl<decltype(z)>(e, xp, yp, true, y[0].cap, static_cast<cudaStream_t>(stream));
    });
}

extern "C" int tpcg_elast_precond(tpcg_elast e, tpcg_ctx c, const tucker_t* s, tucker_t* v, void* stream) {
    if (!e || !c || !s || !v || c->n != e->n || c->dtype != e->dtype) return TPCG_E_INVALID;
    TPCG_TRY(elast_check_block(e, s, "tpcg_elast_precond s"));
    TPCG_TRY(elast_check_block(e, v, "tpcg_elast_precond v"));
    tucker_t* sp[3] = {const_cast<tucker_t*>(&s[0]), const_cast<tucker_t*>(&s[1]), const_cast<tucker_t*>(&s[2])};
    tucker_t* vp[3] = {&v[0], &v[1], &v[2]};
    return elast_by_dtype(e->dtype, [&](auto z) {
        return elast_precond_impl<decltype(z)>(e, c, sp, vp, static_cast<cudaStream_t>(stream));
    });
}

extern "C" int tpcg_elast_solve(tpcg_elast e, tpcg_ctx c, const tpcg_params* prm, tucker_t* x, tpcg_stats* st,
                                void* stream) {
    if (!e || !c || !prm || !x || c->n != e->n || c->dtype != e->dtype || c->lo || prm->tol <= 0 ||
        prm->alpha <= 0 || prm->alpha >= 1 || prm->max_it < 0) {
        set_error("tpcg_elast_solve: invalid arguments (F64/F32 context of the same n and dtype needed)");
        return TPCG_E_INVALID;
    }
    TPCG_TRY(elast_check_block(e, x, "tpcg_elast_solve x"));
    // capacities: y_i = f_i - sum_j A_ij x_j holds rf_i + sum_j R_ij rank columns and 1 + sum_j R_ij blocks
    int need = e->blk[0]->RP * c->rank_cap;
    for (int i = 0; i < 3; ++i) {
        int cols = std::max(e->blk[4 * i]->rf[0], std::max(e->blk[4 * i]->rf[1], e->blk[4 * i]->rf[2]));
        int nblk = 1;
        for (int j = 0; j < 3; ++j) {
            cols += e->blk[3 * i + j]->R * c->rank_cap;
            nblk += e->blk[3 * i + j]->R;
        }
        need = std::max(need, cols);
        if (nblk > TPCG_MAX_BLOCKS) {
            set_error("tpcg_elast_solve: row " + std::to_string(i) + " of the operator has " + std::to_string(nblk) +
                      " blocks (limit " + std::to_string(TPCG_MAX_BLOCKS) + ")");
            return TPCG_E_INVALID;
        }
    }
    if (c->max_cols < need) {
        set_error("tpcg_elast_solve: context max_cols " + std::to_string(c->max_cols) + " < required " +
                  std::to_string(need));
        return TPCG_E_INVALID;
    }
    return elast_by_dtype(e->dtype, [&](auto z) {
        return elast_solve_impl<decltype(z)>(e, c, prm, x, st, static_cast<cudaStream_t>(stream));
    });
}
