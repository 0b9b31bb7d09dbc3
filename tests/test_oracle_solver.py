"""Pins of the oracle's solver path: Tucker arithmetic, truncation, FD application, TPCG. CPU only."""
import numpy as np
import pytest
import scipy.stats

import synth
from oracle import fd, fullcg, lowrank, rounding, tpcg, tucker


def _assembled(terms):
    return fullcg.assemble(terms).toarray()


# ------------------------------------------------------------------------------------ Tucker arithmetic
def test_kron_vec_identity_and_matvec_brute_force():
    n = (5, 6, 4)
    X = synth.random_tucker(n, (2, 3, 2), seed=11)
    mats = [synth.random_banded(n[t], 2, 3, seed=20 + t, symmetric=False) for t in range(3)]
    terms = [(0.5 + j, [mats[0][j], mats[1][j], mats[2][j]]) for j in range(3)]
    A = _assembled(terms)
    xv = tucker.vec(tucker.full(X))
    for form in (True, False):
        Y = tucker.matvec(terms, X, dense=form)
        assert np.abs(tucker.vec(tucker.full(Y)) - A @ xv).max() <= 1e-12 * np.abs(A @ xv).max()
    # eq. kron_vec_multi on one term
    J = [mats[t][0] for t in range(3)]
    lhs = np.kron(J[2], np.kron(J[1], J[0])) @ xv
    rhs = tucker.vec(tucker.contract(tucker.full(X), J))
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_dot_sum_scale_against_full_tensors():
    n = (7, 5, 6)
    X = synth.random_tucker(n, (3, 2, 4), seed=1)
    Y = synth.random_tucker(n, (2, 4, 3), seed=2)
    fx, fy = tucker.full(X), tucker.full(Y)
    assert abs(tucker.dot(X, Y) - np.sum(fx * fy)) <= 1e-12 * np.linalg.norm(fx) * np.linalg.norm(fy)
    S = tucker.add(X, tucker.scale(Y, -0.7))
    assert np.abs(tucker.full(S) - (fx - 0.7 * fy)).max() <= 1e-12 * np.abs(fx).max()
    Sd = tucker.add_dense(X, Y)
    assert np.abs(tucker.full(Sd) - (fx + fy)).max() <= 1e-12 * np.abs(fx).max()
    assert tucker.ranks(S) == (5, 6, 7)


def test_kron_core_index_rule():
    A = np.arange(8.0).reshape(2, 2, 2) + 1
    B = np.arange(27.0).reshape(3, 3, 3) - 5
    C = tucker.kron_core(A, B)
    for i in np.ndindex(2, 2, 2):
        for j in np.ndindex(3, 3, 3):
            k = tuple(j[l] + i[l] * 3 for l in range(3))      # eq. kron_tensors (0-based)
            assert C[k] == A[i] * B[j]


# ------------------------------------------------------------------------------------ truncation
def _rotated_superdiagonal(d, n, seed):
    """Z = superdiag(d) x_t Q_t with orthonormal Q_t: mode singular values are |d| exactly."""
    g = np.random.default_rng(seed)
    Qs = [np.linalg.qr(g.standard_normal((n, len(d))))[0] for _ in range(3)]
    return tucker.contract(tucker.superdiagonal(d), Qs)


def test_sthosvd_rank_rule_closed_form():
    d = np.array([1.0, 0.5, 0.1, 3e-3, 1e-3, 2e-4, 1e-5])
    Z = _rotated_superdiagonal(d, 12, seed=5)
    eps = 2e-3
    core, S, disc = rounding.sthosvd(Z, eps)
    # every unfolding has singular values |d|; after mode 1 the kept ones carry on
    budget = eps ** 2 * np.sum(d ** 2) / 3
    keep = len(d)
    ranks = []
    tail_total = 0.0
    for m in range(3):
        dd = d[:keep]
        s = next(s for s in range(len(dd) + 1) if np.sum(dd[s:] ** 2) <= budget)
        tail_total += np.sum(dd[s:] ** 2)
        ranks.append(s)
        keep = s
    assert list(core.shape) == ranks
    assert abs(disc - tail_total) <= 1e-12 * np.sum(d ** 2)
    err = np.sum((tucker.contract(core, S) - Z) ** 2)
    assert abs(err - disc) <= 1e-12 * np.sum(d ** 2)           # sequential errors add in squares


@pytest.mark.parametrize("eps", [0.0, 1e-10, 1e-4, 1e-2, 0.2])
def test_t_rel_error_bound_and_orthonormal_factors(eps):
    n = (11, 9, 10)
    parts = [synth.random_tucker(n, (3, 3, 3), seed=s, decay=0.3) for s in (1, 3, 5)]
    Y = parts[0]
    for P in parts[1:]:
        Y = tucker.add(Y, P)
    (G, U), info = rounding.t_rel(Y, eps, return_info=True)
    fy = tucker.full(Y)
    err = np.linalg.norm(tucker.full((G, U)) - fy)
    assert err <= eps * np.linalg.norm(fy) + 1e-12 * np.linalg.norm(fy)    # eq. rel_estimate
    assert abs(err ** 2 - info["discarded"]) <= 1e-10 * np.sum(fy ** 2)
    for m in range(3):
        assert np.abs(U[m].T @ U[m] - np.eye(U[m].shape[1])).max() < 1e-12


def test_t_rel_recovers_exact_rank_of_a_sum():
    n = (13, 12, 11)
    A = synth.random_tucker(n, (2, 3, 2), seed=7)
    B = synth.random_tucker(n, (3, 2, 2), seed=9)
    Y = tucker.add(A, tucker.add(B, tucker.scale(A, 2.0)))   # rank (5, 5, 4) although 7/8/6 columns
    G, U = rounding.t_rel(Y, 1e-9)
    assert G.shape == (5, 5, 4)
    assert np.linalg.norm(tucker.full((G, U)) - tucker.full(Y)) <= 1e-9 * np.linalg.norm(tucker.full(Y))


def test_t_rel_wide_factors_when_rank_exceeds_n():
    # k > n (the heavy case of Alg. 1): the QR gives n x n Q_t and n x k R_t
    n = (6, 7, 5)
    Y = synth.random_tucker(n, (9, 10, 8), seed=4)
    G, U = rounding.t_rel(Y, 0.0)
    assert G.shape == (6, 7, 5)
    assert np.abs(tucker.full((G, U)) - tucker.full(Y)).max() <= 1e-11 * np.abs(tucker.full(Y)).max()


def test_dynamic_truncation_lossless_and_monotone():
    n = (9, 9, 9)
    x = rounding.t_rel(synth.random_tucker(n, (3, 3, 3), seed=2), 0.0)
    p = rounding.t_rel(synth.random_tucker(n, (2, 2, 2), seed=3), 0.0)
    xt = tucker.add(x, tucker.scale(p, 0.3))
    # lossless truncation: v = 1 at once
    y, e, trials = rounding.t_dt(x, xt, 1e-12, 0.5, 1e-14, 1e-3)
    assert trials == 1 and e == 1e-12
    # lossy start: tolerance only decreases, never below eps_min / alpha
    p2 = synth.random_tucker(n, (3, 3, 3), seed=8, decay=0.2)
    xt = tucker.add(x, tucker.scale(p2, 1e-3))
    y, e, trials = rounding.t_dt(x, xt, 0.3, 0.5, 1e-6, 1e-3)
    assert e <= 0.3 and e >= 1e-6 * 0.5 - 1e-18
    assert abs(e - 0.3 * 0.5 ** (trials - 1)) < 1e-15


def test_dynamic_truncation_update_ratio_closed_form():
    # Alg. 2 on tensors with one orthonormal basis per mode and superdiagonal cores: x_k = diag(a) on the
    # first two basis vectors, the step Delta x~ = diag(b) on the next five.  Every mode of x~ then has the
    # singular values (a, b), so the ST-HOSVD of Alg. 1 drops exactly the smallest entries e whose squares
    # sum to at most eps^2 ||x~||^2 / 3 (mode 1; the other modes then have nothing left to drop).  The
    # discarded part e lies inside Delta x~ and is orthogonal to what is kept, so the update ratio of Sec. 4.1.2
    # has the closed form v = (Delta x~ . Delta x) / ||Delta x~||^2 = 1 - ||e||^2 / ||Delta x~||^2.
    n = 10
    Q = [np.linalg.qr(np.random.default_rng(40 + t).standard_normal((n, 7)))[0] for t in range(3)]
    a = np.array([3.0, 2.0])
    b = np.array([1.0, 0.3, 0.05, 0.01, 0.002])

    def diag_tensor(vals, off):
        G = np.zeros((len(vals),) * 3)
        for i, v in enumerate(vals):
            G[i, i, i] = v
        return (G, [Q[t][:, off:off + len(vals)] for t in range(3)])

    x = diag_tensor(a, 0)
    xt = tucker.add(x, diag_tensor(b, 2))
    d_all = np.concatenate([a, b])
    total = float(np.sum(d_all ** 2))
    db2 = float(np.sum(b ** 2))

    def dropped(eps):   # squared norm of the entries the rule of Alg. 1 discards at tolerance eps
        s2 = np.sort(d_all ** 2)
        tail = np.cumsum(s2)
        return float(tail[tail <= eps * eps * total / 3.0][-1]) if np.any(tail <= eps * eps * total / 3.0) else 0.0

    eps, alpha, delta, eps_min = 0.1, 0.5, 1e-3, 1e-6
    # the sequence of Alg. 2 written out from the closed form: 0.1, 0.05 and 0.025 drop (0.05, 0.01, 0.002),
    # |v - 1| = 2.4e-3 > delta; 0.0125 drops (0.01, 0.002) only, |v - 1| = 9.5e-5 < delta
    expect_eps, expect_trials = eps, 1
    while abs(dropped(expect_eps) / db2) >= delta and alpha * expect_eps > eps_min:
        expect_eps *= alpha
        expect_trials += 1
    assert (expect_eps, expect_trials) == (0.0125, 4)
    y, e_new, trials = rounding.t_dt(x, xt, eps, alpha, eps_min, delta)
    assert trials == expect_trials and e_new == expect_eps
    # the truncated iterate is x~ without the dropped entries, and v takes its closed-form value
    keep = d_all.copy()
    keep[[5, 6]] = 0.0
    assert np.abs(tucker.full(y) - tucker.full(diag_tensor(keep, 0))).max() < 1e-13
    dx = tucker.add(y, tucker.scale(x, -1.0))
    dxt = tucker.add(xt, tucker.scale(x, -1.0))
    v = tucker.dot(dxt, dx) / tucker.dot(dxt, dxt)
    assert abs(v - (1.0 - (0.01 ** 2 + 0.002 ** 2) / db2)) < 1e-14
    # a swapped denominator (||Delta x||^2) would give v = 1 at the first trial: the pin tells them apart
    assert abs(dropped(0.1) / db2) > delta


# ------------------------------------------------------------------------------------ FD application
def test_alg4_matches_full_formula():
    n, p = 8, 3
    P = fd.ApproxFD(n, p)
    S = synth.random_tucker((n, n, n), (2, 3, 2), seed=13)
    V = P.apply(S)
    U = P.U
    s = tucker.full(S)
    T = tucker.contract(s, [U.T, U.T, U.T])
    Dt = sum(P.omega[j] / P.lmin * np.einsum("i,j,k->ijk", P.diag(j), P.diag(j), P.diag(j)) for j in range(P.RP))
    v = tucker.contract(Dt * T, [U, U, U])
    assert np.abs(tucker.full(V) - v).max() <= 1e-11 * np.abs(v).max()
    assert tucker.ranks(V) == (2 * P.RP, 3 * P.RP, 2 * P.RP)


def test_exact_fd_on_cube_is_the_inverse():
    # eq. FD_prec with Q = I: P = A, so PCG with the exact FD converges in one step
    n, p = 6, 3
    terms = lowrank.cube_terms(n, p)
    A = fullcg.assemble(terms)
    b = np.random.default_rng(0).standard_normal(n ** 3)
    x, its = fullcg.pcg(A, b, lambda r: fd.exact_fd_apply_full(n, p, r), tol=1e-12)
    assert its == 1


# ------------------------------------------------------------------------------------ TPCG
def test_tpcg_cube_rank_one():
    n, p = 14, 2
    terms = lowrank.operator_terms("cube", 0.0, n, p)
    f = lowrank.rhs_tucker("cube", 0.0, n, p)
    P = fd.ApproxFD(n, p)
    x, info = tpcg.tpcg(terms, f, P.apply, tpcg.Params(tol=1e-6))
    xe = fullcg.solve_direct(terms, tucker.vec(tucker.full(f)))
    assert info["res"] <= 1e-6
    assert np.linalg.norm(tucker.vec(tucker.full(x)) - xe) <= 1e-5 * np.linalg.norm(xe)


def test_tpcg_twist_against_direct_solve():
    n, p = 11, 3
    amp = synth.amp_from_seed(7)
    terms = lowrank.operator_terms("twist", amp, n, p)
    f = lowrank.rhs_tucker("twist", amp, n, p)
    P = fd.ApproxFD(n, p)
    x, info = tpcg.tpcg(terms, f, P.apply, tpcg.Params(tol=1e-6))
    A = fullcg.assemble(terms)
    fv = tucker.vec(tucker.full(f))
    xe = fullcg.solve_direct(terms, fv)
    xv = tucker.vec(tucker.full(x))
    assert np.linalg.norm(fv - A @ xv) <= 1.5e-6 * np.linalg.norm(fv)    # truncated residual ~ true residual
    # energy-norm error bounded by the residual and the spectrum of A
    lmin = scipy.sparse.linalg.eigsh(A, k=1, which="SA", return_eigenvectors=False)[0]
    assert np.linalg.norm(xv - xe) <= 2e-6 * np.linalg.norm(fv) / lmin
    assert 5 <= info["iters"] <= 60


def test_thick_quarter_annulus_ranks_and_tpcg_matches_exact_pcg():
    # Sec. 5.2: the untwisted annulus is the paper's thick quarter annulus. Its coefficient ranks are (1, 1, 1)
    # on the diagonal blocks and 0 off them, so A~ has R = 3 Kronecker terms. With the paper's manufactured
    # solution u = (x^2 + y^2 - 1)(x^2 + y^2 - 4) sin(pi z) sin(7 x y), TPCG (Alg. 5 with the relaxed
    # truncations of eq. rel_tol_iterates) needs no more iterations than textbook PCG with the same
    # preconditioner on the assembled system (22 and 22 here): the truncation costs no convergence
    sp = pytest.importorskip("sympy")
    from oracle import bspline, expsum
    x, y, z = sp.symbols("x y z")
    u = (x ** 2 + y ** 2 - 1) * (x ** 2 + y ** 2 - 4) * sp.sin(sp.pi * z) * sp.sin(7 * x * y)
    fx = sp.lambdify((x, y, z), -(sp.diff(u, x, 2) + sp.diff(u, y, 2) + sp.diff(u, z, 2)), "numpy")
    n_el, p = 16, 2
    n = n_el + p - 2
    terms = lowrank.operator_terms("twist", 0.0, n, p)
    assert len(terms) == 3
    # load: det J f(F(eta)) (App. A) on the polar map rho = 1 + eta1, theta = pi eta2 / 2, z = eta3
    xc = lowrank.cheb_points()
    e1, e2, e3 = np.meshgrid(xc, xc, xc, indexing="ij")
    rho, th = 1.0 + e1, 0.5 * np.pi * e2
    core, U = lowrank.tucker_of_samples(0.5 * np.pi * rho * fx(rho * np.cos(th), rho * np.sin(th), e3), 1e-8)
    xs, ws = bspline.quadrature(n_el, p)
    B0 = bspline.dirichlet_basis(n_el, p, xs, 0)
    F = (core, [(B0 * ws) @ lowrank.cheb_eval(U[t], xs) for t in range(3)])
    P0 = fd.ApproxFD(n, p)
    _, om, al, _, _ = expsum.rp_best(P0.MP, 0.1)
    P = fd.ApproxFD(n, p, expsum=(om, al))
    _, info = tpcg.tpcg(terms, F, P.apply, tpcg.Params(tol=1e-6))
    A = fullcg.assemble(terms)
    b = tucker.vec(tucker.full(F))

    def prec(r):
        R = tucker.unvec(r, (n, n, n))
        return tucker.vec(tucker.full(P.apply((R, [np.eye(n)] * 3))))

    _, it_full = fullcg.pcg(A, b, prec, tol=1e-6)
    assert info["iters"] <= it_full
