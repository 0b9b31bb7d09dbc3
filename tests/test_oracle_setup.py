"""Pins of the oracle's setup: B-splines, geometry coefficients, low-rank operator and rhs,
approximate eigenpairs (Table 1) and exponential sums.  CPU only."""
import json
import os

import numpy as np
import pytest

from oracle import bspline, fd, fullcg, geometry, lowrank, tucker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------ B-splines
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_partition_of_unity_and_integrals(p):
    n_el = 9
    kn = bspline.open_uniform_knots(n_el, p)
    x = np.linspace(0.0, 1.0, 301)
    B = bspline.basis(kn, p, x)
    assert np.abs(B.sum(axis=0) - 1.0).max() < 1e-14
    # int b_i = (xi_{i+p+1} - xi_i) / (p + 1)   (de Boor)
    xs, ws = bspline.quadrature(n_el, p)
    ints = bspline.basis(kn, p, xs) @ ws
    expect = (kn[p + 1:] - kn[: len(kn) - p - 1]) / (p + 1)
    assert np.allclose(ints, expect, atol=1e-15, rtol=1e-13)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_derivatives_against_finite_differences(p):
    kn = bspline.open_uniform_knots(7, p)
    x = np.linspace(0.013, 0.987, 57)
    h = 1e-6
    d = bspline.basis(kn, p, x, 1)
    fdiff = (bspline.basis(kn, p, x + h) - bspline.basis(kn, p, x - h)) / (2 * h)
    assert np.abs(d - fdiff).max() < 1e-6 * max(1.0, np.abs(d).max())


@pytest.mark.parametrize("p", [2, 3, 4])
def test_stiffness_kills_constants_before_dirichlet_cut(p):
    # K 1 = 0 on the full basis (Sec. 2.1: partition of unity => derivative of the sum vanishes)
    n_el = 8
    kn = bspline.open_uniform_knots(n_el, p)
    xs, ws = bspline.quadrature(n_el, p)
    D = bspline.basis(kn, p, xs, 1)
    K = (D * ws) @ D.T
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-10


# ------------------------------------------------------------------------------------ geometry
def test_twist_jacobian_matches_finite_differences():
    g = np.random.default_rng(3)
    e = g.uniform(0.05, 0.95, size=(20, 3))
    amp = 0.27
    J = geometry.twist_jacobian(e[:, 0], e[:, 1], e[:, 2], amp)
    h = 1e-6
    for b in range(3):
        ep, em = e.copy(), e.copy()
        ep[:, b] += h
        em[:, b] -= h
        Fp = np.stack(geometry.twist_map(ep[:, 0], ep[:, 1], ep[:, 2], amp), axis=-1)
        Fm = np.stack(geometry.twist_map(em[:, 0], em[:, 1], em[:, 2], amp), axis=-1)
        assert np.abs((Fp - Fm) / (2 * h) - J[:, :, b]).max() < 1e-7


def test_twist_coefficients_closed_forms():
    # the twist is a rigid rotation of each cross-section: det J = pi rho / 2 and Q_33 = det J
    g = np.random.default_rng(4)
    e = g.uniform(0.0, 1.0, size=(50, 3))
    Q, om = geometry.coefficients("twist", 0.3, e[:, 0], e[:, 1], e[:, 2])
    rho = 1.0 + e[:, 0]
    assert np.allclose(om, 0.5 * np.pi * rho, rtol=1e-13)
    assert np.allclose(np.swapaxes(Q, -1, -2), Q, atol=1e-13)
    assert np.all(np.linalg.eigvalsh(Q) > 0)
    Q0, _ = geometry.coefficients("twist", 0.0, e[:, 0], e[:, 1], e[:, 2])
    assert np.allclose(Q0[:, 0, 0], 0.5 * np.pi * rho) and np.allclose(Q0[:, 1, 1], 2.0 / (np.pi * rho))


# ------------------------------------------------------------------------------------ operator / rhs
def test_cube_operator_is_exact_kronecker_sum():
    n, p = 9, 2
    A1 = fullcg.assemble(lowrank.operator_terms("cube", 0.0, n, p)).toarray()
    A2 = fullcg.assemble(lowrank.cube_terms(n, p)).toarray()
    assert np.abs(A1 - A2).max() <= 1e-13 * np.abs(A2).max()


def test_twist_operator_symmetric_spd_and_rank_count():
    n, p = 10, 3
    T0 = lowrank.operator_terms("twist", 0.0, n, p)
    assert len(T0) == 3          # no twist: Q diagonal with separable entries, one term each
    T = lowrank.operator_terms("twist", 0.25, n, p)
    A = fullcg.assemble(T).toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    assert 15 <= len(T) <= 40


def test_lowrank_coefficients_accuracy_at_halton_points():
    # App. A: the separable approximations hold to 10 eps at Halton points.
    eps = 1e-8
    Q, _ = lowrank.sample("twist", 0.3)
    from scipy.stats import qmc
    pts = qmc.Halton(d=3, seed=0, scramble=False).random(2000)
    Qe, _ = geometry.coefficients("twist", 0.3, pts[:, 0], pts[:, 1], pts[:, 2])
    for (k, l) in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        core, U = lowrank.tucker_of_samples(Q[..., k, l], eps)
        vals = [lowrank.cheb_eval(U[t], pts[:, t]) for t in range(3)]
        approx = np.einsum("abc,qa,qb,qc->q", core, vals[0], vals[1], vals[2])
        scale = np.abs(Qe[:, k, l]).max()
        assert np.abs(approx - Qe[:, k, l]).max() <= 10 * eps * max(scale, 1.0)


def test_cube_rhs_matches_direct_quadrature():
    n, p = 12, 3
    core, F = lowrank.rhs_tucker("cube", 0.0, n, p)
    n_el = n - p + 2
    xs, ws = bspline.quadrature(n_el, p)
    f1 = bspline.dirichlet_basis(n_el, p, xs) @ (ws * np.sin(np.pi * xs))
    full = tucker.full((core, F))
    expect = 3 * np.pi ** 2 * np.einsum("i,j,k->ijk", f1, f1, f1)
    assert np.abs(full - expect).max() <= 1e-12 * np.abs(expect).max()


@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_solution_converges_at_optimal_rate(p):
    # unit cube, u = sin(pi x) sin(pi y) sin(pi z): L2 error of the Galerkin solution ~ h^{p+1}
    errs = []
    for n_el in (4, 8):
        n = n_el + p - 2
        terms = lowrank.cube_terms(n, p)
        f = lowrank.rhs_tucker("cube", 0.0, n, p)
        x = fullcg.solve_direct(terms, tucker.vec(tucker.full(f)))
        X = tucker.unvec(x, (n, n, n))
        xs, ws = bspline.quadrature(n_el, p)
        B = bspline.dirichlet_basis(n_el, p, xs)
        uh = tucker.contract(X, [B.T, B.T, B.T])
        s = np.sin(np.pi * xs)
        ue = np.einsum("i,j,k->ijk", s, s, s)
        W = np.einsum("i,j,k->ijk", ws, ws, ws)
        errs.append(np.sqrt(np.sum(W * (uh - ue) ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 1 - 0.35


# ------------------------------------------------------------------------------------ eigenpairs
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_exact_generalized_eigen_identity(p):
    n = 14
    lam, U = fd.exact_eig(n, p)
    n_el = n - p + 2
    K, M = bspline.stiffness(n_el, p), bspline.mass(n_el, p)
    assert np.abs(K @ U - M @ U * lam).max() <= 1e-9 * lam.max()
    assert np.abs(U.T @ M @ U - np.eye(n)).max() <= 1e-10


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_approx_eigenpairs_structure(p):
    n_el = 16
    n = n_el + p - 2
    n1, n2 = fd.split_dims(n_el, p)
    assert n1 + n2 == n                                  # App. B dimensions
    U, lam = fd.approx_eig(n, p)
    assert np.allclose(lam[:n1], (np.arange(1, n1 + 1) * np.pi) ** 2)
    # V1 U1 interpolates the L2-normalised sines at the interpolation points
    x = fd.interpolation_points(n_el, p)
    E = bspline.dirichlet_basis(n_el, p, x).T
    j = np.arange(1, n1 + 1)
    assert np.abs(E @ U[:, :n1] - np.sqrt(2) * np.sin(np.pi * np.outer(x, j))).max() < 1e-10
    # the V1 columns satisfy the even-derivative conditions at both ends
    V1 = fd.v1_basis(n_el, p)
    for d in range(2, p, 2):
        for e in (0.0, 1.0):
            assert np.abs(bspline.dirichlet_basis(n_el, p, np.array([e]), d)[:, 0] @ V1).max() < 1e-8 * n_el ** d
    if n2 > 0:
        M, K = bspline.mass(n_el, p), bspline.stiffness(n_el, p)
        V2U2 = U[:, n1:]
        assert np.abs(V2U2.T @ M @ V1).max() < 1e-12    # M-orthogonal complement
        assert np.abs(V2U2.T @ M @ V2U2 - np.eye(n2)).max() < 1e-10
        assert np.abs(V2U2.T @ K @ V2U2 - np.diag(lam[n1:])).max() < 1e-8 * lam.max()


def test_table1_condition_numbers():
    g = json.load(open(os.path.join(GOLDEN, "table1.json")))
    for p in (2, 3, 4, 5):
        for i, n_el in enumerate(g["n_el"]):
            mp = fd.mp_value_fast(n_el, p)
            ref = g["M_P"][str(p)][i]
            if p == 2:
                assert abs(mp - n_el ** 2) <= 1e-9 * n_el ** 2   # Lambda1 = (j pi)^2 only
            # two significant digits in the printed table
            assert abs(mp - ref) <= 0.06 * ref, (p, n_el, mp, ref)


def test_full_and_fast_mp_agree():
    assert abs(fd.mp_value(20, 3) - fd.mp_value_fast(19, 3)) < 1e-9 * fd.mp_value(20, 3)


# ------------------------------------------------------------------------------------ exponential sums
@pytest.mark.parametrize("M", [50.0, 1.6e4, 2.38e4])
def test_expsum_meets_relative_bound(M):
    R, om, al = fd.expsum_for(M, 0.1)
    assert np.all(om > 0) and np.all(al > 0)                # Prop. 1: positive parameters
    assert fd.expsum_error(om, al, M, 20000) * M <= 0.1    # eq. estimate_prec_rel
    # the best approximation needs no more than Prop. 1's bound; the sinc sums stay within 3x of it
    rb = int(np.ceil(np.log(16 * M / 0.1) * np.log(8 * M) / np.pi ** 2))
    assert R <= 3 * rb


def test_preconditioner_diagonal_bound():
    # eq. prec_bound: ||D^-1||_inf ||D - D~||_inf <= eps_prec on the full diagonal
    P = fd.ApproxFD(10, 3)
    lam = P.lam
    L = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    Dt = sum(P.omega[j] / P.lmin * np.einsum("i,j,k->ijk", P.diag(j), P.diag(j), P.diag(j)) for j in range(P.RP))
    assert np.abs(1.0 / L - Dt).max() * L.max() <= 0.1


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_sine_factorization_is_exact_and_sparse(p):
    # App. B: V1 U1 = W U_dft diag(1/mu) with W the identity on interior rows (odd-reflection symmetry)
    n_el = 18
    n = n_el + p - 2
    n1, n2 = fd.split_dims(n_el, p)
    W, mu, Udft = fd.sine_factorization(n, p)
    U, _ = fd.approx_eig(n, p)
    assert np.abs(W @ Udft / mu - U[:, :n1]).max() <= 1e-11 * np.abs(U[:, :n1]).max()
    shift = n2 // 2
    for i in range(p, n - p):
        row = np.zeros(n1)
        row[i - shift] = 1.0
        assert np.abs(W[i] - row).max() < 1e-10
    assert np.count_nonzero(W) <= n1 + 4 * p * p
