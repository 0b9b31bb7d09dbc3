"""Pins of the oracle's Neumann-end variant of the preconditioner (App. B, last part) and of the spaces with
Neumann ends it lives on.  bc = (k0, k1): 1 = Neumann, 0 = Dirichlet at 0 and 1, the same in every direction.
CPU only.

What fixes each value here is the mathematics, not the oracle: the continuous eigenvalues of -u'' with the
end conditions ((j - k0/2 - k1/2) pi)^2, the counts of App. B, derivatives evaluated from the B-spline
recursion, a manufactured solution's optimal rate, a direct solve."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import bspline, fd, fullcg, geometry, lowrank, tpcg, tucker

MIXED = [(0, 1), (1, 0)]
ALL = [(0, 0), (0, 1), (1, 0), (1, 1)]


@pytest.mark.parametrize("bc", ALL)
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_space_keeps_the_neumann_end_functions(bc, p):
    n_el = 9
    B = bspline.bc_basis(n_el, p, np.array([0.0, 1.0]), 0, bc)
    assert B.shape[0] == n_el + p - 2 + bc[0] + bc[1]
    # a Dirichlet end: every function vanishes there; a Neumann end: the kept end function is 1 there
    for end, k in enumerate(bc):
        col = B[:, end]
        if k == 0:
            assert np.abs(col).max() == 0.0
        else:
            assert abs(col.sum() - 1.0) < 1e-14 and np.count_nonzero(col) == 1
    # the stiffness has the constant in its kernel exactly when both ends are Neumann (partition of unity)
    K = bspline.stiffness(n_el, p, bc)
    k1 = np.abs(K @ np.ones(K.shape[0])).max()
    assert (k1 < 1e-12) == (bc == (1, 1))


@pytest.mark.parametrize("bc", ALL)
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_discrete_eigenvalues_approach_the_shifted_continuous_ones(bc, p):
    # -u'' = lambda u on (0, 1), u = 0 at Dirichlet ends, u' = 0 at Neumann ends: lambda_j = ((j - s) pi)^2,
    # s = (k0 + k1) / 2; the Galerkin pencil (K, M) reproduces the low ones to O(h^{2p})
    n_el = 32
    n = n_el + p - 2 + sum(bc)
    lam = np.sort(fd.exact_eig(n, p, bc)[0])
    s = 0.5 * (bc[0] + bc[1])
    for j in range(1, 5):
        exact = ((j - s) * np.pi) ** 2
        if exact == 0.0:
            assert abs(lam[j - 1]) < 1e-9
        else:
            assert abs(lam[j - 1] - exact) <= 1e-4 * exact
    # the approximate eigenvalues of App. B are exactly those continuous values on V_h,1
    n1, _ = fd.split_dims(n_el, p, bc)
    _, lt = fd.approx_eig(n, p, bc)
    assert np.allclose(lt[:n1], ((np.arange(1, n1 + 1) - s) * np.pi) ** 2, rtol=1e-14, atol=0)


@pytest.mark.parametrize("bc", ALL)
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_splitting_dimensions_and_interpolation_points(bc, p):
    n_el = 12
    n1, n2 = fd.split_dims(n_el, p, bc)
    assert n1 + n2 == n_el + p - 2 + sum(bc)
    if bc == (0, 0):   # the counts App. B prints for two Dirichlet ends
        assert (n1, n2) == ((n_el - 1, p - 1) if p % 2 else (n_el, p - 2))
    # as many interpolation points as functions in V_h,1: the breakpoints without the Dirichlet ends (odd p),
    # the span midpoints (even p)
    x = fd.interpolation_points(n_el, p, bc)
    if p % 2:
        brk = np.arange(n_el + 1) / n_el
        keep = np.ones(n_el + 1, bool)
        keep[0], keep[-1] = bc[0] == 1, bc[1] == 1
        assert np.array_equal(x, brk[keep])
    else:
        assert np.allclose(x, (np.arange(n_el) + 0.5) / n_el)
    assert x.size == n1


@pytest.mark.parametrize("bc", ALL)
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_v1_columns_meet_the_end_conditions(bc, p):
    # V_h,1: odd derivatives up to p - 1 vanish at a Neumann end, even ones (from the second) at a Dirichlet end
    n_el = 14
    n1, _ = fd.split_dims(n_el, p, bc)
    V1 = fd.v1_basis(n_el, p, bc)
    assert np.linalg.matrix_rank(V1) == n1
    h = 1.0 / n_el
    for end, k in enumerate(bc):
        e = np.array([float(end)])
        orders = range(1, p, 2) if k == 1 else range(2, p, 2)
        for d in orders:
            vals = bspline.bc_basis(n_el, p, e, d, bc)[:, 0] @ V1
            assert np.abs(vals).max() < 1e-9 * h ** -d, (end, d)
        # and V_h,1 is no smaller than those conditions allow: the other order of the same parity class
        # (first derivative at a Dirichlet end) is not forced to vanish
        if k == 0 and p >= 2:
            assert np.abs(bspline.bc_basis(n_el, p, e, 1, bc)[:, 0] @ V1).max() > 1e-3


@pytest.mark.parametrize("bc", MIXED + [(1, 1)])
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_approx_eigenvectors_interpolate_the_shifted_sinusoids(bc, p):
    n_el = 16
    n = n_el + p - 2 + sum(bc)
    n1, n2 = fd.split_dims(n_el, p, bc)
    U, lam = fd.approx_eig(n, p, bc)
    x = fd.interpolation_points(n_el, p, bc)
    E = bspline.bc_basis(n_el, p, x, 0, bc).T
    s = 0.5 * (bc[0] + bc[1])
    w = (np.arange(1, n1 + 1) - s) * np.pi
    c = np.where(w == 0.0, 1.0, np.sqrt(2.0))            # L2-normalised on [0, 1]
    expect = c * np.sin(np.outer(x, w) + bc[0] * np.pi / 2)
    assert np.abs(E @ U[:, :n1] - expect).max() < 1e-10
    # the interpolants have zero slope at the Neumann ends
    for end, k in enumerate(bc):
        if k == 1:
            d1 = bspline.bc_basis(n_el, p, np.array([float(end)]), 1, bc)[:, 0] @ U[:, :n1]
            assert np.abs(d1).max() < 1e-8 * n_el
    if n2 > 0:
        M, K = bspline.mass(n_el, p, bc), bspline.stiffness(n_el, p, bc)
        V1 = fd.v1_basis(n_el, p, bc)
        V2U2 = U[:, n1:]
        assert np.abs(V2U2.T @ M @ V1).max() < 1e-12    # M-orthogonal complement
        assert np.abs(V2U2.T @ M @ V2U2 - np.eye(n2)).max() < 1e-10
        assert np.abs(V2U2.T @ K @ V2U2 - np.diag(lam[n1:])).max() < 1e-8 * lam.max()


@pytest.mark.parametrize("bc", MIXED)
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_sine_factorization_is_exact_and_sparse_with_neumann_ends(bc, p):
    n_el = 18
    n = n_el + p - 2 + sum(bc)
    n1, _ = fd.split_dims(n_el, p, bc)
    W, mu, Udft = fd.sine_factorization(n, p, bc)
    U, _ = fd.approx_eig(n, p, bc)
    assert np.abs(W @ Udft / mu - U[:, :n1]).max() <= 1e-11 * np.abs(U[:, :n1]).max()
    # interior rows: a unit vector at the interpolation point that is the function's centre
    x = fd.interpolation_points(n_el, p, bc)
    kn = bspline.open_uniform_knots(n_el, p)
    for i in range(p + 1, n - p - 1):
        f = i + (1 - bc[0])                            # full B-spline index
        centre = 0.5 * (kn[f] + kn[f + p + 1])
        row = np.zeros(n1)
        row[int(np.argmin(np.abs(x - centre)))] = 1.0
        assert np.abs(W[i] - row).max() < 1e-10, i
    assert np.count_nonzero(W) <= n1 + 4 * p * p


@pytest.mark.parametrize("p", [2, 3, 4])
def test_neumann_fd_is_spectrally_equivalent_on_the_cube(p):
    # the preconditioner P~ = U~^-T (Lambda~ (+) Lambda~ (+) Lambda~) U~^-1 against A on the unit cube: the
    # spread of the spectrum of P~^-1 A stays within twice that of the Dirichlet case and below 10
    def kappa(bc):
        n_el = 10
        n = n_el + p - 2 + sum(bc)
        M, K = bspline.mass(n_el, p, bc), bspline.stiffness(n_el, p, bc)
        U, lam = fd.approx_eig(n, p, bc)
        Kt, Mt = U.T @ K @ U, U.T @ M @ U
        A = np.kron(np.kron(Kt, Mt), Mt) + np.kron(np.kron(Mt, Kt), Mt) + np.kron(np.kron(Mt, Mt), Kt)
        d = 1.0 / np.sqrt((lam[:, None, None] + lam[None, :, None] + lam[None, None, :]).ravel())
        ev = scipy.linalg.eigvalsh(d[:, None] * A * d[None, :])
        return ev.max() / ev.min()
    k_dd = kappa((0, 0))
    for bc in MIXED:
        k = kappa(bc)
        assert k <= 2.0 * k_dd and k < 10.0


def test_singular_all_neumann_preconditioner_rejected():
    with pytest.raises(ValueError):
        fd.ApproxFD(12, 3, bc=(1, 1))


@pytest.mark.parametrize("bc", MIXED)
@pytest.mark.parametrize("p", [2, 3])
def test_mixed_bc_manufactured_solution_converges_at_optimal_rate(bc, p):
    # unit cube, u = s(x) s(y) s(z), s(t) = sin(w t + k0 pi/2): zero at the Dirichlet faces, zero normal
    # derivative at the Neumann faces; L2 error of the Galerkin solution ~ h^{p+1}
    errs = []
    for n_el in (4, 8):
        n = n_el + p - 2 + sum(bc)
        terms = lowrank.cube_terms(n, p, bc)
        f = lowrank.rhs_tucker("cube", 0.0, n, p, bc=bc)
        x = fullcg.solve_direct(terms, tucker.vec(tucker.full(f)))
        X = tucker.unvec(x, (n, n, n))
        xs, ws = bspline.quadrature(n_el, p)
        B = bspline.bc_basis(n_el, p, xs, 0, bc)
        uh = tucker.contract(X, [B.T, B.T, B.T])
        w = (1.0 - 0.5 * sum(bc)) * np.pi
        s = np.sin(w * xs + bc[0] * np.pi / 2)
        ue = np.einsum("i,j,k->ijk", s, s, s)
        W = np.einsum("i,j,k->ijk", ws, ws, ws)
        errs.append(np.sqrt(np.sum(W * (uh - ue) ** 2)))
    assert np.log2(errs[0] / errs[1]) > p + 1 - 0.35
    # the oracle's closed form of the 1-D factor is the same function
    assert np.allclose(geometry.cube_solution_1d(xs, bc)[0], s)


@pytest.mark.parametrize("bc", MIXED)
def test_tpcg_twist_with_neumann_faces_against_direct_solve(bc):
    n, p = 12, 3
    amp = synth.amp_from_seed(7)
    terms = lowrank.operator_terms("twist", amp, n, p, bc=bc)
    f = lowrank.rhs_tucker("twist", amp, n, p, bc=bc)
    P = fd.ApproxFD(n, p, bc=bc)
    x, info = tpcg.tpcg(terms, f, P.apply, tpcg.Params(tol=1e-6))
    fv = tucker.vec(tucker.full(f))
    xe = fullcg.solve_direct(terms, fv)
    xv = tucker.vec(tucker.full(x))
    assert info["res"] <= 1e-6
    assert np.linalg.norm(xv - xe) <= 1e-5 * np.linalg.norm(xe)
    assert 5 <= info["iters"] <= 60
