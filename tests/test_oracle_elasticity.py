"""Pins of the elasticity oracle (Sec. 5.3) against the mathematics: a manufactured solution on the cube
(Galerkin error at the optimal rate), translations in the kernel of the unconstrained form, symmetry and
positivity of the block matrix, the preconditioner bound, and block TPCG against the direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bspline, elasticity, fd, lowrank, tucker
from oracle import tpcg as otp

LAM, MU = 0.3 / 0.52, 1.0 / 2.6      # E = 1, nu = 0.3 (the paper's Lame parameters)


def _cube_manufactured_load(n_el, p, a):
    """Load of f = -mu Lap u - (lam + mu) grad div u for u_i = a_i sin(pi x) sin(pi y) sin(pi z), computed
    from the closed-form derivatives of the sines and 1-D Gauss quadrature (independent of the oracle's
    coefficient code)."""
    xs, ws = bspline.quadrature(n_el, p)
    B = bspline.dirichlet_basis(n_el, p, xs)
    Ls = (B * ws) @ np.sin(np.pi * xs)
    Lc = (B * ws) @ np.cos(np.pi * xs)
    F = []
    for j in range(3):
        # f_j = pi^2 [ (4 mu + lam) a_j s s s - (lam + mu) sum_{i != j} a_i c_i c_j s_k ]
        t = (4 * MU + LAM) * a[j] * np.einsum("i,j,k->ijk", Ls, Ls, Ls)
        for i in range(3):
            if i == j:
                continue
            vecs = [Ls, Ls, Ls]
            vecs[i] = Lc
            vecs[j] = Lc
            t = t - (LAM + MU) * a[i] * np.einsum("i,j,k->ijk", *vecs)
        F.append(np.pi ** 2 * t)
    return F


@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_elasticity_solution_converges_at_optimal_rate(p):
    a = (1.0, -0.5, 0.25)
    errs = []
    for n_el in (4, 8):
        n = n_el + p - 2
        blocks = elasticity.operator_blocks("cube", 0.0, n, p, LAM, MU)
        A = elasticity.assemble(blocks)
        F = _cube_manufactured_load(n_el, p, a)
        rhs = np.concatenate([tucker.vec(Fj) for Fj in F])
        x = spla.spsolve(A.tocsc(), rhs)
        xs, ws = bspline.quadrature(n_el, p)
        B = bspline.dirichlet_basis(n_el, p, xs)
        s = np.sin(np.pi * xs)
        W = np.einsum("i,j,k->ijk", ws, ws, ws)
        e2 = 0.0
        for j in range(3):
            X = tucker.unvec(x[j * n ** 3:(j + 1) * n ** 3], (n, n, n))
            uh = tucker.contract(X, [B.T, B.T, B.T])
            e2 += np.sum(W * (uh - a[j] * np.einsum("i,j,k->ijk", s, s, s)) ** 2)
        errs.append(np.sqrt(e2))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 1 - 0.35


def test_translations_are_in_the_kernel_without_boundary_conditions():
    # with the full B-spline basis (no Dirichlet cut) a constant displacement has zero strain: A_ij 1 = 0
    n_el, p, amp = 4, 2, 0.27
    xs, ws = bspline.quadrature(n_el, p)
    kn = bspline.open_uniform_knots(n_el, p)
    B0 = bspline.basis(kn, p, xs, 0)
    B1 = bspline.basis(kn, p, xs, 1)
    xc = lowrank.cheb_points()
    e1, e2, e3 = np.meshgrid(xc, xc, xc, indexing="ij")
    C = elasticity.coefficients("twist", amp, LAM, MU, e1, e2, e3)
    N = B0.shape[0]
    ones = np.ones(N ** 3)
    for i in range(3):
        for j in range(3):
            y = np.zeros(N ** 3)
            for k in range(3):
                for l in range(3):
                    core, U = lowrank.tucker_of_samples(C[..., i, j, k, l], 1e-10)
                    g = [lowrank.cheb_eval(U[t], xs) for t in range(3)]
                    mats = []
                    for t in range(3):
                        Bi = B1 if t == l else B0
                        Bj = B1 if t == k else B0
                        mats.append([(Bi * (ws * g[t][:, a])) @ Bj.T for a in range(g[t].shape[1])])
                    Y = np.zeros((N, N, N))
                    X1 = np.ones((N, N, N))
                    for a1 in range(core.shape[0]):
                        for a2 in range(core.shape[1]):
                            for a3 in range(core.shape[2]):
                                c = core[a1, a2, a3]
                                if c != 0.0:
                                    Y += c * tucker.contract(X1, [mats[0][a1], mats[1][a2], mats[2][a3]])
                    y += tucker.vec(Y)
            scale = np.abs(C[..., i, j, :, :]).max() + 1e-300
            assert np.abs(y).max() <= 1e-9 * scale, (i, j)
    assert ones.size == N ** 3


def test_block_matrix_symmetric_positive_definite_on_twist():
    n, p = 6, 2
    A = elasticity.assemble(elasticity.operator_blocks("twist", 0.2, n, p, LAM, MU))
    D = A.toarray()
    assert np.abs(D - D.T).max() <= 1e-9 * np.abs(D).max()
    assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > 0.0


def test_block_preconditioner_bound_on_the_cube():
    # on the cube the diagonal blocks are the weighted Kronecker sums the block FD diagonalises: with the exact
    # eigenpairs (K U = M U Lambda) only the exponential sum approximates, so the spectrum of P~_i^-1 A_ii lies
    # in [1 - eps_prec, 1 + eps_prec] (eq. prec_bound) for every direction weighting
    n, p = 10, 2
    blocks = elasticity.operator_blocks("cube", 0.0, n, p, LAM, MU)
    base = fd.ApproxFD(n, p)
    base.lam, base.U = fd.exact_eig(n, p)
    P = elasticity.BlockFD(n, p, LAM, MU, base=base)
    from oracle import fullcg
    N = n ** 3
    for i in range(3):
        Aii = fullcg.assemble(blocks[i][i]).toarray()
        cols = []
        for e in range(N):
            v = np.zeros(N)
            v[e] = 1.0
            S = tucker.unvec(v, (n, n, n))
            Y = P.apply_one(i, (S, [np.eye(n)] * 3))
            cols.append(tucker.vec(tucker.full(Y)))
        Pinv = np.array(cols).T
        ev = np.linalg.eigvals(Pinv @ Aii).real
        assert ev.min() >= 1 - 0.1 - 1e-9 and ev.max() <= 1 + 0.1 + 1e-9, (i, ev.min(), ev.max())


def test_block_tpcg_matches_direct_solve():
    n, p, amp = 8, 2, 0.21
    blocks = elasticity.operator_blocks("twist", amp, n, p, LAM, MU)
    f = elasticity.rhs("twist", amp, n, p, (0.1, 0.2, -1.0))
    P = elasticity.BlockFD(n, p, LAM, MU)
    x, info = elasticity.tpcg(blocks, f, P.apply, otp.Params(tol=1e-8))
    A = elasticity.assemble(blocks)
    fv = elasticity.bvec(f)
    xd = spla.spsolve(A.tocsc(), fv)
    xv = elasticity.bvec(x)
    assert np.linalg.norm(fv - A @ xv) <= 2e-8 * np.linalg.norm(fv)
    assert np.linalg.norm(xv - xd) <= 1e-6 * np.linalg.norm(xd)
    assert info["iters"] < 100


# ------------------------------------------------------------------------------------ Neumann faces
def _outer(vecs):
    return np.einsum("i,j,k->ijk", *vecs)


def _neumann_manufactured_load(n_el, p, a, bc=(0, 1)):
    """Load of u_i = a_i S(x) S(y) S(z), S(t) = sin(pi t / 2), on the cube clamped at the faces eta_t = 0 and
    loaded by the traction g = sigma(u) n on the faces eta_t = 1: the body term int f . v with
    f = -mu Lap u - (lam + mu) grad div u, plus the face terms int g . v.  Closed-form derivatives of the
    sines and 1-D Gauss quadrature only (independent of the oracle's coefficient code)."""
    h = 0.5 * np.pi
    xs, ws = bspline.quadrature(n_el, p)
    B = bspline.bc_basis(n_el, p, xs, 0, bc)
    Ls = (B * ws) @ np.sin(h * xs)
    Lc = (B * ws) @ np.cos(h * xs)
    e1 = bspline.bc_basis(n_el, p, np.array([1.0]), 0, bc)[:, 0]    # test functions at eta = 1
    F = []
    for j in range(3):
        t = h * h * (4 * MU + LAM) * a[j] * _outer([Ls, Ls, Ls])
        for i in range(3):
            if i != j:
                v = [Ls, Ls, Ls]
                v[i], v[j] = Lc, Lc
                t = t - h * h * (LAM + MU) * a[i] * _outer(v)
        for d in range(3):   # face eta_d = 1, outward normal e_d; S(1) = 1, S'(1) = 0
            if j == d:       # normal traction lam div u = lam h sum_{k != d} a_k C(x_k) S(x_m)
                for k in range(3):
                    if k != d:
                        v = [Ls, Ls, Ls]
                        v[d], v[k] = e1, Lc
                        t = t + LAM * h * a[k] * _outer(v)
            else:            # shear traction mu d_j u_d = mu h a_d C(x_j) S(x_m)
                v = [Ls, Ls, Ls]
                v[d], v[j] = e1, Lc
                t = t + MU * h * a[d] * _outer(v)
        F.append(t)
    return F


@pytest.mark.parametrize("p", [2, 3])
def test_elasticity_with_neumann_faces_converges_at_optimal_rate(p):
    # Neumann flags (0, 1): clamped at eta_t = 0, traction data on eta_t = 1 (the natural condition the space
    # carries); the Galerkin error of the manufactured solution falls as h^{p+1}
    a = (1.0, -0.5, 0.25)
    bc = (0, 1)
    errs = []
    for n_el in (4, 8):
        n = n_el + p - 1
        blocks = elasticity.operator_blocks("cube", 0.0, n, p, LAM, MU, bc=bc)
        A = elasticity.assemble(blocks)
        F = _neumann_manufactured_load(n_el, p, a, bc)
        x = spla.spsolve(A.tocsc(), np.concatenate([tucker.vec(Fj) for Fj in F]))
        xs, ws = bspline.quadrature(n_el, p)
        B = bspline.bc_basis(n_el, p, xs, 0, bc)
        s = np.sin(0.5 * np.pi * xs)
        W = _outer([ws, ws, ws])
        e2 = 0.0
        for j in range(3):
            X = tucker.unvec(x[j * n ** 3:(j + 1) * n ** 3], (n, n, n))
            uh = tucker.contract(X, [B.T, B.T, B.T])
            e2 += np.sum(W * (uh - a[j] * _outer([s, s, s])) ** 2)
        errs.append(np.sqrt(e2))
    assert np.log2(errs[0] / errs[1]) > p + 1 - 0.35


@pytest.mark.parametrize("bc", [(0, 1), (1, 0)])
def test_neumann_faces_block_matrix_spd_and_tpcg_matches_direct_solve(bc):
    n, p, amp = 8, 2, 0.21
    blocks = elasticity.operator_blocks("twist", amp, n, p, LAM, MU, bc=bc)
    A = elasticity.assemble(blocks)
    D = A.toarray()
    assert np.abs(D - D.T).max() <= 1e-9 * np.abs(D).max()
    assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > 0.0     # clamped faces remove the rigid motions
    f = elasticity.rhs("twist", amp, n, p, (0.1, 0.2, -1.0), bc=bc)
    P = elasticity.BlockFD(n, p, LAM, MU, bc=bc)
    x, info = elasticity.tpcg(blocks, f, P.apply, otp.Params(tol=1e-8))
    fv = elasticity.bvec(f)
    xd = spla.spsolve(A.tocsc(), fv)
    xv = elasticity.bvec(x)
    assert np.linalg.norm(fv - A @ xv) <= 2e-8 * np.linalg.norm(fv)
    assert np.linalg.norm(xv - xd) <= 1e-6 * np.linalg.norm(xd)
    assert info["iters"] < 150    # 114 with traction-free faces at eta = 1: the block-diagonal FD sees no coupling
