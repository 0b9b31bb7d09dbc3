"""Oracle pins of the non-homogeneous Dirichlet lifting (the Remark in Sec. 3, oracle/lifting.py).

1. A solution inside the discrete space is reproduced exactly: on the unit cube with p = 2 the polynomial
   u = (1 + x + x^2)(2 - y)(1 + z - z^2) is a spline of the full space, so with f = -Laplace(u) and g = u on
   the boundary the lifted system's solution plus the boundary coefficients must equal u's coefficients (to
   the solver's tolerance).  A wrong sign of the correction, a shifted boundary column or a wrong restriction
   breaks it.
2. On the twisted quarter annulus (p = 3) with the harmonic g = x^2 + y^2 - 2 z^2 + x y and f = 0, the L2
   error of u_h against g on the physical domain falls at the optimal rate h^(p+1) when the mesh is halved.
"""
import numpy as np

import synth
from oracle import bspline, fd, geometry, lifting, lowrank, tpcg, tucker


def _solve(kind, amp, n, p, G, f_fun, tol=1e-10):
    terms = lowrank.operator_terms(kind, amp, n, p)
    terms_full = lowrank.operator_terms(kind, amp, n, p, trial="full")
    c = lifting.projection_coefficients(G, kind, amp, n, p)
    if f_fun is None:
        f = (np.zeros((1, 1, 1)), [np.zeros((n, 1))] * 3)
    else:
        f = lifting.rhs_of(f_fun, kind, amp, n, p)
    fl = lifting.lifted_rhs(terms_full, terms, f, c)
    P = fd.ApproxFD(n, p)
    x, info = tpcg.tpcg(terms, fl, P.apply, tpcg.Params(tol=tol, eps_min=tol * 1e-2))
    return lifting.full_solution(c, x), c, info


def test_lifting_reproduces_a_solution_in_the_spline_space():
    n_el, p = 6, 2
    n = n_el + p - 2
    u = lambda x, y, z: (1 + x + x * x) * (2 - y) * (1 + z - z * z)
    lap = lambda x, y, z: 2 * (2 - y) * (1 + z - z * z) - 2 * (1 + x + x * x) * (2 - y)
    uh, c, info = _solve("cube", 0.0, n, p, u, lambda x, y, z: -lap(x, y, z))
    assert info["res"] <= 1e-10
    ref = tucker.full(c)                      # u is in the space: its projection is u itself
    assert np.linalg.norm(tucker.full(uh) - ref) <= 1e-8 * np.linalg.norm(ref)
    # the lifting was not trivial: the boundary data alone are far from u
    cb = tucker.full(lifting.full_solution(c, (np.zeros((1, 1, 1)), [np.zeros((n, 1))] * 3)))
    assert np.linalg.norm(cb - ref) > 0.3 * np.linalg.norm(ref)


def _l2_error(uh, G, kind, amp, n_el, p):
    xs, ws = bspline.quadrature(n_el, p)
    Bf = bspline.basis(bspline.open_uniform_knots(n_el, p), p, xs, 0)
    core, U = uh
    vals = tucker.contract(core, [Bf.T @ U[t] for t in range(3)])
    e1, e2, e3 = np.meshgrid(xs, xs, xs, indexing="ij")
    det = np.linalg.det(geometry.twist_jacobian(e1, e2, e3, amp))
    w = ws[:, None, None] * ws[None, :, None] * ws[None, None, :] * np.abs(det)
    g = G(*lifting.physical_points(kind, amp, e1, e2, e3))
    return np.sqrt(np.sum(w * (vals - g) ** 2)), np.sqrt(np.sum(w * g * g))


def test_lifting_optimal_rate_on_the_twisted_annulus():
    p, amp = 3, synth.amp_from_seed(7)
    G = lambda x, y, z: x * x + y * y - 2 * z * z + x * y
    errs = []
    for n_el in (4, 8):
        n = n_el + p - 2
        uh, _, info = _solve("twist", amp, n, p, G, None, tol=1e-11)
        e, gn = _l2_error(uh, G, "twist", amp, n_el, p)
        errs.append(e / gn)
    assert errs[1] < 3e-5
    assert errs[0] / errs[1] >= 8.0           # h^(p+1) = 16 per halving at p = 3
