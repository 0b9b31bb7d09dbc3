"""The library's host setup (C++, tpcg_setup_host: no GPU call) against the oracle's construction, on the CPU:
operator action, right-hand side, App. B tables (Lambda~, mu, W, V2 U2) and M_P, for Dirichlet and Neumann
ends, odd and even degree, cube and twisted annulus.  The two are independent constructions (the C++ de Boor
table and Chebyshev interpolation against the oracle's recursion and dense Chebyshev solve), so the operator
and rhs agree to the approximation tolerance of the Chebyshev step, the App. B tables to rounding."""
import numpy as np
import pytest

import synth
from oracle import fd, lowrank, tucker

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_2306_00632_gb300 import api as a
    from paper_2306_00632_gb300 import lib
    lib.load()
    # the sinc sums are the oracle's default; the best sums are checked separately (test_abi, GPU tests)
    a.set_option(lib.OPT_EXPSUM_BEST, 0)
    yield a
    a.set_option(lib.OPT_EXPSUM_BEST, 1)


def _dense(band, n, p):
    K = np.zeros((n, n))
    for d in range(2 * p + 1):
        for i in range(n):
            j = i + d - p
            if 0 <= j < n:
                K[i, j] = band[d, i]
    return K


@pytest.mark.parametrize("kind,amp,n,p,bc", [
    ("cube", 0.0, 12, 2, (0, 0)), ("twist", 0.1, 13, 3, (0, 0)), ("twist", 0.1, 14, 3, (0, 1)),
    ("twist", 0.05, 15, 4, (1, 0)), ("cube", 0.0, 16, 5, (0, 1)), ("twist", 0.2, 14, 5, (1, 0))])
def test_host_setup_matches_the_oracle(api, kind, amp, n, p, bc):
    from paper_2306_00632_gb300 import lib
    kid = lib.GEOM_CUBE if kind == "cube" else lib.GEOM_TWIST
    h = api.setup_host(kid, amp, p, n, bc=bc)
    info = h["info"]
    assert (info.k0, info.k1) == bc and info.n1 + info.n2 == n
    # App. B tables and M_P
    P = fd.ApproxFD(n, p, bc=bc)
    W, mu, _ = fd.sine_factorization(n, p, bc)
    assert np.allclose(h["lam"], P.lam, rtol=1e-12)
    assert np.allclose(h["mu"], mu, rtol=1e-11)
    Wc = np.zeros((n, info.n1))
    rp = h["w_rowptr"]
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            Wc[i, h["w_col"][e]] = h["w_val"][e]
    assert np.abs(Wc - W).max() <= 1e-10 * np.abs(W).max()
    if info.n2:
        assert np.abs(np.abs(h["v2u2"]) - np.abs(P.U[:, info.n1:])).max() <= 1e-9 * np.abs(P.U[:, info.n1:]).max()
    assert abs(info.MP - P.MP) <= 1e-10 * P.MP
    assert info.RP == P.RP                      # the same sinc-sum search
    # operator action and rhs
    terms = lowrank.operator_terms(kind, amp, n, p, bc=bc)
    X = synth.random_tucker((n, n, n), (3, 2, 3), seed=5)
    got = sum(h["w"][j] * tucker.contract(tucker.full(X), [_dense(h["bands"][j, t], n, p) for t in range(3)])
              for j in range(info.R))
    ref = tucker.full(tucker.matvec(terms, X))
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
    f = lowrank.rhs_tucker(kind, amp, n, p, bc=bc)
    F = tucker.full((h["f_core"], h["f_U"]))
    assert np.linalg.norm(F - tucker.full(f)) <= 1e-9 * np.linalg.norm(tucker.full(f))


def test_host_setup_refuses_neumann_everywhere(api):
    from paper_2306_00632_gb300 import lib
    with pytest.raises(RuntimeError):
        api.setup_host(lib.GEOM_CUBE, 0.0, 3, 14, bc=(1, 1))
