"""Elasticity block system (Sec. 5.3) on the GPU against the elasticity oracle: block products, residual,
block-diagonal preconditioner, block TPCG (FP64 and FP32), and the library's own setup."""
import functools

import numpy as np
import pytest

import synth
from oracle import elasticity, fullcg, tucker
from oracle import tpcg as otp
from tests.gpu_helpers import oracle_problem, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LAM, MU = 0.3 / 0.52, 1.0 / 2.6
FORCE = (0.1, 0.2, -1.0)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api as a
    from paper_2306_00632_gb300 import lib
    lib.load()
    return a


@functools.lru_cache(maxsize=None)
def _oracle(kind, amp, n, p, bc=(0, 0)):
    blocks = elasticity.operator_blocks(kind, amp, n, p, LAM, MU, bc=bc)
    f = elasticity.rhs(kind, amp, n, p, FORCE, bc=bc)
    tables = oracle_problem("cube", 0.0, n, p, bc)[3]
    P = elasticity.BlockFD(n, p, LAM, MU, base=oracle_problem("cube", 0.0, n, p, bc)[2], bc=bc)
    return blocks, f, tables, P


def _gpu(api, kind, amp, n, p, dtype=0, bc=(0, 0)):
    blocks, f, tables, _ = _oracle(kind, amp, n, p, bc)
    return api.tpcg_elast_create(n, p, blocks, f, tables, LAM, MU, dtype=dtype)


def _bfull(X):
    return [tucker.full(x) for x in X]


def _brel(A, B):
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(A, B)))
    den = np.sqrt(sum(np.sum(b ** 2) for b in B))
    return num / den


def test_block_apply_and_residual(api):
    n, p, amp = 10, 2, 0.21
    blocks, f, _, _ = _oracle("twist", amp, n, p)
    e = _gpu(api, "twist", amp, n, p)
    X = [synth.random_tucker((n, n, n), r, seed=50 + i) for i, r in enumerate([(3, 2, 4), (2, 2, 2), (1, 3, 2)])]
    x = [api.Tucker.from_numpy(c, F) for c, F in X]
    cap = 1 + sum(e.R) * 4
    y = [api.Tucker(n, cap=cap, core_cap=64) for _ in range(3)]
    api.elast_apply(e, x, y)
    got = [tucker.full(yi.to_numpy(others=x)) for yi in y]
    ref = _bfull(elasticity.bmatvec(blocks, X))
    assert _brel(got, ref) < 1e-12
    api.elast_residual(e, x, y)
    # the residual starts from a copy of f_i in y_i's own buffers (factors orthonormalised by the library)
    got = [tucker.full(yi.to_numpy(others=x)) for yi in y]
    ref = _bfull([tucker.add(f[i], tucker.scale(elasticity.bmatvec(blocks, X)[i], -1.0)) for i in range(3)])
    assert _brel(got, ref) < 1e-12


def test_block_preconditioner(api):
    n, p, amp = 12, 3, 0.1
    _, _, _, P = _oracle("twist", amp, n, p)
    e = _gpu(api, "twist", amp, n, p)
    S = [synth.random_tucker((n, n, n), (2, 3, 2), seed=60 + i) for i in range(3)]
    s = [api.Tucker.from_numpy(c, F) for c, F in S]
    ctx = api.Ctx(n, e.RP * 4 + 8, 8)
    v = [api.Tucker(n, cap=e.RP * 4 + 8, core_cap=1) for _ in range(3)]
    api.elast_precond(e, ctx, s, v)
    got = [tucker.full(vi.to_numpy(others=s)) for vi in v]
    assert _brel(got, _bfull(P.apply(S))) < 1e-11


def _solve(api, e, n, rc, dtype=0, **kw):
    cap = max(max(sum(e.R[3 * i:3 * i + 3]) * rc + 4 for i in range(3)), e.RP * rc)
    ctx = api.Ctx(n, cap, rc, dtype)
    x = [api.Tucker(n, cap=rc, core_cap=rc ** 3, dtype=dtype) for _ in range(3)]
    st = api.elast_solve(e, ctx, x, rank_cap=rc, **kw)
    return st, [xi.to_numpy() for xi in x]


def test_block_tpcg_matches_oracle_and_direct_solve(api):
    n, p, amp = 8, 2, 0.21
    blocks, f, _, P = _oracle("twist", amp, n, p)
    e = _gpu(api, "twist", amp, n, p)
    st, X = _solve(api, e, n, n, tol=1e-8)
    assert st.status == 0 and st.true_rel_res <= 1e-8
    xo, info = elasticity.tpcg(blocks, f, P.apply, otp.Params(tol=1e-8))
    assert abs(st.iters - info["iters"]) <= 3
    A = elasticity.assemble(blocks)
    fv = elasticity.bvec(f)
    xg = elasticity.bvec(X)
    assert np.linalg.norm(fv - A @ xg) <= 2e-8 * np.linalg.norm(fv)
    assert rel(xg, elasticity.bvec(xo)) < 1e-6


def test_block_tpcg_f32(api):
    n, p, amp = 10, 3, 0.15
    blocks, f, _, _ = _oracle("twist", amp, n, p)
    e = _gpu(api, "twist", amp, n, p, dtype=1)
    # FP32 throughout: the recomputed residual carries FP32 cancellation (about 1e-7 kappa), so the FP32 form
    # is run to 2e-3 and checked against the assembled FP64 system
    st, X = _solve(api, e, n, n, dtype=1, tol=2e-3, max_it=200)
    assert st.status == 0
    A = elasticity.assemble(blocks)
    fv = elasticity.bvec(f)
    assert np.linalg.norm(fv - A @ elasticity.bvec(X)) <= 5e-3 * np.linalg.norm(fv)


def test_library_setup_matches_oracle_operator(api):
    from paper_2306_00632_gb300 import lib
    n, p, amp = 10, 3, 0.27
    blocks, f, _, _ = _oracle("twist", amp, n, p)
    e = api.tpcg_elast_setup(lib.GEOM_TWIST, amp, p, n, LAM, MU, FORCE)
    assert e.R == [len(blocks[i][j]) for i in range(3) for j in range(3)]
    X = [synth.random_tucker((n, n, n), (2, 2, 2), seed=70 + i) for i in range(3)]
    x = [api.Tucker.from_numpy(c, F) for c, F in X]
    y = [api.Tucker(n, cap=1 + sum(e.R) * 2, core_cap=1) for _ in range(3)]
    api.elast_apply(e, x, y)
    got = [tucker.full(yi.to_numpy(others=x)) for yi in y]
    # two independent constructions of the same coefficients (C++ and numpy): agreement to the
    # approximation tolerance of the Chebyshev step, not to rounding
    assert _brel(got, _bfull(elasticity.bmatvec(blocks, X))) < 1e-7
    assert abs(e.norm_f - elasticity.bnorm(f)) <= 1e-7 * elasticity.bnorm(f)


@pytest.mark.parametrize("bc", [(0, 1), (1, 0)])
def test_traction_free_faces(api, bc):
    # Neumann flags: the faces eta_t = 1 (or 0) traction-free for every component.  The library's own setup
    # against the oracle's operator and load, and block TPCG on oracle-built blocks against the direct solve.
    from paper_2306_00632_gb300 import lib
    n, p, amp = 10, 3, 0.27
    blocks, f, _, _ = _oracle("twist", amp, n, p, bc)
    e = api.tpcg_elast_setup(lib.GEOM_TWIST, amp, p, n, LAM, MU, FORCE, bc=bc)
    assert e.R == [len(blocks[i][j]) for i in range(3) for j in range(3)]
    X = [synth.random_tucker((n, n, n), (2, 2, 2), seed=80 + i) for i in range(3)]
    x = [api.Tucker.from_numpy(c, F) for c, F in X]
    y = [api.Tucker(n, cap=1 + sum(e.R) * 2, core_cap=1) for _ in range(3)]
    api.elast_apply(e, x, y)
    got = [tucker.full(yi.to_numpy(others=x)) for yi in y]
    assert _brel(got, _bfull(elasticity.bmatvec(blocks, X))) < 1e-7
    assert abs(e.norm_f - elasticity.bnorm(f)) <= 1e-7 * elasticity.bnorm(f)
    n, p, amp = 8, 2, 0.21
    blocks, f, _, P = _oracle("twist", amp, n, p, bc)
    eg = _gpu(api, "twist", amp, n, p, bc=bc)
    st, Xg = _solve(api, eg, n, n, tol=1e-8, max_it=300)
    assert st.status == 0 and st.true_rel_res <= 1e-8
    A = elasticity.assemble(blocks)
    fv = elasticity.bvec(f)
    import scipy.sparse.linalg as spla
    xd = spla.spsolve(A.tocsc(), fv)
    assert rel(elasticity.bvec(Xg), xd) < 1e-6
