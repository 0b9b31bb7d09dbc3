"""Non-homogeneous Dirichlet data (the Remark in Sec. 3) through the CUDA solver.  The oracle's lifting (L2
projection c of the extension of g on the full tensor B-spline space; lifted right-hand side
f - A_(I,all) c + A_(I,I) c_I) is the right-hand side of a problem whose operator and preconditioner the library
sets up (twisted annulus, p = 3, harmonic g = x^2 + y^2 - 2 z^2 + x y, f = 0).  FP64 Alg. 5 on the GPU solves for
the interior coefficients x, and u_h = c + E(x - c_I) on the host.  The GPU's u_h equals the oracle's own lifted
solve, and its L2 error against g falls at the optimal rate h^(p+1) = h^4 (16 per halving)."""
import numpy as np
import pytest

import synth
from oracle import lifting, lowrank, tucker
from tests.test_oracle_lifting import _l2_error, _solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api, lib
    lib.load()
    return api, lib


def test_lifted_solve_on_the_gpu(mods):
    api, lib = mods
    p, amp = 3, synth.amp_from_seed(7)
    G = lambda x, y, z: x * x + y * y - 2 * z * z + x * y
    errs = []
    for n_el in (4, 8):
        n = n_el + p - 2
        terms = lowrank.operator_terms("twist", amp, n, p)
        terms_full = lowrank.operator_terms("twist", amp, n, p, trial="full")
        c = lifting.projection_coefficients(G, "twist", amp, n, p)
        f0 = (np.zeros((1, 1, 1)), [np.zeros((n, 1))] * 3)
        fl = lifting.lifted_rhs(terms_full, terms, f0, c)
        base = api.tpcg_setup(lib.GEOM_TWIST, amp, p, n, lib.F64)
        ex = base.export()
        ex["v2u2"] = ex["v2u2"][: n * base.info.n2]
        pb = api.problem_from_export(ex, base.info, dtype=lib.F64, pinned=False, rhs=fl)
        ctx = api.Ctx(n, api.max_cols_for(pb.info, n, lib.F64), n, lib.F64)
        x = api.Tucker(n, cap=n, core_cap=n ** 3, dtype=lib.F64)
        st = api.tpcg_solve(pb, ctx, x, tol=1e-11, rank_cap=n)
        torch.cuda.synchronize()
        assert st.status == 0
        u_gpu = lifting.full_solution(c, x.to_numpy())
        u_orc, _, _ = _solve("twist", amp, n, p, G, None, tol=1e-11)
        ref = tucker.full(u_orc)
        # the library's operator approximates the geometry to 1e-8, like the oracle's
        assert np.linalg.norm(tucker.full(u_gpu) - ref) <= 1e-7 * np.linalg.norm(ref)
        e, gn = _l2_error(u_gpu, G, "twist", amp, n_el, p)
        errs.append(e / gn)
    assert errs[1] < 3e-5
    assert errs[0] / errs[1] >= 8.0, errs
