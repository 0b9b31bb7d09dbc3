"""The benchmark's own workload at full size (twisted quarter annulus, p = 3, n = 128, mixed form, launched
as bench.py launches it): the returned Tucker solution is checked by the oracle's Tucker arithmetic against
the operator and right-hand side the library set up (exported to the host), so the true relative residual
is recomputed independently of the CUDA path."""
import numpy as np
import pytest

import synth
from oracle import tucker

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _terms_from_bands(ex, info):
    """Dense banded matrices from the exported band layout bands[((j*3+t)*(2p+1)+d)*n + i] = K_t^j[i, i+d-p]."""
    n, p, R = info.n, info.p, info.R
    bw = 2 * p + 1
    bands = np.asarray(ex["bands"]).reshape(R, 3, bw, n)
    terms = []
    for j in range(R):
        mats = []
        for t in range(3):
            K = np.zeros((n, n))
            for d in range(bw):
                for i in range(n):
                    jj = i + d - p
                    if 0 <= jj < n:
                        K[i, jj] = bands[j, t, d, i]
            mats.append(K)
        terms.append((float(ex["w"][j]), mats))
    return terms


def _oracle_residual(terms, f, x):
    """||f - A x|| by Alg. 1 steps 1-2 with eps = 0: QR of the factors, then ||core x_t R_t||."""
    y = tucker.add(f, tucker.scale(tucker.matvec(terms, x), -1.0))
    core, U = y
    Rs = [np.linalg.qr(U[m], mode="r") for m in range(3)]
    return float(np.linalg.norm(tucker.contract(core, Rs)))


@pytest.mark.parametrize("dtype_name,seed", [("MIXED", 7), ("MIXED", 8)])
def test_full_size_solution_residual(dtype_name, seed):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_00632_gb300 import api, lib
    dt = getattr(lib, dtype_name)
    n, p, rc = 128, 3, 96
    pb = api.tpcg_setup(lib.GEOM_TWIST, synth.amp_from_seed(seed), p, n, dt)
    ctx = api.Ctx(n, api.max_cols_for(pb.info, rc, dt), rc, dt)
    x = api.Tucker(n, cap=rc, core_cap=rc ** 3, dtype=dt)
    st = api.tpcg_solve(pb, ctx, x, tol=1e-6, rank_cap=rc, stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    assert st.status == 0
    X = x.to_numpy()
    ex = pb.export()
    info = pb.info
    terms = _terms_from_bands(ex, info)
    rf = tuple(info.rf)
    f = (np.asarray(ex["f_core"]).reshape(rf, order="F"),
         [np.asarray(ex[f"f_U{t}"]).reshape(n, rf[t], order="F") for t in range(3)])
    nf = tucker.norm(f)
    assert abs(nf - info.norm_f) <= 1e-12 * nf
    rel = _oracle_residual(terms, f, X) / nf
    assert rel <= 1e-6
    assert abs(rel - st.true_rel_res) <= 1e-9 + 1e-6 * rel
