"""Write tests/golden/ref_twist128_seed7.npz: the oracle's solution of the benchmark workload and the
oracle's iteration count on it.  Calls only oracle/ (and synth/ for the seeded amplitude).

Workload: twisted quarter annulus, p = 3, n = 128 dofs per direction, amplitude from seed 7, f = 1; the FD
preconditioner with the best exponential sums of Prop. 1 for this M_P (as the library's setup builds it).

Stored:
  * iters_tol6 / res_tol6: Alg. 5 (paper defaults, tol 1e-6) iterations to convergence, and the final
    relative residual;
  * core, U0, U1, U2: the solution of Alg. 5 run to tol 1e-10 with eps_min 1e-12, rounded by Alg. 1 to
    relative accuracy 1e-9 for storage (a reference whose own error is far below the 1e-6 solutions it is
    compared with);
  * mass: the 1-D B-spline mass matrix of the Dirichlet basis (Sec. 2.2), for L2 norms of the discrete
    function on the parametric cube, ||u_h||^2 = vec(C)^T (M (x) M (x) M) vec(C);
  * amp, n, p, tol_ref.

Runtime on 8 x86 cores: about 15 minutes.  Usage: python tests/golden/make_ref_twist128.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import bspline, expsum, fd, lowrank, rounding, tpcg, tucker  # noqa: E402

N, P, SEED = 128, 3, 7


def main(out=os.path.join(HERE, "ref_twist128_seed7.npz")):
    amp = synth.amp_from_seed(SEED)
    t0 = time.time()
    terms = lowrank.operator_terms("twist", amp, N, P)
    f = lowrank.rhs_tucker("twist", amp, N, P)
    _, om, al, _, _ = expsum.rp_best(fd.mp_value(N, P), 0.1)
    Pc = fd.ApproxFD(N, P, expsum=(om, al))
    print(f"setup {time.time() - t0:.1f}s: R = {len(terms)}, R_P = {Pc.RP}", flush=True)
    t0 = time.time()
    _, info6 = tpcg.tpcg(terms, f, Pc.apply, tpcg.Params(tol=1e-6))
    print(f"tol 1e-6: {info6['iters']} iterations, res {info6['res']:.3e}, {time.time() - t0:.1f}s", flush=True)
    t0 = time.time()
    x, info = tpcg.tpcg(terms, f, Pc.apply, tpcg.Params(tol=1e-10, eps_min=1e-12))
    print(f"tol 1e-10: {info['iters']} iterations, res {info['res']:.3e}, ranks {tucker.ranks(x)}, "
          f"{time.time() - t0:.1f}s", flush=True)
    core, U = rounding.t_rel(x, 1e-9)
    print(f"stored ranks {core.shape}", flush=True)
    n_el = N - P + 2
    np.savez_compressed(out, core=core, U0=U[0], U1=U[1], U2=U[2], mass=bspline.mass(n_el, P),
                        iters_tol6=info6["iters"], res_tol6=info6["res"], iters_ref=info["iters"],
                        res_ref=info["res"], amp=amp, n=N, p=P, tol_ref=1e-10)
    print("wrote", out)


if __name__ == "__main__":
    main()
