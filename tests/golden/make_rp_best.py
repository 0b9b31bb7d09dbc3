"""Writes rp_best_table1.json: the oracle's best-exponential-sum R_P (eq. estimate_prec_rel, eps_prec = 0.1)
for the 16 M_P values printed in Table 1, with E_R M_P for R = R_P and R = R_P - 1.  Calls only oracle/.
Run from the repository root: python tests/golden/make_rp_best.py  (about half an hour on 8 cores)."""
import json
import pathlib
import sys

ROOT = pathlib.Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import expsum  # noqa: E402

here = pathlib.Path(__file__).parent
t1 = json.loads((here / "table1.json").read_text())
out = {"source": "oracle/expsum.py rp_best(M_P, 0.1) on Table 1's printed M_P (written by make_rp_best.py)",
       "n_el": t1["n_el"], "R_P": {}, "EM_at_RP": {}, "EM_at_RP_minus_1": {}}
for p in ("2", "3", "4", "5"):
    out["R_P"][p], out["EM_at_RP"][p], out["EM_at_RP_minus_1"][p] = [], [], []
    for M in t1["M_P"][p]:
        R, _, _, E, E_prev = expsum.rp_best(M, 0.1)
        out["R_P"][p].append(R)
        out["EM_at_RP"][p].append(round(E * M, 6))
        out["EM_at_RP_minus_1"][p].append(round(E_prev * M, 6))
        print(p, M, R, E * M, E_prev * M, flush=True)
(here / "rp_best_table1.json").write_text(json.dumps(out, indent=1) + "\n")
