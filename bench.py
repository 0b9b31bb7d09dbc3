#!/usr/bin/env python
"""TPCG benchmark on GB300: solves/sec to relative residual 1e-6 (plus p50/p99 latency) for the
single deformed-geometry Poisson workload (twisted quarter annulus, p = 3, n = 128 dofs per direction).

One step = ``--concurrent`` (default 32) complete TPCG solves (Alg. 5 with Alg. 1, 2, 4; every hot-path
kernel) of resident problems of the same family (one seed each), run at once; the single-solve latency is
measured separately.  ``python bench.py --gpus N --steps K --warmup W`` prints one JSON line on rank 0.
``--impl reference`` times the FP64 CPU oracle on the host cores instead (a bounded sample).
Multi-GPU: independent replicas (one solve stream per GPU, no collective), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
# concurrent solves run on separate streams: give the device as many hardware work queues as it has
# (the default of 8 makes streams beyond the eighth share queues and wait on each other's kernels); this must
# be set before the CUDA context exists
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

N_DOF, DEGREE, SEED = 128, 3, 7
AMP = synth.amp_from_seed(SEED)
TOL = 1e-6
WORKLOAD = f"twisted quarter annulus Poisson, p={DEGREE}, n={N_DOF}/direction, amp={AMP:.4f} (seed {SEED})"
METRIC = "TPCG solves/sec to rel-residual 1e-6"
# the oracle's own solution of this workload (tol 1e-10, rounded to 1e-9) and its iteration count at tol 1e-6,
# written by tests/golden/make_ref_twist128.py (oracle only)
REF_FILE = os.path.join(ROOT, "tests", "golden", "ref_twist128_seed7.npz")


def oracle_reference():
    """The stored oracle data of the workload: iteration count at tol 1e-6 and the reference solution."""
    z = np.load(REF_FILE)
    return {"iters": int(z["iters_tol6"]), "core": z["core"], "U": [z["U0"], z["U1"], z["U2"]], "mass": z["mass"],
            "tol_ref": float(z["tol_ref"])}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--dtype", default="mixed", choices=["mixed", "f64", "f32"])
    ap.add_argument("--concurrent", type=int, default=32, help="solves per step, run at once")
    ap.add_argument("--rank-cap", type=int, default=96)
    ap.add_argument("--inner-tol", type=float, default=2e-2, help="mixed form: inner FP32 solve tolerance")
    ap.add_argument("--refine-keep", type=float, default=3e-2, help="mixed form: accuracy kept of each correction")
    ap.add_argument("--max-outer", type=int, default=12, help="mixed form: cap on FP64 refinements")
    ap.add_argument("--gemm-ctas-per-sm", type=int, default=2, help="grouped-GEMM CTA budget per SM (0: uncapped)")
    ap.add_argument("--eig", type=int, default=1, choices=[0, 1],
                    help="FP32 Gram eigensolver: 1 pivoted Cholesky + one-sided Jacobi, 0 two-sided Jacobi")
    ap.add_argument("--dst", type=int, default=1, choices=[0, 1], help="FD sine transforms: 1 FFT, 0 dense")
    ap.add_argument("--gram-min-k", type=int, default=0, help="least reduction length per partial Gram (0: most partials)")
    ap.add_argument("--gemm-kind", type=int, default=2, choices=[0, 1, 2],
                    help="FP32 SIMT GEMM: 1 8x4 per thread, 2 the same with cp.async stages, 0 4x4")
    ap.add_argument("--tc", type=int, default=-1, choices=[-1, 0, 1],
                    help="FP32 contractions: 1 tensor cores (tcgen05), 0 SIMT, -1 the library default")
    ap.add_argument("--torch-streams", action="store_true", help="give each solve a torch stream (<= 32)")
    ap.add_argument("--serve", type=float, default=0.0,
                    help="instead of the batch benchmark: serve a Poisson-arrival stream at this rate (requests/s)")
    ap.add_argument("--requests", type=int, default=48, help="requests in the --serve stream")
    ap.add_argument("--serve-nmax", type=int, default=128,
                    help="largest Poisson n of the --serve stream (sizes 32, 64, 96, 128, 192, 256, 384 up to it)")
    ap.add_argument("--serve-setup", action="store_true",
                    help="--serve: build each uncached operator after its request arrives, inside its latency")
    ap.add_argument("--mix-caps", default="20,60", help="--mix: range of the rank caps (lo,hi)")
    ap.add_argument("--mix", type=int, default=0,
                    help="instead of the batch benchmark: this many independent solves of uneven n, p, rank cap and "
                         "geometry (n in {32..256}, p in {2,3,4}, caps 20-60), all submitted at once")
    ap.add_argument("--large", type=int, default=0, help="n of the large configuration (e.g. 512); 0: off")
    ap.add_argument("--kernels", type=int, default=0, help="time apply / FD / one truncation at this n; 0: off")
    ap.add_argument("--kernels-dtype", default="both", choices=["f32", "f64", "both"])
    ap.add_argument("--large-cap", type=int, default=80, help="large configuration: rank cap")
    ap.add_argument("--large-concurrent", type=int, default=2, help="large configuration: solves at once")
    ap.add_argument("--large-fp64", action="store_true", help="large configuration: also the FP64 form")
    ap.add_argument("--profile-batch", action="store_true",
                    help="per-class CUDA-event times of one extra, untimed step of concurrent solves")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-form measurement beside the mixed one")
    ap.add_argument("--fp64-concurrent", type=int, default=32, help="FP64 form: solves at once (0: single only)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------- CPU oracle
def _oracle_setup(n=N_DOF, p=DEGREE, amp=AMP):
    from oracle import expsum, fd, lowrank
    terms = lowrank.operator_terms("twist", amp, n, p)
    f = lowrank.rhs_tucker("twist", amp, n, p)
    # the preconditioner with the best exponential sums for this M_P, as the library's setup builds it
    _, om, al, _, _ = expsum.rp_best(fd.mp_value(n, p), 0.1)
    return terms, f, fd.ApproxFD(n, p, expsum=(om, al))


class _Stamps(list):
    """A record list for the oracle's Alg. 5 that stamps the wall clock as each iteration ends."""

    def append(self, item):
        item["t"] = time.perf_counter()
        super().append(item)


def oracle_iterations(max_it: int, setup=None):
    """Run the oracle's Alg. 5 on the workload for at most max_it iterations; returns (start time, per-iteration
    end stamps, info)."""
    from oracle import tpcg as otp
    terms, f, P = setup or _oracle_setup()
    rec = _Stamps()
    t0 = time.perf_counter()
    _, info = otp.tpcg(terms, f, P.apply, otp.Params(tol=TOL, max_it=max_it), record=rec)
    return t0, [r["t"] for r in rec], info


def oracle_sample():
    """Time one whole solve of the oracle's Alg. 5 on the same workload (its stored iteration count to
    convergence, setup excluded): solves/sec from the time per iteration over all of them."""
    iters = oracle_reference()["iters"]
    t0, stamps, info = oracle_iterations(iters)
    dt = stamps[-1] - t0
    per_iter = dt / max(len(stamps), 1)
    return {"value": 1.0 / (per_iter * iters), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(stamps)} TPCG iterations of the {N_DOF}^3 p={DEGREE} twisted-annulus solve (the "
                      f"oracle's whole {iters}-iteration solve) in {dt:.1f}s, setup excluded"}


def run_reference(args):
    """The oracle on the host cores: Alg. 5 runs on the workload timed in steps of CHUNK consecutive
    iterations, CHUNK chosen so that the K steps cover at least one whole solve (the iterates' ranks grow along
    a solve, so early iterations alone would flatter the CPU); a run that converges is restarted until K steps
    are timed; W untimed warm-up iterations first.  value = 1 / (mean time per iteration x the oracle's
    iteration count to convergence); ms_per_step is the mean measured time of a step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    K = max(args.steps, 1)
    iters = oracle_reference()["iters"]
    CHUNK = max(2, -(-iters // K))
    setup = _oracle_setup()
    if args.warmup > 0:
        oracle_iterations(args.warmup, setup)
    steps, runs, converged = [], 0, False
    while len(steps) < K:
        t0, stamps, info = oracle_iterations((K - len(steps)) * CHUNK, setup)
        runs += 1
        converged = converged or bool(info["res"] <= TOL)
        marks = [t0] + stamps
        for k in range(0, len(stamps) - CHUNK + 1, CHUNK):
            steps.append(marks[k + CHUNK] - marks[k])
        if len(stamps) < CHUNK:
            break
    steps = steps[:K]
    per_iter = sum(steps) / (CHUNK * len(steps))
    v = 1.0 / (per_iter * iters)
    sample = (f"{len(steps)} steps of {CHUNK} consecutive oracle Alg. 5 iterations in {runs} run(s) "
              f"({sum(steps):.1f}s, setup excluded; a run reached tol: {converged}), "
              f"scaled to the oracle's {iters}-iteration solve")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": len(steps), "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tol": TOL},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------- replicas
def max_over_ranks(x: float, device: str) -> float:
    """The slowest rank's time: replicas finish when the last one does."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, solves_per_step: int, steps: int, total_ms: float) -> float:
    """Whole-job solves/s: every rank solved `solves_per_step` problems per step (weak scaling)."""
    return world * solves_per_step * steps / (total_ms * 1e-3)


def rank_seeds(rank: int, solves_per_step: int):
    """Seeds of the problems one rank solves: replicas take disjoint seed ranges."""
    return [SEED + rank * solves_per_step + i for i in range(solves_per_step)]


# ------------------------------------------------------------------------------------------- GPU arm
def _profile(L, lib):
    import ctypes as C
    prof = {}
    for name, kind in list(lib.PROF_KINDS.items()) + [("sweeps", lib.PROF_SWEEPS)]:
        ms, cnt, fl, by = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        L.tpcg_profile_get(kind, C.byref(ms), C.byref(cnt), C.byref(fl), C.byref(by))
        prof[name] = {"ms": ms.value, "launches": cnt.value, "flops": fl.value, "bytes": by.value}
    return prof


def _roofline(prof, dt_name, lib, step_ms_total):
    """Roofline of the dominant kernel class: algorithmic work per launch / measured launch time."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    src = "of measured" if peaks else "of fallback"
    # FP32/FP64 SIMT peaks derived from the measured sustained bf16 rate and the nominal ratios
    # (bf16 2250, FP32 75, FP64 1.25 TFLOP/s dense nominal)
    alu = {"f64": bf16 * 1.25 / 2250.0, "f32": bf16 * 75.0 / 2250.0}
    classes = ["zgemm", "zblk", "gram", "eig", "proj", "qr", "apply", "fd"]
    # DRAM bytes per launch of the FP32 eigensolver from one ncu capture of this workload (dram__bytes_read.sum +
    # dram__bytes_write.sum, mean of 2 launches of hestenes_eig_kernel); other kernels: no capture, traffic null
    ncu_traffic = {"eig": 118656.0} if dt_name == "mixed" else {}
    dom = max(classes, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    roof = {"kernel": dom, "share_of_step": d["ms"] / max(step_ms_total, 1e-9), "launches": d["launches"],
            "ms_per_launch": per_launch_ms}
    if dom in ("apply", "fd"):
        ach = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
        roof.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": None, "peak_source": f"hbm_gbs {src}"})
    else:
        # the eigensolver's algorithmic work is the dense symmetric eigen-decomposition count 9 n'^3 per Gram
        # (the mixed form's eigensolver launches are FP32 apart from the FP64 truncations of x)
        prec = "f32" if (dom == "eig" and dt_name == "mixed") or dt_name == "f32" else "f64"
        pk = alu[prec]
        ach = d["flops"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
        roof.update({"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                     "traffic": ncu_traffic.get(dom),
                     "peak_source": f"{prec.upper()} SIMT peak = bf16_tflops_sustained {src} x nominal "
                                    f"{'75' if prec == 'f32' else '1.25'}/2250"})
    return roof


# ------------------------------------------------------------------------------------------- solution error
def _band_matrix_product(bands, j, t, Q, p):
    """K_t^j Q for the banded matrix stored as bands[j, t, d, i] = K_t^j[i, i + d - p]."""
    n = Q.shape[0]
    out = np.zeros_like(Q)
    for d in range(2 * p + 1):
        o = d - p
        lo, hi = max(0, -o), min(n, n - o)
        out[lo:hi] += bands[j, t, d, lo:hi, None] * Q[lo + o:hi + o]
    return out


def _quad(Z, mats):
    """<Z, Z x_1 M_1 x_2 M_2 x_3 M_3> for a dense core Z and symmetric matrices M_t."""
    Y = np.einsum("ia,ajk->ijk", mats[0], Z, optimize=True)
    Y = np.einsum("jb,ibk->ijk", mats[1], Y, optimize=True)
    Y = np.einsum("kc,ijc->ijk", mats[2], Y, optimize=True)
    return float(np.sum(Z * Y))


def _norms(core, U, w, bands, p, mass):
    """Coefficient 2-norm, parametric L2 norm and energy norm of a Tucker vector given by core and factors
    with orthonormal-izable columns: a QR of every factor moves it into the core first, so a difference of two
    close solutions is formed entry by entry in the small core (no cancellation in the quadratic forms)."""
    Q, Z = [], core
    for t in range(3):
        q, r = np.linalg.qr(U[t])
        Q.append(q)
        Z = np.moveaxis(np.tensordot(r, Z, axes=(1, t)), 0, t)
    l2c = float(np.linalg.norm(Z))
    l2 = _quad(Z, [q.T @ mass @ q for q in Q]) if mass is not None else 0.0
    en = 0.0
    for j in range(len(w)):
        en += w[j] * _quad(Z, [Q[t].T @ _band_matrix_product(bands, j, t, Q[t], p) for t in range(3)])
    return l2c, np.sqrt(max(l2, 0.0)), np.sqrt(max(en, 0.0))


def solution_error(X, ex, info, ref):
    """Relative errors of a solution X = (core, factors) against the oracle's stored solution of the same
    workload: coefficient 2-norm, L2 norm of the discrete function on the parametric cube (B-spline mass
    matrix), and energy norm x^T A x with the library's operator."""
    n, p, R = info.n, info.p, info.R
    bands = np.asarray(ex["bands"]).reshape(R, 3, 2 * p + 1, n)
    w = np.asarray(ex["w"])
    core_x, Ux = X
    core_r, Ur = ref["core"], ref["U"]
    r1, r2 = core_x.shape, core_r.shape
    G = np.zeros(tuple(a + b for a, b in zip(r1, r2)))
    G[:r1[0], :r1[1], :r1[2]] = core_x
    G[r1[0]:, r1[1]:, r1[2]:] = -core_r
    mass = ref.get("mass")
    e = _norms(G, [np.hstack([Ux[t], Ur[t]]) for t in range(3)], w, bands, p, mass)
    r = _norms(core_r, Ur, w, bands, p, mass)
    out = {"rel_l2_coeff": e[0] / r[0], "rel_energy": e[2] / r[2],
           "reference": ref.get("label", f"oracle FP64 Alg. 5 at tol {ref.get('tol_ref', 0):g} (stored), seed {SEED}")}
    if mass is not None:
        out["rel_l2_param"] = e[1] / r[1]
    return out


# ------------------------------------------------------------------------------------------- FP64 arm
FP64_STOP = 0.9


def fp64_arm(api, lib, pbs, rc, args, flush):
    """The plain FP64 form on the same problems: a single solve alone (the comparison arm), then
    args.fp64_concurrent solves at once; FP64 problems are re-created from the setup's exported tables."""
    import torch
    main = torch.cuda.current_stream()
    B = min(max(args.fp64_concurrent, 1), len(pbs))
    exs = []
    for pb in pbs[:B]:
        ex = pb.export()
        ex["v2u2"] = ex["v2u2"][: pb.info.n * pb.info.n2]
        exs.append((ex, pb.info))
    pb64 = [api.problem_from_export(ex, info, dtype=lib.F64, pinned=False) for ex, info in exs]
    ctx64 = [_ctx_for(api, p.info, lib.F64, rc) for p in pb64]
    x64 = [api.Tucker(N_DOF, cap=rc, core_cap=rc ** 3, dtype=lib.F64) for _ in range(B)]
    # FP64 Alg. 5 stops on the truncated residual, which the true one may exceed by the last truncations
    # (eta_k): the stop tolerance is set 10% below the target so that every solve reaches a true residual
    # <= TOL, the metric's definition
    kw = dict(tol=FP64_STOP * TOL, rank_cap=rc)
    api.tpcg_solve(pb64[0], ctx64[0], x64[0], **kw)     # warm-up (graphs captured)
    torch.cuda.synchronize()
    lat, sts = [], []
    for _ in range(2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        sts.append(api.tpcg_solve(pb64[0], ctx64[0], x64[0], **kw))
        b.record(main)
        torch.cuda.synchronize()
        lat.append(a.elapsed_time(b))
    out = {"stop_tol": kw["tol"], "single_solve_ms": float(np.median(lat)), "single_solves_per_s": 1000.0 / float(np.median(lat)),
           "single_true_rel_res": float(sts[-1].true_rel_res), "single_iters": int(sts[-1].iters),
           "single_status": int(sts[-1].status)}
    x_single = x64[0].to_numpy()
    if args.fp64_concurrent > 1:
        streams = [None] * B
        api.tpcg_solve_batch(pb64, ctx64, x64, streams, **kw)   # warm-up of every context
        torch.cuda.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        codes, bst = api.tpcg_solve_batch(pb64, ctx64, x64, streams, **kw)
        b.record(main)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out.update({"concurrent": B, "batch_ms": ms, "batch_solves_per_s": B * 1000.0 / ms,
                    "batch_status": [int(c) for c in codes],
                    "batch_true_rel_res_max": float(max(s.true_rel_res for s in bst))})
    return out, x_single, exs[0]


def _make_problem(api, lib, dt, seed):
    return api.tpcg_setup(lib.GEOM_TWIST, synth.amp_from_seed(seed), DEGREE, N_DOF, dt)


def _ctx_for(api, info, dt, rc):
    return api.Ctx(N_DOF, api.max_cols_for(info, rc, dt), rc, dt)


def run_gpu(args):
    import torch
    from paper_2306_00632_gb300 import api, lib

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    L = lib.load()
    dt = {"f64": lib.F64, "f32": lib.F32, "mixed": lib.MIXED}[args.dtype]
    B = max(args.concurrent, 1)
    rc = min(args.rank_cap, N_DOF)
    # B problems of the same family (seeds SEED .. SEED+B-1), one context, solution and stream each
    seeds = rank_seeds(rank, B)
    pbs = [_make_problem(api, lib, dt, sd) for sd in seeds]
    ctxs = [_ctx_for(api, p.info, dt, rc) for p in pbs]
    xs = [api.Tucker(N_DOF, cap=rc, core_cap=rc ** 3, dtype=dt) for _ in range(B)]
    # by default the library gives each solve a stream of its own (torch's pool holds 32 streams per priority)
    if args.torch_streams and B > 32:
        raise SystemExit("--torch-streams: torch's pool has 32 streams per priority; concurrent solves need their own")
    streams = [torch.cuda.Stream() for _ in range(B)] if args.torch_streams else [None] * B
    lib.check(L.tpcg_set_option(lib.OPT_GEMM_CTAS_PER_SM, args.gemm_ctas_per_sm), "tpcg_set_option")
    lib.check(L.tpcg_set_option(lib.OPT_EIG, args.eig), "tpcg_set_option")
    lib.check(L.tpcg_set_option(lib.OPT_DST, args.dst), "tpcg_set_option")
    lib.check(L.tpcg_set_option(lib.OPT_GRAM_MIN_K, args.gram_min_k), "tpcg_set_option")
    lib.check(L.tpcg_set_option(lib.OPT_GEMM_KIND, args.gemm_kind), "tpcg_set_option")
    if args.tc >= 0:
        lib.check(L.tpcg_set_option(lib.OPT_TC, args.tc), "tpcg_set_option")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    main = torch.cuda.current_stream()

    kw = dict(tol=TOL, rank_cap=rc, inner_tol=args.inner_tol, refine_keep=args.refine_keep)

    # (1) single-solve latency and the per-kernel profile (problem 0 on the main stream)
    for _ in range(max(args.warmup, 0)):
        api.tpcg_solve(pbs[0], ctxs[0], xs[0], **kw)
    torch.cuda.synchronize()
    L.tpcg_profile_reset()
    L.tpcg_profile_enable(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    single = []
    torch.cuda.profiler.start()   # an external profiler started with --profile-from-start off sees this region
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(main)
        st = api.tpcg_solve(pbs[0], ctxs[0], xs[0], **kw)
        ev[k][1].record(main)
        single.append(st)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    L.tpcg_profile_enable(0)
    lat_ms = [a.elapsed_time(b) for a, b in ev]
    prof = _profile(L, lib)

    # (2) throughput: K steps of B concurrent solves (tpcg_solve_batch), timed on the device
    def batch():
        return api.tpcg_solve_batch(pbs, ctxs, xs, streams, **kw)

    for _ in range(max(args.warmup, 0)):
        batch()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.tpcg_launch_count()
    import resource
    ru0 = resource.getrusage(resource.RUSAGE_SELF)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    torch.cuda.synchronize()
    g0.record(main)
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()   # the flush completes before the solve streams start
        codes, sts = batch()
        results.append((codes, sts))
    g1.record(main)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches = L.tpcg_launch_count() - launches0
    ru1 = resource.getrusage(resource.RUSAGE_SELF)
    host_cpu_s = (ru1.ru_utime - ru0.ru_utime) + (ru1.ru_stime - ru0.ru_stime)
    clk = clocks.stop()
    total_ms = g0.elapsed_time(g1)
    if ws > 1:
        total_ms = max_over_ranks(total_ms, "cuda")

    prof_batch = None
    if args.profile_batch:   # one more (untimed) step with per-class CUDA events on every solve's stream
        L.tpcg_profile_reset()
        L.tpcg_profile_enable(1)
        batch()
        torch.cuda.synchronize()
        L.tpcg_profile_enable(0)
        pb_ = _profile(L, lib)
        prof_batch = {k: {"ms_per_solve": round(v["ms"] / B, 3), "launches_per_solve": round(v["launches"] / B, 1)}
                      for k, v in pb_.items() if k != "sweeps"}
    roof = _roofline(prof, args.dtype, lib, sum(lat_ms))
    value = job_throughput(ws, B, args.steps, total_ms)
    last = results[-1][1]
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
           "config": {"workload": WORKLOAD, "solves_per_step": B, "inner_tol": args.inner_tol,
                      "gemm_ctas_per_sm": args.gemm_ctas_per_sm, "eig": args.eig, "dst": args.dst, "tc": args.tc,
                      "gram_min_k": args.gram_min_k, "gemm_kind": args.gemm_kind,
                      "refine_keep": args.refine_keep,
                      "seeds": f"{seeds[0]}..{seeds[-1]} on rank 0, disjoint ranges per rank (amp from seed)",
                      "tol": TOL, "rank_cap": rc,
                      "R": [p.info.R for p in pbs], "RP": pbs[0].info.RP, "parallelism": f"replicas x{ws}",
                      "l2": "256 MB buffer written between timed steps"},
           "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                          "what": "single solve alone on the device (CUDA events)"},
           "solve": {"status": [int(c) for c in results[-1][0]],
                     "true_rel_res": [float(s.true_rel_res) for s in last],
                     "inner_iters": [int(s.iters) for s in last], "outer_iters": [int(s.outer_iters) for s in last],
                     "rank": [list(s.rank) for s in last]},
           "single": {"iters": [int(s.iters) for s in single], "true_rel_res": [float(s.true_rel_res) for s in single]},
           "gpu_launches": int(launches), "roofline": roof,
           "host_cpu_s_per_step": host_cpu_s / args.steps, "host_cores": os.cpu_count(),
           "kernel_ms_single": {k: round(v["ms"], 3) for k, v in prof.items() if k != "sweeps"},
           "kernel_tflops_single": {k: round(v["flops"] / (v["ms"] * 1e9), 3) for k, v in prof.items()
                                    if k in ("zgemm", "zblk", "gram", "proj", "eig", "apply", "fd") and v["ms"] > 0},
           "eig_sweeps_per_gram": prof["sweeps"]["flops"] / max(prof["sweeps"]["bytes"], 1.0),
           **({"kernel_classes_in_batch": prof_batch} if prof_batch else {}),
           "clocks": clk}

    # the solution of seed SEED (problem 0) from the last timed step, against the oracle's stored solution
    x_main = xs[0].to_numpy()
    if rank == 0 and not args.no_fp64 and args.dtype != "f64":
        fp64, x64, (ex0, info0) = fp64_arm(api, lib, pbs, rc, args, flush)
        out["fp64"] = fp64
    else:
        ex0 = pbs[0].export()
        info0, x64 = pbs[0].info, None
    if rank == 0:
        try:
            ref = oracle_reference()
            err = {args.dtype: solution_error(x_main, ex0, info0, ref)}
            if x64 is not None:
                err["f64"] = solution_error(x64, ex0, info0, ref)
            out["error_vs_oracle"] = err
        except Exception as e:   # the error report must not hide the GPU line
            out["error_vs_oracle"] = {"error": str(e)[:200]}
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e(api, lib, pbs, dt, ctxs, xs, streams, kw, args)
    if rank == 0 and not args.no_cpu and ws == 1:
        try:
            out["cpu_baseline"] = oracle_sample()
        except Exception as e:   # the baseline must not hide the GPU line
            out["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def e2e(api, lib, pbs, dt, ctxs, xs, streams, kw, args):
    """Same metric through the public API with host inputs: every step re-creates the B problems from pinned
    host arrays (host -> device copies inside tpcg_problem_create), solves them at once and reads the
    solutions back to the host."""
    import torch
    exs = []
    for pb in pbs:
        ex = pb.export()
        ex["v2u2"] = ex["v2u2"][: pb.info.n * pb.info.n2]
        exs.append((ex, pb.info))
    h2d = 0
    for ex, _ in exs:
        h2d += 8 * sum(int(np.asarray(ex[k]).size) for k in ("w", "bands", "f_core", "f_U0", "f_U1", "f_U2", "lam",
                                                            "mu", "w_val", "v2u2", "omega", "alpha"))
        h2d += 4 * (int(ex["w_rowptr"].size) + int(ex["w_col"].size))
    K = max(2, min(args.steps, 3))
    times = []
    d2h = 0
    for k in range(K + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pb2 = [api.problem_from_export(ex, info, dtype=dt, pinned=True) for ex, info in exs]
        api.tpcg_solve_batch(pb2, ctxs, xs, streams, **kw)
        d2h = 0
        for x in xs:
            core, fac = x.to_numpy()
            d2h += (core.size + sum(f.size for f in fac)) * (4 if dt == lib.F32 else 8)
        torch.cuda.synchronize()
        if k > 0:
            times.append(time.perf_counter() - t0)
        del pb2
    return {"value": len(pbs) / statistics.median(times), "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": K}


def run_serve(args):
    """Continuous-batching server under a Poisson-arrival stream: half scalar Poisson requests (mixed form,
    n in {32, 64, 96, 128}, p in {2, 3}), half elasticity requests (FP64, n in {16, 24, 32}, lambda = 1,
    mu in [0.3, 1], body force (0, 0.1, -1)), seeded.  Prints p50/p99 latency and throughput."""
    import torch
    from paper_2306_00632_gb300 import lib, serve
    lib.load()
    arr = synth.poisson_arrivals(args.serve, args.requests, seed=SEED)
    sizes = tuple(v for v in (32, 64, 96, 128, 192, 256, 384) if v <= max(args.serve_nmax, 32))
    reqs = []
    for i, t in enumerate(arr):
        sd = SEED + 1000 + i
        if i % 2 == 0:
            n = sizes[int(synth.unit_from_seed(sd, 2) * len(sizes))]
            p = 2 + int(synth.unit_from_seed(sd, 3) * 2)
            reqs.append(serve.Request(lib.GEOM_TWIST, synth.amp_from_seed(sd), p, n, min(n, 96), tol=TOL,
                                      dtype=lib.MIXED, arrival=float(t)))
        else:
            n = (16, 24, 32)[int(synth.unit_from_seed(sd, 2) * 3)]
            mu = 0.3 + 0.7 * synth.unit_from_seed(sd, 5)
            reqs.append(serve.Request(lib.GEOM_TWIST, synth.amp_from_seed(sd), 2, n, n, tol=TOL, dtype=lib.F64,
                                      arrival=float(t), problem="elasticity", lame_lambda=1.0, lame_mu=mu,
                                      force=(0.0, 0.1, -1.0)))
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(int(free * 0.6), max_slots=32, setup_in_latency=args.serve_setup)
    if args.serve_setup:   # warm-up on descriptions outside the stream: its operators stay uncached
        srv.run([serve.Request(lib.GEOM_CUBE, 0.0, 2, 24, 24, tol=TOL, dtype=lib.MIXED),
                 serve.Request(lib.GEOM_CUBE, 0.0, 2, 16, 16, tol=TOL, dtype=lib.F64, problem="elasticity",
                               lame_lambda=1.0, lame_mu=0.5, force=(0.0, 0.1, -1.0))])
    else:
        srv.run(reqs[:4])   # warm-up: operators cached, contexts and graphs exercised
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    lat = serve.percentiles(res)
    ok = sum(1 for r in res if r.status == 0 and r.true_rel_res <= TOL)
    line = {"metric": "served TPCG requests: p50/p99 latency and solves/s", "unit": "s",
            "rate_hz": args.serve, "requests": len(res), "converged": ok,
            "latency_s": {"p50": lat["p50"], "p99": lat["p99"]},
            "solves_per_s": len(res) / max(max(r.finished for r in res), 1e-9), "wall_s": wall,
            "mix": f"50/50 Poisson (mixed form, n {sizes[0]}-{sizes[-1]}, rank cap min(n, 96)) / elasticity "
                   "(FP64, n 16-32), seeded twisted annuli",
            "setup_in_latency": bool(args.serve_setup),
            "max_slots": 32}
    if args.serve_setup:
        st = sorted(r.setup_s for r in res)
        line["operator_cache_hit_rate"] = sum(1 for r in res if r.cache_hit) / len(res)
        line["setup_s"] = {"p50": st[len(st) // 2], "max": st[-1]}
    by = {}
    for r in res:
        k = r.request.problem
        d = by.setdefault(k, {"requests": 0, "status": {}, "iters": [], "latency_s": [], "n": []})
        d["requests"] += 1
        d["status"][str(r.status)] = d["status"].get(str(r.status), 0) + 1
        d["iters"].append(r.iters)
        d["latency_s"].append(round(r.latency, 2))
        d["n"].append(r.request.n)
    line["by_problem"] = by
    print(json.dumps(line), flush=True)


def run_mix(args):
    """Many independent solves of uneven size at once: the mixed form (FP32 inner solves, FP64 refinement)
    on seeded twisted annuli with n in {32, 64, 96, 128, 192, 256}, p in {2, 3, 4}, amplitude in [0, 0.3] and
    rank caps in --mix-caps (default 20-60), all submitted at t = 0 to the continuous-batching server (at most 32
    in flight, admitted by device memory).  Operators are built before the clock starts.  `value` counts the
    solves that reached true relative residual 1e-6 (a cap below the solution's rank cannot); the per-n status
    follows."""
    import torch
    from paper_2306_00632_gb300 import lib, serve
    lib.load()
    caps = tuple(int(v) for v in args.mix_caps.split(","))
    mix = synth.batch_mix(args.mix, seed0=SEED, caps=caps)
    reqs = [serve.Request(lib.GEOM_TWIST, pr.amp, pr.degree, pr.n, min(cap, pr.n), tol=TOL, dtype=lib.MIXED,
                          arrival=0.0) for pr, cap in mix]
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(int(free * 0.7), max_slots=32)
    t0 = time.perf_counter()
    srv.prepare(reqs, workers=min(16, os.cpu_count() or 8))
    setup_s = time.perf_counter() - t0
    srv.run(reqs[:8])   # warm-up: kernels loaded, per-device attributes set
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    ok = [r for r in res if r.status == 0 and r.true_rel_res <= TOL]
    by_n = {}
    for r in res:
        d = by_n.setdefault(str(r.request.n), {"solves": 0, "converged": 0, "iters": []})
        d["solves"] += 1
        d["converged"] += int(r.status == 0 and r.true_rel_res <= TOL)
        d["iters"].append(r.iters)
    line = {"metric": "independent mixed-precision TPCG solves/sec to rel-residual 1e-6 (uneven n, p, rank cap)",
            "value": len(ok) / wall, "unit": "solves/s", "all_solves_per_s": len(res) / wall, "solves": len(res),
            "converged": len(ok), "wall_s": wall,
            "setup_s_untimed": setup_s, "max_in_flight": 32, "dtype": "mixed", "data": "synthetic",
            "config": {"workload": "twisted quarter annuli, n in {32,64,96,128,192,256}, p in {2,3,4}, amp in "
                                   f"[0,0.3], rank caps {caps[0]}-{caps[1]} (at most n)",
                       "seeds": f"{SEED}..{SEED + args.mix - 1}", "tol": TOL},
            "latency_s": serve.percentiles(res), "max_true_rel_res": max(r.true_rel_res for r in res),
            "by_n": by_n}
    print(json.dumps(line), flush=True)


def run_large(args):
    """The large configuration: one twisted-annulus Poisson problem family at n = args.large dofs per direction
    (p = 3, rank cap args.large_cap, mixed form: FP32 inner solves with their Grams above 128 reduced by the
    Rayleigh-Ritz step, FP64 refinement), args.large_concurrent solves at once.  Reports solves/s, a single
    solve's per-kernel-class times with the roofline fractions of the operator apply (HBM) and of the rounding's
    contractions (FP32 SIMT, or TF32 tensor cores with --tc 1), and with --large-fp64 the FP64 form's single
    solve on the same problem and the difference between the two solutions."""
    import torch
    from paper_2306_00632_gb300 import api, lib
    L = lib.load()
    n, rc, B = args.large, min(args.large_cap, args.large), max(args.large_concurrent, 1)
    if args.tc >= 0:
        lib.check(L.tpcg_set_option(lib.OPT_TC, args.tc), "tpcg_set_option")
    seeds = [SEED + i for i in range(B)]
    pbs = [api.tpcg_setup(lib.GEOM_TWIST, synth.amp_from_seed(sd), DEGREE, n, lib.MIXED) for sd in seeds]
    ctxs = [api.Ctx(n, api.max_cols_for(p.info, rc, lib.MIXED), rc, lib.MIXED) for p in pbs]
    xs = [api.Tucker(n, cap=rc, core_cap=rc ** 3, dtype=lib.MIXED) for _ in range(B)]
    kw = dict(tol=TOL, rank_cap=rc, inner_tol=args.inner_tol, refine_keep=args.refine_keep, max_outer=args.max_outer)
    main = torch.cuda.current_stream()
    api.tpcg_solve(pbs[0], ctxs[0], xs[0], **kw)   # warm-up: graphs captured
    torch.cuda.synchronize()
    L.tpcg_profile_reset()
    L.tpcg_profile_enable(1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(main)
    st0 = api.tpcg_solve(pbs[0], ctxs[0], xs[0], **kw)
    b.record(main)
    torch.cuda.synchronize()
    L.tpcg_profile_enable(0)
    single_ms = a.elapsed_time(b)
    prof = _profile(L, lib)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    src = "of measured" if peaks else "of fallback"
    tc_on = args.tc == 1
    # FP32 contractions: SIMT peak (nominal 75 of 2250 bf16), or TF32 tensor peak (nominal 1125 of 2250) / 3
    # for the three MMAs of the 3xTF32 split
    f32_peak = bf16 * (1125.0 / 2250.0 / 3.0 if tc_on else 75.0 / 2250.0)
    classes = {}
    for k in ("apply", "fd", "zgemm", "zblk", "gram", "eig", "proj", "qr", "dot", "round"):
        d = prof[k]
        row = {"ms": round(d["ms"], 3), "launches": d["launches"]}
        if d["ms"] > 0 and k in ("apply", "fd"):
            ach = d["bytes"] / (d["ms"] * 1e-3) / 1e9
            row.update({"bound": "hbm", "achieved_gbs": ach, "frac": ach / hbm})
        elif d["ms"] > 0 and k in ("zgemm", "zblk", "gram", "proj", "eig"):
            ach = d["flops"] / (d["ms"] * 1e-3) / 1e12
            row.update({"bound": "tensor" if tc_on else "alu", "achieved_tflops": ach, "frac": ach / f32_peak})
        classes[k] = row
    # throughput: steps of B concurrent solves
    def batch():
        return api.tpcg_solve_batch(pbs, ctxs, xs, [None] * B, **kw)
    batch()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(main)
    res = []
    for _ in range(args.steps):
        res.append(batch())
    g1.record(main)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = g0.elapsed_time(g1)
    codes, sts = res[-1]
    out = {"metric": f"TPCG solves/sec to rel-residual 1e-6 at n={n}", "value": B * args.steps * 1000.0 / total_ms,
           "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "dtype": "mixed", "data": "synthetic",
           "config": {"workload": f"twisted quarter annulus Poisson, p={DEGREE}, n={n}/direction", "rank_cap": rc,
                      "solves_per_step": B, "seeds": f"{seeds[0]}..{seeds[-1]}", "tol": TOL, "tc": args.tc,
                      "R": [p.info.R for p in pbs], "RP": pbs[0].info.RP, "inner_tol": args.inner_tol,
                      "refine_keep": args.refine_keep, "max_outer": args.max_outer},
           "status": [int(c) for c in codes], "true_rel_res": [float(s.true_rel_res) for s in sts],
           "inner_iters": [int(s.iters) for s in sts], "outer_iters": [int(s.outer_iters) for s in sts],
           "rank": [list(s.rank) for s in sts],
           "single": {"ms": single_ms, "iters": int(st0.iters), "true_rel_res": float(st0.true_rel_res)},
           "kernel_classes_single": classes,
           "peaks": {"hbm_gbs": hbm, "f32_tflops": f32_peak, "source": src}, "clocks": clk}
    if args.large_fp64:
        ex = pbs[0].export()
        ex["v2u2"] = ex["v2u2"][: pbs[0].info.n * pbs[0].info.n2]
        pb64 = api.problem_from_export(ex, pbs[0].info, dtype=lib.F64, pinned=False)
        ctx64 = api.Ctx(n, api.max_cols_for(pb64.info, rc, lib.F64), rc, lib.F64)
        x64 = api.Tucker(n, cap=rc, core_cap=rc ** 3, dtype=lib.F64)
        a.record(main)
        s64 = api.tpcg_solve(pb64, ctx64, x64, tol=FP64_STOP * TOL, rank_cap=rc)
        b.record(main)
        torch.cuda.synchronize()
        X64 = x64.to_numpy()
        Xm = xs[0].to_numpy()   # problem 0's solution from the last timed step
        err = solution_error(Xm, ex, pbs[0].info, {"core": X64[0], "U": list(X64[1]),
                                                  "label": f"FP64 Alg. 5 on the GPU, stop tol {FP64_STOP * TOL:g}"})
        out["fp64"] = {"single_ms": a.elapsed_time(b), "iters": int(s64.iters), "status": int(s64.status),
                       "true_rel_res": float(s64.true_rel_res), "rank": list(s64.rank),
                       "mixed_vs_fp64": err}
    print(json.dumps(out), flush=True)


def run_kernels(args):
    """The operator pieces at n = args.kernels (p = 3, twisted annulus, seed 7) on a solver-like input of rank
    args.large_cap (random orthonormal factors, geometric core): the banded apply y = A x, the preconditioner
    v = P^-1 x and one truncation of A x (Alg. 1 at eps 1e-3), in FP32 and FP64, each timed alone with CUDA
    events on its stream (median of the repeats, L2 flushed before each).  Reports the algorithmic bytes or
    flops per launch (the library's device-side accounting from the actual ranks) over the measured time,
    against the measured HBM copy peak or the FP32/FP64 SIMT peaks."""
    import torch
    from paper_2306_00632_gb300 import api, lib
    L = lib.load()
    n, r = args.kernels, args.large_cap
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    alu = {lib.F32: bf16 * 75.0 / 2250.0, lib.F64: bf16 * 1.25 / 2250.0}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    main = torch.cuda.current_stream()
    g = np.random.default_rng(SEED)
    core = np.einsum("i,j,k->ijk", *[0.7 ** np.arange(r)] * 3) * g.standard_normal((r, r, r))
    U = [np.linalg.qr(g.standard_normal((n, r)))[0] for _ in range(3)]
    out = {"metric": f"operator pieces at n={n}: fraction of roofline", "n": n, "rank": r, "kernels": {},
           "peaks": {"hbm_gbs": hbm, "f32_tflops": alu[lib.F32], "f64_tflops": alu[lib.F64],
                     "source": "of measured" if peaks else "of fallback"}, "l2": "256 MB buffer written before each launch"}

    def timed(fn, reps):
        # the 256 MB flush keeps the stream busy while the host enqueues the start event and the launches, so the
        # events bracket the kernels and not the host's launch latency
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            fn()
            b.record(main)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    kinds = {"f32": [(lib.F32, "f32")], "f64": [(lib.F64, "f64")], "both": [(lib.F32, "f32"), (lib.F64, "f64")]}
    for dt, name in kinds[args.kernels_dtype]:
        pb = api.tpcg_setup(lib.GEOM_TWIST, AMP, DEGREE, n, dt)
        R, RP = pb.info.R, pb.info.RP
        x = api.Tucker.from_numpy(core, U, cap=r, core_cap=r ** 3, dtype=dt)
        y = api.Tucker(n, cap=R * r, core_cap=1, dtype=dt)
        v = api.Tucker(n, cap=RP * r, core_cap=1, dtype=dt)
        ctx = api.Ctx(n, max(R, RP) * r, r, dt)
        api.tucker_apply(pb, x, y)
        api.fd_precond_apply(pb, ctx, x, v)
        torch.cuda.synchronize()
        for kind, fn, reps in (("apply", lambda: api.tucker_apply(pb, x, y), 20),
                               ("fd", lambda: api.fd_precond_apply(pb, ctx, x, v), 20)):
            L.tpcg_profile_reset()
            L.tpcg_profile_enable(1)
            fn()
            torch.cuda.synchronize()
            L.tpcg_profile_enable(0)
            work = _profile(L, lib)[kind]
            ms = timed(fn, reps)
            ach = work["bytes"] / (ms * 1e-3) / 1e9
            out["kernels"][f"{kind}_{name}"] = {"ms": ms, "bytes": work["bytes"], "flops": work["flops"],
                                                "achieved_gbs": ach, "bound": "hbm", "frac": ach / hbm}
        # one truncation of A x (k = R r columns per mode), re-applied before every repeat
        yr = api.Tucker(n, cap=R * r, core_cap=r ** 3, dtype=dt)
        ctx2 = api.Ctx(n, R * r, r, dt)

        def trunc():
            api.tucker_round(ctx2, yr, 1e-3)

        ts, work = [], None
        for rep in range(4):
            api.tucker_apply(pb, x, yr)
            torch.cuda.synchronize()
            flush.zero_()
            L.tpcg_profile_reset()
            L.tpcg_profile_enable(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            trunc()
            b.record(main)
            torch.cuda.synchronize()
            L.tpcg_profile_enable(0)
            if rep > 0:
                ts.append(a.elapsed_time(b))
            work = _profile(L, lib)
        ms = float(np.median(ts))
        fl = sum(work[k]["flops"] for k in ("zgemm", "zblk", "gram", "proj"))
        cls = {k: round(work[k]["ms"], 3) for k in ("qr", "zblk", "zgemm", "gram", "eig", "proj")}
        ach = fl / (ms * 1e-3) / 1e12
        out["kernels"][f"round_{name}"] = {"ms": ms, "contraction_flops": fl, "achieved_tflops": ach,
                                           "bound": "alu", "frac": ach / alu[dt], "class_ms": cls,
                                           "k": R * r}
        del pb, x, y, v, ctx, yr, ctx2
        torch.cuda.synchronize()
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.kernels > 0:
        run_kernels(args)
    elif args.large > 0:
        run_large(args)
    elif args.mix > 0:
        run_mix(args)
    elif args.serve > 0:
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
