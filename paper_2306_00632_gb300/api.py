"""Python-facing wrappers with the names of the C ABI (include/tpcg.h).

Device memory and streams come from PyTorch; everything else is a call into the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import struct

import numpy as np
import torch

from . import lib as L
from .lib import check

_TORCH_DT = {L.F64: torch.float64, L.F32: torch.float32, L.MIXED: torch.float64}


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dptr(ptr_or_tensor):
    if ptr_or_tensor is None:
        return None
    if isinstance(ptr_or_tensor, torch.Tensor):
        return C.c_void_p(ptr_or_tensor.data_ptr())
    return C.c_void_p(int(ptr_or_tensor))


class Tucker:
    """Caller-owned device buffers of one Tucker tensor (factors n x cap, core, descriptor)."""

    def __init__(self, n: int, cap: int, core_cap: int, dtype: int = L.F64, device="cuda"):
        td = _TORCH_DT[dtype]
        self.n, self.cap, self.core_cap, self.dtype = n, cap, core_cap, dtype
        self.U = [torch.zeros((cap, n), dtype=td, device=device) for _ in range(3)]   # column-major n x cap
        self.core = torch.zeros(max(core_cap, 1), dtype=td, device=device)
        self.desc = torch.zeros(L.DESC_BYTES, dtype=torch.uint8, device=device)
        sdt = L.F64 if dtype == L.MIXED else dtype      # tensors of a mixed-precision problem are FP64
        self.t = L.TuckerT(sdt, n, cap, core_cap, (C.c_void_p * 3)(*[u.data_ptr() for u in self.U]),
                           self.core.data_ptr(), self.desc.data_ptr())

    @property
    def ref(self):
        return C.byref(self.t)

    # ------------------------------------------------------------------ host <-> device
    @classmethod
    def from_numpy(cls, core, factors, cap=None, core_cap=None, dtype=L.F64):
        n = factors[0].shape[0]
        r = core.shape
        cap = cap or max(r)
        core_cap = core_cap or int(np.prod(r))
        T = cls(n, cap, core_cap, dtype)
        T.upload(core, factors)
        return T

    def upload(self, core, factors):
        r = tuple(int(x) for x in core.shape)
        td = _TORCH_DT[self.dtype]
        for t in range(3):
            u = torch.as_tensor(np.ascontiguousarray(factors[t].T), dtype=td)
            self.U[t][: r[t]].copy_(u)
        flat = torch.as_tensor(np.asarray(core, dtype=np.float64).reshape(-1, order="F").copy(), dtype=td)
        self.core[: flat.numel()].copy_(flat)
        check(L.load().tucker_set_plain(self.ref, r[0], r[1], r[2], _stream()), "tucker_set_plain")

    def read_desc(self):
        """(nblk, ranks, blocks) with blocks = [(off, r, core_ptr, scale)]."""
        torch.cuda.current_stream().synchronize()
        raw = self.desc.cpu().numpy().tobytes()
        nblk, r1, r2, r3 = struct.unpack_from("4i", raw, 0)
        blocks = []
        for b in range(nblk):
            o = 32 + 40 * b
            off = struct.unpack_from("3i", raw, o)
            rr = struct.unpack_from("3i", raw, o + 12)
            ptr, = struct.unpack_from("Q", raw, o + 24)
            sc, = struct.unpack_from("d", raw, o + 32)
            blocks.append((off, rr, ptr, sc))
        return nblk, (r1, r2, r3), blocks

    def factors_numpy(self, ranks):
        return [self.U[t][: ranks[t]].double().cpu().numpy().T.copy() for t in range(3)]

    def to_numpy(self, others=(), fallback=None):
        """(core, factors) on the host; a block core is returned as a dense block-diagonal array, with
        block cores looked up among this tensor and ``others`` by device pointer (``fallback(shape)``
        supplies a host array for a block whose core is owned by the library, e.g. the rhs)."""
        nblk, ranks, blocks = self.read_desc()
        fac = self.factors_numpy(ranks)
        pool = {self.core.data_ptr(): self}
        for o in others:
            pool[o.core.data_ptr()] = o
        core = np.zeros(ranks)
        for off, rr, ptr, sc in blocks:
            src = None
            for base, T in pool.items():
                end = base + T.core.numel() * T.core.element_size()
                if base <= ptr < end:
                    src = (T, (ptr - base) // T.core.element_size())
            if src is None:
                if fallback is None:
                    raise KeyError("block core not among the known tensors")
                g = np.asarray(fallback(rr), dtype=np.float64)
            else:
                T, start = src
                cnt = rr[0] * rr[1] * rr[2]
                g = T.core[start:start + cnt].double().cpu().numpy().reshape(rr, order="F")
            core[off[0]:off[0] + rr[0], off[1]:off[1] + rr[1], off[2]:off[2] + rr[2]] += sc * g
        return core, fac


class Problem:
    def __init__(self, handle, dtype):
        self.h = C.c_void_p(handle)
        self.dtype = dtype
        self.info = L.ProblemInfo()
        check(L.load().tpcg_problem_get_info(self.h, C.byref(self.info)), "tpcg_problem_get_info")

    def __del__(self):
        try:
            if self.h:
                L.load().tpcg_problem_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def export(self):
        """Host copies of the setup data (double)."""
        i = self.info
        n, p, R, n1, n2, RP = i.n, i.p, i.R, i.n1, i.n2, i.RP
        out = {"w": np.zeros(R), "bands": np.zeros(R * 3 * (2 * p + 1) * n), "f_core": np.zeros(i.rf[0] * i.rf[1] * i.rf[2]),
               "f_U0": np.zeros(n * i.rf[0]), "f_U1": np.zeros(n * i.rf[1]), "f_U2": np.zeros(n * i.rf[2]),
               "lam": np.zeros(n), "mu": np.zeros(n1), "v2u2": np.zeros(max(n * n2, 1)), "omega": np.zeros(RP),
               "alpha": np.zeros(RP)}
        keys = ["w", "bands", "f_core", "f_U0", "f_U1", "f_U2", "lam", "mu", "v2u2", "omega", "alpha"]
        ptrs = [out[k].ctypes.data_as(C.c_void_p) for k in keys]
        check(L.load().tpcg_problem_export(self.h, *ptrs), "tpcg_problem_export")
        rowptr = np.zeros(n + 1, dtype=np.int32)
        col = np.zeros(max(i.w_nnz, 1), dtype=np.int32)
        val = np.zeros(max(i.w_nnz, 1))
        check(L.load().tpcg_problem_export_w(self.h, rowptr.ctypes.data_as(C.c_void_p), col.ctypes.data_as(C.c_void_p),
                                             val.ctypes.data_as(C.c_void_p)), "tpcg_problem_export_w")
        W = np.zeros((n, n1))
        for r in range(n):
            for e in range(rowptr[r], rowptr[r + 1]):
                W[r, col[e]] = val[e]
        out["W"] = W
        out["w_rowptr"], out["w_col"], out["w_val"] = rowptr, col, val
        return out


def tpcg_setup(kind: int, amp: float, degree: int, n: int, dtype: int = L.F64, eps_geo=0.0, eps_prec=0.0,
               bc=(0, 0)) -> Problem:
    """bc = (k0, k1): 1 marks a homogeneous Neumann condition on the faces eta_t = 0 (k0) / eta_t = 1 (k1) of
    every direction, 0 a homogeneous Dirichlet one."""
    g = L.Geometry(kind, amp, eps_geo, eps_prec, int(bc[0]), int(bc[1]))
    h = C.c_void_p()
    check(L.load().tpcg_setup(C.byref(g), degree, n, dtype, C.byref(h)), "tpcg_setup")
    return Problem(h.value, dtype)


def problem_from_export(ex, info, dtype=L.F64, pinned=True, rhs=None) -> Problem:
    """Re-create a problem from exported host arrays (bands and W in CSR as stored by the library).
    With ``pinned`` the arrays are first placed in page-locked host memory.  ``rhs`` = (core, [U1, U2, U3])
    replaces the exported right-hand side (any Tucker tensor of the problem's n, e.g. the load vector of
    another source term or a lifted right-hand side)."""
    keep = []

    def host(a, np_dt):
        a = np.ascontiguousarray(a, dtype=np_dt)
        if pinned:
            t = torch.from_numpy(a).pin_memory()
            keep.append(t)
            return t.data_ptr()
        keep.append(a)
        return a.ctypes.data

    n, p, R = info.n, info.p, info.R
    a = L.ProblemArrays()
    a.n, a.p, a.R, a.dtype = n, p, R, dtype
    dptr = lambda arr: C.cast(host(arr, np.float64), C.POINTER(C.c_double))
    iptr = lambda arr: C.cast(host(arr, np.int32), C.POINTER(C.c_int))
    a.w = dptr(ex["w"])
    a.bands = dptr(ex["bands"])
    if rhs is None:
        a.rf = (C.c_int * 3)(*info.rf)
        a.f_core = dptr(ex["f_core"])
        a.f_U = (C.POINTER(C.c_double) * 3)(*[dptr(ex[f"f_U{t}"]) for t in range(3)])
    else:
        core, U = rhs
        a.rf = (C.c_int * 3)(*[int(d) for d in np.shape(core)])
        a.f_core = dptr(np.asarray(core, dtype=np.float64).reshape(-1, order="F"))
        a.f_U = (C.POINTER(C.c_double) * 3)(*[dptr(np.asarray(U[t], dtype=np.float64).reshape(-1, order="F"))
                                              for t in range(3)])
    a.n1, a.n2, a.RP, a.w_nnz = info.n1, info.n2, info.RP, info.w_nnz
    a.lam = dptr(ex["lam"])
    a.mu = dptr(ex["mu"])
    a.w_rowptr = iptr(ex["w_rowptr"])
    a.w_col = iptr(ex["w_col"])
    a.w_val = dptr(ex["w_val"])
    a.v2u2 = dptr(ex["v2u2"]) if info.n2 > 0 else C.POINTER(C.c_double)()
    a.omega = dptr(ex["omega"])
    a.alpha = dptr(ex["alpha"])
    a.lambda_min = info.lambda_min
    a.k0, a.k1 = info.k0, info.k1
    h = C.c_void_p()
    check(L.load().tpcg_problem_create(C.byref(a), C.byref(h)), "tpcg_problem_create")
    return Problem(h.value, dtype)


def _problem_arrays(n, p, terms, f_core, f_U, fd, dtype, keep):
    """tpcg_problem_arrays from host arrays (the numpy buffers are appended to `keep`)."""
    R = len(terms)
    bw = 2 * p + 1
    bands = np.zeros((R, 3, bw, n))
    for j, (w, mats) in enumerate(terms):
        for t in range(3):
            K = mats[t]
            for d in range(bw):
                for i in range(n):
                    jj = i + d - p
                    if 0 <= jj < n:
                        bands[j, t, d, i] = K[i, jj]

    def dp(a, ct=C.c_double):
        a = np.ascontiguousarray(a, dtype=np.float64 if ct is C.c_double else np.int32)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(ct))

    W = np.asarray(fd["W"])
    n1 = W.shape[1]
    rowptr, cols, vals = [0], [], []
    for i in range(n):
        nz = np.nonzero(W[i])[0]
        cols += list(nz)
        vals += list(W[i, nz])
        rowptr.append(len(cols))
    a = L.ProblemArrays()
    a.n, a.p, a.R, a.dtype = n, p, R, dtype
    a.w = dp(np.array([t[0] for t in terms], dtype=np.float64))
    a.bands = dp(bands.reshape(-1))
    r = f_core.shape
    a.rf = (C.c_int * 3)(*r)
    a.f_core = dp(np.asarray(f_core).reshape(-1, order="F"))
    a.f_U = (C.POINTER(C.c_double) * 3)(*[dp(np.asarray(f_U[t]).reshape(-1, order="F")) for t in range(3)])
    n2 = n - n1
    a.n1, a.n2, a.RP = n1, n2, len(fd["omega"])
    a.w_nnz = len(vals)
    a.lam = dp(fd["lam"])
    a.mu = dp(fd["mu"])
    a.w_rowptr = dp(np.array(rowptr), C.c_int)
    a.w_col = dp(np.array(cols if cols else [0]), C.c_int)
    a.w_val = dp(np.array(vals if vals else [0.0]))
    a.v2u2 = dp(np.asarray(fd["v2u2"]).reshape(-1, order="F")) if n2 > 0 else C.POINTER(C.c_double)()
    a.omega = dp(fd["omega"])
    a.alpha = dp(fd["alpha"])
    a.lambda_min = float(fd["lambda_min"])
    a.k0, a.k1 = (int(v) for v in fd.get("bc", (0, 0)))
    return a


def tpcg_problem_create(n, p, terms, f_core, f_U, fd, dtype=L.F64) -> Problem:
    """Problem from host arrays.  terms: list of (w, [K1, K2, K3]) dense banded n x n matrices;
    fd: dict with lam, mu, W (dense n x n1), v2u2 (n x n2), omega, alpha, lambda_min and optionally bc = (k0, k1),
    the Neumann flags of the ends (default (0, 0))."""
    keep = []
    a = _problem_arrays(n, p, terms, f_core, f_U, fd, dtype, keep)
    h = C.c_void_p()
    check(L.load().tpcg_problem_create(C.byref(a), C.byref(h)), "tpcg_problem_create")
    return Problem(h.value, dtype)


class Ctx:
    def __init__(self, n, max_cols, rank_cap, dtype=L.F64):
        h = C.c_void_p()
        check(L.load().tpcg_ctx_create(n, max_cols, rank_cap, dtype, C.byref(h)), "tpcg_ctx_create")
        self.h = h
        self.n, self.max_cols, self.rank_cap, self.dtype = n, max_cols, rank_cap, dtype

    def __del__(self):
        try:
            if self.h:
                L.load().tpcg_ctx_destroy(self.h)
                self.h = None
        except Exception:
            pass


def tucker_apply(pb: Problem, x: Tucker, y: Tucker, stream=None):
    check(L.load().tucker_apply(pb.h, x.ref, y.ref, _stream(stream)), "tucker_apply")


def tucker_residual(pb: Problem, x: Tucker, y: Tucker, stream=None):
    check(L.load().tucker_residual(pb.h, x.ref, y.ref, _stream(stream)), "tucker_residual")


def tucker_axpby(a, x: Tucker, b, y: Tucker, z: Tucker, stream=None):
    """z = a x + b y; a, b are floats or one-element float64 cuda tensors."""
    ad = a if isinstance(a, torch.Tensor) else None
    bd = b if isinstance(b, torch.Tensor) else None
    check(L.load().tucker_axpby(0.0 if ad is not None else float(a), _dptr(ad), x.ref,
                                0.0 if bd is not None else float(b), _dptr(bd), y.ref, z.ref, _stream(stream)),
          "tucker_axpby")


def tucker_dot(ctx: Ctx, x: Tucker, y: Tucker, out=None, stream=None):
    o = out if out is not None else torch.zeros(1, dtype=torch.float64, device="cuda")
    check(L.load().tucker_dot(ctx.h, x.ref, y.ref, _dptr(o), _stream(stream)), "tucker_dot")
    return o


def tucker_dot_static(x: Tucker, y: Tucker, out=None, stream=None):
    """<x, y> through the allocation-free entry point (ranks <= 64, no context)."""
    o = out if out is not None else torch.zeros(1, dtype=torch.float64, device="cuda")
    check(L.load().tucker_dot_static(x.ref, y.ref, _dptr(o), _stream(stream)), "tucker_dot_static")
    return o


def tucker_round(ctx: Ctx, y: Tucker, eps, rank_cap=0, info=None, stream=None):
    ed = eps if isinstance(eps, torch.Tensor) else None
    check(L.load().tucker_round(ctx.h, y.ref, 0.0 if ed is not None else float(eps), _dptr(ed), int(rank_cap),
                                _dptr(info), _stream(stream)), "tucker_round")


def fd_precond_apply(pb: Problem, ctx: Ctx, s: Tucker, v: Tucker, stream=None):
    check(L.load().fd_precond_apply(pb.h, ctx.h, s.ref, v.ref, _stream(stream)), "fd_precond_apply")


def max_cols_for(info, rank_cap: int, dtype: int) -> int:
    """Factor columns a context needs for solves of this problem at this rank cap: residuals hold the rhs
    columns plus R rank_cap (in the mixed form the inner rhs is itself a residual of rank <= rank_cap),
    preconditioner outputs R_P rank_cap, sums 2 rank_cap."""
    rhs = max(max(info.rf), rank_cap) if dtype == L.MIXED else max(info.rf)
    return max(info.R * rank_cap + rhs, info.RP * rank_cap, 2 * rank_cap)


def setup_host(kind: int, amp: float, degree: int, n: int, eps_geo=0.0, eps_prec=0.0, bc=(0, 0)):
    """tpcg_setup_host: the library's FP64 setup tables on the host (no GPU call), as numpy arrays in the
    layout of tpcg_problem_arrays: w, bands (R, 3, 2p+1, n), f_core (rf, Fortran order), f_U[t] (n x rf_t),
    lam, mu, v2u2 (n x n2), omega, alpha, W in CSR (w_rowptr, w_col, w_val), and the info struct."""
    g = L.Geometry(kind, amp, eps_geo, eps_prec, int(bc[0]), int(bc[1]))
    info = L.ProblemInfo()
    lib = L.load()
    nul = C.POINTER(C.c_double)()
    inul = C.POINTER(C.c_int)()
    check(lib.tpcg_setup_host(C.byref(g), degree, n, C.byref(info), *([nul] * 11), inul, inul, nul),
          "tpcg_setup_host")
    p, R, rf, n1, n2 = degree, info.R, tuple(info.rf), info.n1, info.n2
    out = {"w": np.zeros(R), "bands": np.zeros(R * 3 * (2 * p + 1) * n), "f_core": np.zeros(int(np.prod(rf))),
           "f_U0": np.zeros(n * rf[0]), "f_U1": np.zeros(n * rf[1]), "f_U2": np.zeros(n * rf[2]), "lam": np.zeros(n),
           "mu": np.zeros(n1), "v2u2": np.zeros(max(n * n2, 1)), "omega": np.zeros(info.RP),
           "alpha": np.zeros(info.RP), "w_rowptr": np.zeros(n + 1, np.int32),
           "w_col": np.zeros(max(info.w_nnz, 1), np.int32), "w_val": np.zeros(max(info.w_nnz, 1))}
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    check(lib.tpcg_setup_host(C.byref(g), degree, n, C.byref(info), dp(out["w"]), dp(out["bands"]),
                              dp(out["f_core"]), dp(out["f_U0"]), dp(out["f_U1"]), dp(out["f_U2"]), dp(out["lam"]),
                              dp(out["mu"]), dp(out["v2u2"]), dp(out["omega"]), dp(out["alpha"]), ip(out["w_rowptr"]),
                              ip(out["w_col"]), dp(out["w_val"])), "tpcg_setup_host")
    out["bands"] = out["bands"].reshape(R, 3, 2 * p + 1, n)
    out["f_core"] = out["f_core"].reshape(rf, order="F")
    out["f_U"] = [out.pop(f"f_U{t}").reshape((n, rf[t]), order="F") for t in range(3)]
    out["v2u2"] = out["v2u2"][:n * n2].reshape((n, n2), order="F")
    out["info"] = info
    return out


def expsum_best(M: float, eps_prec: float = 0.1, rmax: int = 60):
    """tpcg_expsum_best: the best exponential sum for 1/lambda on [1, M] with the fewest terms meeting
    E_R(M) <= eps_prec / M (Prop. 1, eq. estimate_prec_rel).  Host computation.  Returns (omega, alpha, E)."""
    om = (C.c_double * rmax)()
    al = (C.c_double * rmax)()
    R = C.c_int(0)
    E = C.c_double(0.0)
    check(L.load().tpcg_expsum_best(M, eps_prec, rmax, om, al, C.byref(R), C.byref(E)), "tpcg_expsum_best")
    return np.array(om[:R.value]), np.array(al[:R.value]), E.value


def set_option(key: int, value: int):
    """tpcg_set_option (process-wide)."""
    check(L.load().tpcg_set_option(key, value), "tpcg_set_option")


def tpcg_params(**kw):
    p = L.Params()
    L.load().tpcg_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def tpcg_solve(pb: Problem, ctx: Ctx, x: Tucker, stream=None, **kw):
    prm = tpcg_params(**kw)
    st = L.Stats()
    code = L.load().tpcg_solve(pb.h, ctx.h, C.byref(prm), x.ref, C.byref(st), _stream(stream))
    if code not in (0, 3):
        check(code, "tpcg_solve")
    return st


HIST_FIELDS = ("res", "omega", "beta", "xi", "eps", "v", "trials", "eta")


def ctx_history(ctx: "Ctx", max_rows: int = 4096):
    """tpcg_ctx_history: per-iteration scalars of the last Alg. 5 run on ctx, as a list of dicts (row 0 is the
    state after the set-up steps, row k >= 1 the state after iteration k)."""
    buf = np.zeros((max_rows, L.HIST_COLS))
    rows = C.c_int(0)
    check(L.load().tpcg_ctx_history(ctx.h, buf.ctypes.data_as(C.POINTER(C.c_double)), max_rows, C.byref(rows)),
          "tpcg_ctx_history")
    m = min(rows.value, max_rows)
    return [dict(zip(HIST_FIELDS, buf[k])) for k in range(m)]


def ctx_stream(ctx: "Ctx"):
    """The context's own CUDA stream as a torch stream (tpcg_ctx_stream): a stream no other solve shares."""
    h = C.c_void_p()
    check(L.load().tpcg_ctx_stream(ctx.h, C.byref(h)), "tpcg_ctx_stream")
    return torch.cuda.ExternalStream(h.value)


def tpcg_solve_batch(problems, ctxs, xs, streams, **kw):
    """Independent solves at once (tpcg_solve_batch): one host thread and one stream per solve.
    Returns (statuses, stats)."""
    k = len(problems)
    if not (len(ctxs) == len(xs) == len(streams) == k):
        raise ValueError("tpcg_solve_batch: problems, ctxs, xs and streams must have the same length")
    prm = (L.Params * k)(*[tpcg_params(**kw) for _ in range(k)])
    sts = (L.Stats * k)()
    pbs = (C.c_void_p * k)(*[p.h for p in problems])
    cts = (C.c_void_p * k)(*[c.h for c in ctxs])
    ts = (L.TuckerT * k)(*[x.t for x in xs])
    ss = (C.c_void_p * k)(*[(s.cuda_stream if s is not None else None) for s in streams])
    codes = (C.c_int * k)()
    code = L.load().tpcg_solve_batch(k, pbs, cts, prm, ts, sts, ss, codes)
    if code not in (0, 3):
        check(code, "tpcg_solve_batch")
    return [int(c) for c in codes], [sts[i] for i in range(k)]


# ------------------------------------------------------------------------------------------- elasticity
class Elast:
    """Elasticity block system (Sec. 5.3) owned by the library."""

    def __init__(self, handle, dtype):
        self.h = C.c_void_p(handle)
        self.dtype = dtype
        R = (C.c_int * 9)()
        RP = C.c_int()
        nf = C.c_double()
        check(L.load().tpcg_elast_get_info(self.h, R, C.byref(RP), C.byref(nf)), "tpcg_elast_get_info")
        self.R = [R[q] for q in range(9)]
        self.RP = RP.value
        self.norm_f = nf.value

    def __del__(self):
        try:
            if self.h:
                L.load().tpcg_elast_destroy(self.h)
                self.h = None
        except Exception:
            pass


def tpcg_elast_setup(kind, amp, degree, n, lame_lambda, lame_mu, force, dtype=L.F64, eps_geo=0.0, eps_prec=0.0,
                     bc=(0, 0)):
    """bc = (k0, k1): 1 makes the faces eta_t = 0 (k0) / eta_t = 1 (k1) of every direction traction-free,
    0 clamps them."""
    g = L.Geometry(kind, amp, eps_geo, eps_prec, int(bc[0]), int(bc[1]))
    f = (C.c_double * 3)(*[float(v) for v in force])
    h = C.c_void_p()
    check(L.load().tpcg_elast_setup(C.byref(g), degree, n, float(lame_lambda), float(lame_mu), f, dtype, C.byref(h)),
          "tpcg_elast_setup")
    return Elast(h.value, dtype)


def tpcg_elast_create(n, p, blocks, f, fd, lame_lambda, lame_mu, dtype=L.F64) -> Elast:
    """blocks[i][j]: Kronecker terms of A_ij; f[i]: Tucker rhs component (core, factors); fd: FD tables."""
    keep = []
    arr = (L.ProblemArrays * 9)()
    for i in range(3):
        for j in range(3):
            arr[3 * i + j] = _problem_arrays(n, p, blocks[i][j], f[i][0], f[i][1], fd, dtype, keep)
    h = C.c_void_p()
    check(L.load().tpcg_elast_create(arr, float(lame_lambda), float(lame_mu), C.byref(h)), "tpcg_elast_create")
    return Elast(h.value, dtype)


def _block(ts):
    return (L.TuckerT * 3)(*[t.t for t in ts])


def elast_apply(e: Elast, x, y, stream=None):
    check(L.load().tpcg_elast_apply(e.h, _block(x), _block(y), _stream(stream)), "tpcg_elast_apply")


def elast_residual(e: Elast, x, y, stream=None):
    check(L.load().tpcg_elast_residual(e.h, _block(x), _block(y), _stream(stream)), "tpcg_elast_residual")


def elast_precond(e: Elast, ctx: Ctx, s, v, stream=None):
    check(L.load().tpcg_elast_precond(e.h, ctx.h, _block(s), _block(v), _stream(stream)), "tpcg_elast_precond")


def elast_solve(e: Elast, ctx: Ctx, x, stream=None, **kw):
    prm = tpcg_params(**kw)
    st = L.Stats()
    code = L.load().tpcg_elast_solve(e.h, ctx.h, C.byref(prm), _block(x), C.byref(st), _stream(stream))
    if code not in (0, 3):
        check(code, "tpcg_elast_solve")
    return st
