"""ctypes binding of libecg (include/ecg.h).

Argument marshalling only: every step of the solve runs in the CUDA
library.  Host arrays are numpy float64/int arrays; device arrays are torch
CUDA tensors (PyTorch provides device memory and streams).  There is no CPU
fallback: if libecg.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK, ENOCONV, EINVAL, ENOMEM, ECUDA, EBREAKDOWN, ENOTSPD, ETIMEOUT = 0, 1, -1, -2, -3, -4, -5, -6
SRE, MSDO, MODMSDO = 0, 1, 2
PRE_CHOLQR, A_CHOLQR = 0, 1
FP64, MIXED = 0, 1
VARIANTS = {"sre": SRE, "msdo": MSDO, "modmsdo": MODMSDO}


class EcgError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class _Csr(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("nnz", C.c_int64),
        ("rowptr", C.c_void_p),
        ("col", C.c_void_p),
        ("val", C.c_void_p),
        ("on_device", C.c_int),
    ]


class _Opts(C.Structure):
    _fields_ = [
        ("variant", C.c_int),
        ("trunc", C.c_int),
        ("switch_tol", C.c_double),
        ("ortho", C.c_int),
        ("check_every", C.c_int),
        ("use_graph", C.c_int),
        ("precision", C.c_int),
        ("inner_tol", C.c_double),
        ("restart_every", C.c_int),
        ("restart_tol", C.c_double),
        ("restart_max", C.c_int),
        ("restart_at_switch", C.c_int),
        ("stop_rule", C.c_int),
        ("block_residual", C.c_int),
        ("tensor_cores", C.c_int),
        ("stream", C.c_void_p),
    ]


class _BatchOpts(C.Structure):
    _fields_ = [
        ("trunc", C.c_int),
        ("ortho", C.c_int),
        ("precision", C.c_int),
        ("inner_tol", C.c_double),
        ("slice_height", C.c_int),
        ("sort_window", C.c_int),
        ("ctas_per_sm", C.c_int),
        ("wait_limit_s", C.c_double),
        ("debug_barrier_extra", C.c_int),
        ("stream", C.c_void_p),
    ]


class _Result(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("switch_it", C.c_int),
        ("restarts", C.c_int),
        ("status", C.c_int),
        ("mem_vectors", C.c_int64),
        ("relres", C.c_double),
        ("relres_true", C.c_double),
        ("device_ms", C.c_double),
        ("history", C.POINTER(C.c_double)),
    ]


_lib = None
_P = C.c_void_p
_I = C.c_int
_D = C.c_double

# Every function declared in include/ecg.h, with its ctypes signature.
SIGNATURES = {
    "ecg_default_opts": (None, [C.POINTER(_Opts)]),
    "ecg_create": (_I, [C.POINTER(_Csr), _P, _I, C.POINTER(_Opts), C.POINTER(_P)]),
    "ecg_solve": (_I, [_P, _P, _P, _P, _D, _I, C.POINTER(_Result)]),
    "ecg_destroy": (None, [_P]),
    "ecg_strerror": (C.c_char_p, [_I]),
    "ecg_probe_fp64": (_I, [_I, C.POINTER(C.c_double)]),
    "ecg_profile_enable": (_I, [_P, _I]),
    "ecg_profile_read": (_I, [_P, _I, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "ecg_op_split": (_I, [_P, _P, _P, _I]),
    "ecg_op_spmm": (_I, [_P, _P, _P, _I]),
    "ecg_op_tdot": (_I, [_P, _I, _P, _P, _P, _I, _P]),
    "ecg_op_cgs2": (_I, [_P, _I, _P, _P, _P, _P, _I]),
    "ecg_op_block_sub": (_I, [_P, _I, _P, _P, _P, _P, _I]),
    "ecg_op_a_orthonormalize": (_I, [_P, _P, _P, _I]),
    "ecg_op_block_update": (_I, [_P, _P, _P, _I, _P, _P, C.POINTER(C.c_double)]),
    "ecg_op_msdo_generate": (_I, [_P, _P, _P, _P, _I, _P]),
    "ecg_tdot_noalloc": (_I, [C.c_int64, _I, _P, _P, _P, _I, _P, _P]),
    "ecg_set_preconditioner": (_I, [_P, _P, _I, _I]),
    "ecg_smooth": (_I, [_P, _P, _P, _I, _D]),
    "ecg_batch_default_opts": (None, [C.POINTER(_BatchOpts)]),
    "ecg_batch_create": (_I, [_I, _P, _P, _I, C.POINTER(_BatchOpts), C.POINTER(_P)]),
    "ecg_batch_solve": (_I, [_P, _P, _P, _P, _D, _I, _P]),
    "ecg_batch_layout": (_I, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_D), C.POINTER(_I)]),
    "ecg_batch_destroy": (None, [_P]),
    "ecg_op_prec_apply": (_I, [_P, _P, _P, _I]),
}

PREC_NONE, PREC_IC0 = 0, 1
STOP_R0, STOP_B = 0, 1


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libecg.so (building it in-tree when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libecg.so is not built ({path}); run paper_2305_19013_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().ecg_strerror(int(code)).decode()


def _ptr(a):
    """Pointer of a numpy array or a torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _check_tensor(a, shape, name):
    import torch

    if not (_is_torch_cuda(a) and a.dtype == torch.float64 and a.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")


@dataclass
class SolveResult:
    x: object
    iters: int
    switch_it: int
    status: int
    mem_vectors: int
    relres: float
    relres_true: float
    device_ms: float
    history: np.ndarray
    restarts: int = 0


class Solver:
    """A solver context: the matrix, its partition and the options
    (ecg_create); ``solve`` runs ecg_solve."""

    def __init__(
        self,
        rowptr,
        col,
        val,
        part,
        t: int,
        variant="sre",
        trunc: int = 0,
        switch_tol: float = 0.0,
        ortho: int = PRE_CHOLQR,
        check_every: int = 16,
        use_graph: bool = True,
        precision: int = FP64,
        inner_tol: float = 0.0,
        restart_every: int = 0,
        restart_tol: float = 0.0,
        restart_max: int = 0,
        restart_at_switch: bool = False,
        block_residual: bool = False,
        stop_rule: int = 0,
        tensor_cores: bool = True,
        stream=None,
    ):
        lib = load()
        self._lib = lib
        self._ctx = None
        on_dev = _is_torch_cuda(val)
        if on_dev:
            self._keep = (rowptr, col, val, part)
        else:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
            part = np.ascontiguousarray(part, dtype=np.int32)
            self._keep = (rowptr, col, val, part)
        n = int(rowptr.shape[0]) - 1
        self.n = n
        self.t = int(t)
        csr = _Csr(n, int(col.shape[0]), _ptr(rowptr), _ptr(col), _ptr(val), 1 if on_dev else 0)
        o = _Opts()
        lib.ecg_default_opts(C.byref(o))
        o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o.trunc = int(trunc)
        o.switch_tol = float(switch_tol)
        o.ortho = int(ortho)
        o.check_every = int(check_every)
        o.use_graph = 1 if use_graph else 0
        o.precision = int(precision)
        o.inner_tol = float(inner_tol)
        o.restart_every = int(restart_every)
        o.restart_tol = float(restart_tol)
        o.restart_max = int(restart_max)
        o.restart_at_switch = 1 if restart_at_switch else 0
        o.block_residual = 1 if block_residual else 0
        o.stop_rule = int(stop_rule)
        o.tensor_cores = int(tensor_cores)  # 0, 1 (True) or 2
        o.stream = stream
        ctx = C.c_void_p()
        rc = lib.ecg_create(C.byref(csr), _ptr(part), self.t, C.byref(o), C.byref(ctx))
        if rc != OK:
            raise EcgError(rc, "ecg_create")
        self._ctx = ctx

    @classmethod
    def from_problem(cls, p, **kw):
        return cls(p.rowptr, p.col, p.val, p.part, p.t, **kw)

    def close(self):
        if self._ctx is not None:
            self._lib.ecg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, b, x0=None, tol: float = 1e-8, maxit: int = 1000, x_out=None, raise_on_error=True) -> SolveResult:
        """b, x0, x_out: numpy arrays (host) or float64 CUDA tensors (device).
        Returns the iterate in x_out (allocated like b when None)."""
        if _is_torch_cuda(b):
            import torch

            _check_tensor(b, (self.n,), "b")
            if x0 is not None:
                _check_tensor(x0, (self.n,), "x0")
            if x_out is None:
                x_out = torch.empty_like(b)
        else:
            b = np.ascontiguousarray(b, dtype=np.float64)
            if x0 is not None:
                x0 = np.ascontiguousarray(x0, dtype=np.float64)
            if x_out is None:
                x_out = np.empty(self.n)
        res = _Result()
        rc = self._lib.ecg_solve(self._ctx, _ptr(b), _ptr(x0), _ptr(x_out), float(tol), int(maxit), C.byref(res))
        if rc < 0 and rc != EBREAKDOWN and raise_on_error:
            raise EcgError(rc, "ecg_solve")
        hist = np.ctypeslib.as_array(res.history, shape=(res.iters + 1,)).copy() if res.history else np.zeros(0)
        return SolveResult(
            x=x_out,
            iters=res.iters,
            switch_it=res.switch_it,
            status=rc,
            mem_vectors=res.mem_vectors,
            relres=res.relres,
            relres_true=res.relres_true,
            device_ms=res.device_ms,
            history=hist,
            restarts=res.restarts,
        )

    # ---------------------------------------------------------- profiling

    def profile(self, on: bool = True):
        rc = self._lib.ecg_profile_enable(self._ctx, 1 if on else 0)
        if rc != OK:
            raise EcgError(rc, "ecg_profile_enable")

    def profile_read(self) -> dict:
        ncls = self._lib.ecg_profile_read(self._ctx, -1, None, None, None)
        out = {}
        for c in range(ncls):
            name = C.c_char_p()
            ms = C.c_double()
            cnt = C.c_longlong()
            self._lib.ecg_profile_read(self._ctx, c, C.byref(name), C.byref(ms), C.byref(cnt))
            out[name.value.decode()] = (ms.value, cnt.value)
        return out

    # ------------------------------------------------------- step level

    def _rc(self, rc, what):
        if rc < 0:
            raise EcgError(rc, what)
        return rc

    def set_preconditioner(self, pblock, nblocks: int, kind: int = PREC_IC0):
        """Block Jacobi preconditioning with IC(0) diagonal blocks (Section 3,
        Algorithm 5); kind=PREC_NONE removes it."""
        import numpy as np

        if kind == PREC_NONE:
            self._rc(self._lib.ecg_set_preconditioner(self._ctx, None, 0, PREC_NONE), "ecg_set_preconditioner")
            return
        pb = np.ascontiguousarray(pblock, dtype=np.int32)
        if pb.shape != (self.n,):
            raise ValueError("pblock must have n entries")
        self._rc(
            self._lib.ecg_set_preconditioner(self._ctx, pb.ctypes.data_as(C.c_void_p), int(nblocks), int(kind)),
            "ecg_set_preconditioner",
        )

    def smooth(self, b, x, sweeps: int, omega: float = 0.8):
        """sweeps damped Jacobi sweeps on A x = b, x updated in place (device
        tensors)."""
        _check_tensor(b, (self.n,), "b")
        _check_tensor(x, (self.n,), "x")
        self._rc(self._lib.ecg_smooth(self._ctx, _ptr(b), _ptr(x), int(sweeps), float(omega)), "ecg_smooth")
        return x

    def prec_apply(self, X):
        """M^{-1} X for an n-vector or an n x w block (step-level call)."""
        import torch

        w = 1 if X.dim() == 1 else X.shape[1]
        _check_tensor(X, (self.n,) if X.dim() == 1 else (self.n, w), "X")
        out = torch.empty_like(X)
        self._rc(self._lib.ecg_op_prec_apply(self._ctx, _ptr(X), _ptr(out), int(w)), "ecg_op_prec_apply")
        return out

    def split(self, r, half: bool = False):
        import torch

        _check_tensor(r, (self.n,), "r")
        w = self.t // 2 if half else self.t
        W = torch.empty((self.n, w), dtype=torch.float64, device=r.device)
        self._rc(self._lib.ecg_op_split(self._ctx, _ptr(r), _ptr(W), 1 if half else 0), "ecg_op_split")
        return W

    def spmm(self, X):
        import torch

        w = X.shape[1]
        _check_tensor(X, (self.n, w), "X")
        Y = torch.empty_like(X)
        self._rc(self._lib.ecg_op_spmm(self._ctx, _ptr(X), _ptr(Y), int(w)), "ecg_op_spmm")
        return Y

    def tdot(self, Xs, Y):
        import torch

        if Y.dim() == 1:
            Y = Y.reshape(-1, 1)
        wy = Y.shape[1]
        _check_tensor(Y, (self.n, wy), "Y")
        for X in Xs:
            _check_tensor(X, (self.n, X.shape[1]), "X")
        m = len(Xs)
        ptrs = (C.c_void_p * m)(*[X.data_ptr() for X in Xs])
        ws = (C.c_int * m)(*[int(X.shape[1]) for X in Xs])
        tot = sum(int(X.shape[1]) for X in Xs)
        Cm = torch.empty((tot, wy), dtype=torch.float64, device=Y.device)
        self._rc(
            self._lib.ecg_op_tdot(self._ctx, m, C.cast(ptrs, C.c_void_p), C.cast(ws, C.c_void_p), _ptr(Y), int(wy), _ptr(Cm)),
            "ecg_op_tdot",
        )
        return Cm

    def cgs2(self, Qs, Vs, W):
        w = W.shape[1]
        _check_tensor(W, (self.n, w), "W")
        W = W.clone()
        m = len(Qs)
        qp = (C.c_void_p * m)(*[q.data_ptr() for q in Qs])
        vp = (C.c_void_p * m)(*[v.data_ptr() for v in Vs])
        ws = (C.c_int * m)(*[int(q.shape[1]) for q in Qs])
        for q, v in zip(Qs, Vs):
            _check_tensor(q, (self.n, q.shape[1]), "Q")
            _check_tensor(v, tuple(q.shape), "V")
        self._rc(
            self._lib.ecg_op_cgs2(
                self._ctx, m, C.cast(qp, C.c_void_p), C.cast(vp, C.c_void_p), C.cast(ws, C.c_void_p), _ptr(W), int(w)
            ),
            "ecg_op_cgs2",
        )
        return W

    def block_sub(self, Qs, Cm, W):
        """W - [Q_0 .. Q_{m-1}] C (ecg_op_block_sub) on a copy of W."""
        w = W.shape[1]
        _check_tensor(W, (self.n, w), "W")
        W = W.clone()
        m = len(Qs)
        for q in Qs:
            _check_tensor(q, (self.n, q.shape[1]), "Q")
        tot = sum(int(q.shape[1]) for q in Qs)
        _check_tensor(Cm, (tot, w), "C")
        qp = (C.c_void_p * m)(*[q.data_ptr() for q in Qs])
        ws = (C.c_int * m)(*[int(q.shape[1]) for q in Qs])
        self._rc(
            self._lib.ecg_op_block_sub(self._ctx, m, C.cast(qp, C.c_void_p), C.cast(ws, C.c_void_p), _ptr(Cm), _ptr(W),
                                       int(w)),
            "ecg_op_block_sub",
        )
        return W

    def a_orthonormalize(self, W):
        """Returns (W_k, A W_k, status)."""
        import torch

        w = W.shape[1]
        _check_tensor(W, (self.n, w), "W")
        W = W.clone()
        V = torch.empty_like(W)
        rc = self._lib.ecg_op_a_orthonormalize(self._ctx, _ptr(W), _ptr(V), int(w))
        if rc < 0 and rc != EBREAKDOWN:
            raise EcgError(rc, "ecg_op_a_orthonormalize")
        return W, V, rc

    def block_update(self, W, x, r):
        """Returns (W_k, V_k, x, r, rho, status); x and r are updated copies."""
        import torch

        w = W.shape[1]
        _check_tensor(W, (self.n, w), "W")
        _check_tensor(x, (self.n,), "x")
        _check_tensor(r, (self.n,), "r")
        W, x, r = W.clone(), x.clone(), r.clone()
        V = torch.empty_like(W)
        rho = C.c_double()
        rc = self._lib.ecg_op_block_update(self._ctx, _ptr(W), _ptr(V), int(w), _ptr(x), _ptr(r), C.byref(rho))
        if rc < 0 and rc != EBREAKDOWN:
            raise EcgError(rc, "ecg_op_block_update")
        return W, V, x, r, rho.value, rc

    def msdo_generate(self, r, P_prev, V_prev):
        import torch

        w = P_prev.shape[1]
        _check_tensor(r, (self.n,), "r")
        _check_tensor(P_prev, (self.n, w), "P_prev")
        _check_tensor(V_prev, (self.n, w), "V_prev")
        P = torch.empty_like(P_prev)
        self._rc(
            self._lib.ecg_op_msdo_generate(self._ctx, _ptr(r), _ptr(P_prev), _ptr(V_prev), int(w), _ptr(P)),
            "ecg_op_msdo_generate",
        )
        return P



class BatchSolver:
    """Many independent systems solved together by truncated SRE-CG2 in one
    persistent launch per round (ecg_batch_* in include/ecg.h)."""

    def __init__(
        self,
        problems,
        trunc: int = 2,
        ortho: int = PRE_CHOLQR,
        precision: int = MIXED,
        inner_tol: float = 1e-5,
        slice_height: int = 0,
        sort_window: int = 0,
        ctas_per_sm: int = 0,
        wait_limit_s: float = 1.0,
        debug_barrier_extra: int = 0,
        stream=None,
    ):
        self._lib = load()
        self._ctx = None
        ts = {int(p.t) for p in problems}
        if len(ts) != 1:
            raise ValueError("all systems of a batch share t")
        self.t = ts.pop()
        self.ns = [int(p.n) for p in problems]
        self._keep = []
        csrs = (_Csr * len(problems))()
        parts = (C.c_void_p * len(problems))()
        for k, p in enumerate(problems):
            rp = np.ascontiguousarray(p.rowptr, dtype=np.int64)
            ci = np.ascontiguousarray(p.col, dtype=np.int32)
            va = np.ascontiguousarray(p.val, dtype=np.float64)
            pt = np.ascontiguousarray(p.part, dtype=np.int32)
            self._keep += [rp, ci, va, pt]
            csrs[k] = _Csr(int(p.n), int(len(ci)), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0)
            parts[k] = pt.ctypes.data
        o = _BatchOpts()
        self._lib.ecg_batch_default_opts(C.byref(o))
        o.trunc, o.ortho, o.precision, o.inner_tol = int(trunc), int(ortho), int(precision), float(inner_tol)
        o.slice_height, o.sort_window, o.ctas_per_sm = int(slice_height), int(sort_window), int(ctas_per_sm)
        o.wait_limit_s, o.debug_barrier_extra = float(wait_limit_s), int(debug_barrier_extra)
        o.stream = stream
        ctx = C.c_void_p()
        rc = self._lib.ecg_batch_create(len(problems), csrs, parts, self.t, C.byref(o), C.byref(ctx))
        self._keep = []
        if rc != OK:
            raise EcgError(rc, "ecg_batch_create")
        self._ctx = ctx

    def layout(self) -> dict:
        c, s, g, ms, gr = _I(), _I(), _I(), _D(), _I()
        self._lib.ecg_batch_layout(self._ctx, C.byref(c), C.byref(s), C.byref(g), C.byref(ms), C.byref(gr))
        return {"slice_height": c.value, "sort_window": s.value, "ctas": g.value, "spmm_ms": ms.value,
                "graph": bool(gr.value)}

    def solve(self, bs, x0s=None, tol: float = 1e-8, maxit: int = 1000, outs=None):
        """bs: list of n_s arrays (numpy, or torch CUDA tensors).  Returns
        (status of the batch, list of SolveResult)."""
        ns = len(self.ns)
        dev = _is_torch_cuda(bs[0])
        if outs is None:
            if dev:
                import torch

                outs = [torch.empty(n, dtype=torch.float64, device=bs[0].device) for n in self.ns]
            else:
                outs = [np.empty(n) for n in self.ns]
        keep = [np.ascontiguousarray(b, dtype=np.float64) if not dev else b for b in bs]
        bp = (C.c_void_p * ns)(*[_ptr(b) for b in keep])
        xp = None
        if x0s is not None:
            keep0 = [np.ascontiguousarray(x, dtype=np.float64) if not dev else x for x in x0s]
            xp = (C.c_void_p * ns)(*[_ptr(x) for x in keep0])
        op = (C.c_void_p * ns)(*[_ptr(x) for x in outs])
        res = (_Result * ns)()
        rc = self._lib.ecg_batch_solve(self._ctx, bp, xp, op, float(tol), int(maxit), res)
        if rc < 0 and rc not in (EBREAKDOWN, ETIMEOUT):
            raise EcgError(rc, "ecg_batch_solve")
        out = []
        for k in range(ns):
            r = res[k]
            hist = np.ctypeslib.as_array(r.history, shape=(r.iters + 1,)).copy() if r.history else np.zeros(1)
            out.append(
                SolveResult(
                    x=outs[k], iters=r.iters, switch_it=0, status=r.status, mem_vectors=r.mem_vectors,
                    relres=r.relres, relres_true=r.relres_true, device_ms=r.device_ms, history=hist,
                )
            )
        return rc, out

    def close(self):
        if self._ctx is not None:
            self._lib.ecg_batch_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tdot_noalloc(Xs, Y, out=None, stream=None):
    """[X_0 .. X_{m-1}]^T Y through ecg_tdot_noalloc, which allocates no
    device memory of its own (its scratch is a static array inside the
    library).  Xs: a non-empty list of float64 CUDA tensors n x w_j; Y:
    n x wy (or n); all on one device, on which the call runs.  out: a
    preallocated contiguous float64 (sum w_j) x wy tensor on that device, or
    None to let torch allocate the result here in Python.  stream: a
    cudaStream_t handle, or None for torch's current stream on that device.
    Returns (status, out)."""
    import torch

    lib = load()
    if len(Xs) == 0:
        raise ValueError("tdot_noalloc needs at least one block X_j")
    if Y.dim() == 1:
        Y = Y.reshape(-1, 1)
    n, wy = int(Y.shape[0]), int(Y.shape[1])
    _check_tensor(Y, (n, wy), "Y")
    for X in Xs:
        _check_tensor(X, (n, X.shape[1]), "X")
        if X.device != Y.device:
            raise ValueError("every X_j must be on Y's device")
    m = len(Xs)
    ptrs = (C.c_void_p * m)(*[X.data_ptr() for X in Xs])
    ws = (C.c_int * m)(*[int(X.shape[1]) for X in Xs])
    tot = sum(int(X.shape[1]) for X in Xs)
    if out is None:
        out = torch.empty((tot, wy), dtype=torch.float64, device=Y.device)
    _check_tensor(out, (tot, wy), "out")
    if out.device != Y.device:
        raise ValueError("out must be on Y's device")
    with torch.cuda.device(Y.device):
        if stream is None:
            stream = torch.cuda.current_stream(Y.device).cuda_stream
        rc = lib.ecg_tdot_noalloc(n, m, C.cast(ptrs, C.c_void_p), C.cast(ws, C.c_void_p), _ptr(Y), wy, _ptr(out),
                                  stream)
    return rc, out


def probe_fp64(iters: int = 20000) -> float:
    """This GPU's FP64 FMA rate in TFLOP/s (ecg_probe_fp64), the bound of the
    FP64 block kernels that run on CUDA cores."""
    lib = load()
    out = C.c_double(0.0)
    rc = lib.ecg_probe_fp64(int(iters), C.byref(out))
    if rc != OK:
        raise EcgError(rc, "ecg_probe_fp64")
    return float(out.value)
