"""ctypes front end of the plain FP64 CPU oracle (``ecg_oracle.c``).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
path.  Every function here marshals numpy arrays and calls the C oracle; the
arithmetic is all in C, following the paper (S. Moufawad, "Flexibly Enlarged
Conjugate Gradient methods", arXiv 2305.19013):

- ``spmv``/``spmm``: the products A x and A W (Algorithm 1 lines 1, 6).
- ``split``/``split_half``: [T^t(r)] and [T^{t/2}(r)] (eq. (Tt), Section 4).
- ``block_tdot``/``block_sub``: X^T Y and W - Q C (block inner products and
  the CGS update, Sections 2-3).
- ``msdo_direction``: the MSDO-CG block [T(r)] + P_{k-1} diag(beta) with
  beta = -V_{k-1}^T r (Algorithm 2).
- ``cholesky``/``householder_qr``/``a_orthonormalize``/``cgs2``: the
  A-orthonormalisation (Section 2.1, Section 5).
- ``ecg_solve``: SRE-CG2, MSDO-CG, modified MSDO-CG, truncated and flexible
  forms (Algorithms 1-4, Section 3).
- ``cg_solve``: classical CG (Section 1).
- ``becg_solve``: the block-residual enlarged CG mentioned in Section 1
  (R_0 = [T^t(r_0)], x = x_0 + sum of the block solution's columns).
- ``BlockJacobi``: the block Jacobi preconditioner M = L L^T of Section 3
  ("Preconditioned versions") and Section 5, with exact Cholesky or IC(0)
  diagonal blocks; ``ecg_solve(..., prec=...)`` runs the preconditioned
  methods (eq. (zsre2), (zmsd2), Algorithm 5).
- ``dense_spd_solve``: Cholesky solve of a small dense SPD system.

Parity of the solver against the paper's own iteration counts is unpinned
(its test matrices are not available); every function is pinned by the
``-m "not gpu"`` tests to closed forms, invariants, library routines and
brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ecg_oracle.c")
_LIB = os.path.join(_HERE, "libecg_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libecg_oracle_omp.so")  # same source, -fopenmp

OK, ENOCONV, EINVAL, ENOMEM, EBREAKDOWN, ENOTSPD = 0, 1, -1, -2, -4, -5

_libs = {}          # path -> loaded CDLL
_use_omp = False    # route calls to the OpenMP build (see threads())


def _compile(out, extra):
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"]
    )
    os.replace(tmp, out)


def _stale(lib):
    return not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction): the
    single-threaded library and, when the compiler offers OpenMP, the same
    source with -fopenmp.  Both sum every reduction over rows in the same
    fixed chunks, so they return the same bits."""
    if force or _stale(_LIB):
        _compile(_LIB, [])
    if force or _stale(_LIB_OMP):
        try:
            _compile(_LIB_OMP, ["-fopenmp"])
        except (subprocess.CalledProcessError, OSError):
            pass  # no OpenMP: threads() stays at one thread
    return _LIB


def have_threads() -> bool:
    """True when the OpenMP build of the oracle exists."""
    build()
    return os.path.exists(_LIB_OMP)


def threads(n: int | None = None) -> int:
    """Route oracle calls to the OpenMP build with n threads (n > 1; None:
    every core) or back to the single-threaded build (n == 1).  Returns the
    number of threads now in use.  The results do not change."""
    global _use_omp
    if n == 1 or not have_threads():
        _use_omp = False
        return 1
    _use_omp = True
    return int(_load().or_set_threads(int(n) if n else os.cpu_count() or 1))


class _Res(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("switch_it", C.c_int),
        ("status", C.c_int),
        ("mem_vectors", C.c_int64),
        ("relres", C.c_double),
        ("relres_true", C.c_double),
        ("restarts", C.c_int),
    ]


class _Restart(C.Structure):
    _fields_ = [("every", C.c_int), ("tol", C.c_double), ("max_count", C.c_int), ("at_switch", C.c_int)]


_P = C.c_void_p
_I64 = C.c_int64
_INT = C.c_int
_D = C.c_double


def _load():
    path = _LIB_OMP if _use_omp else _LIB
    lib = _libs.get(path)
    if lib is not None:
        return lib
    build()
    lib = C.CDLL(path)
    sigs = {
        "or_set_threads": (_INT, [_INT]),
        "or_spmv": (None, [_I64, _P, _P, _P, _P, _P]),
        "or_spmm": (None, [_I64, _P, _P, _P, _INT, _P, _P]),
        "or_split": (None, [_I64, _P, _INT, _P, _P]),
        "or_split_half": (None, [_I64, _P, _INT, _P, _P]),
        "or_block_tdot": (None, [_I64, _INT, _P, _INT, _P, _P]),
        "or_block_sub": (None, [_I64, _INT, _P, _INT, _P, _P]),
        "or_right_trsm": (None, [_I64, _INT, _P, _P]),
        "or_cholesky": (_INT, [_INT, _P, _P]),
        "or_householder_qr": (_INT, [_I64, _INT, _P, _P, _P]),
        "or_dense_spd_solve": (_INT, [_INT, _P, _P, _P]),
        "or_a_orthonormalize": (_INT, [_I64, _P, _P, _P, _INT, _INT, _P, _P]),
        "or_cgs2": (_INT, [_I64, _INT, _P, _P, _P, _INT, _P]),
        "or_ecg_solve": (
            _INT,
            [_I64, _P, _P, _P, _P, _INT, _INT, _INT, _D, _INT, _P, _P, _D, _INT, _P, _P, _P, _P, _I64, _P, _P, _P,
             _P],
        ),
        "or_prec_setup": (_INT, [_I64, _P, _P, _P, _P, _INT, _INT, C.POINTER(C.c_void_p)]),
        "or_prec_free": (None, [_P]),
        "or_prec_nnz": (_I64, [_P]),
        "or_prec_export": (None, [_P, _P, _P, _P]),
        "or_prec_lsolve": (None, [_P, _INT, _P]),
        "or_prec_ltsolve": (None, [_P, _INT, _P]),
        "or_prec_apply": (None, [_P, _INT, _P]),
        "or_cg_solve": (_INT, [_I64, _P, _P, _P, _P, _P, _D, _INT, _P, _P, _P, _P]),
        "or_becg_solve": (_INT, [_I64, _P, _P, _P, _P, _INT, _INT, _INT, _P, _P, _D, _INT, _P, _P, _P, _P, _P]),
        "or_mem_flexible": (_I64, [_INT, _INT, _INT]),
        "or_msdo_direction": (None, [_I64, _INT, _P, _P, _P, _P, _P]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _libs[path] = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _csr(A):
    """Accept a scipy CSR matrix or a (rowptr, col, val) triple."""
    if hasattr(A, "indptr"):
        return (
            np.ascontiguousarray(A.indptr, dtype=np.int64),
            np.ascontiguousarray(A.indices, dtype=np.int32),
            _f64(A.data),
            A.shape[0],
        )
    rowptr, col, val = A
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    return rowptr, np.ascontiguousarray(col, dtype=np.int32), _f64(val), len(rowptr) - 1


def spmv(A, x):
    rp, ci, va, n = _csr(A)
    x = _f64(x)
    y = np.empty(n)
    _load().or_spmv(n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def spmm(A, X):
    rp, ci, va, n = _csr(A)
    X = _f64(X)
    w = X.shape[1]
    Y = np.empty((n, w))
    _load().or_spmm(n, _p(rp), _p(ci), _p(va), w, _p(X), _p(Y))
    return Y


def split(part, t, r):
    part = np.ascontiguousarray(part, dtype=np.int32)
    r = _f64(r)
    W = np.empty((len(r), t))
    _load().or_split(len(r), _p(part), t, _p(r), _p(W))
    return W


def split_half(part, t, r):
    part = np.ascontiguousarray(part, dtype=np.int32)
    r = _f64(r)
    W = np.empty((len(r), t // 2))
    _load().or_split_half(len(r), _p(part), t, _p(r), _p(W))
    return W


def block_tdot(X, Y):
    X = _f64(X if X.ndim == 2 else X[:, None])
    Y = _f64(Y if Y.ndim == 2 else Y[:, None])
    Cm = np.empty((X.shape[1], Y.shape[1]))
    _load().or_block_tdot(X.shape[0], X.shape[1], _p(X), Y.shape[1], _p(Y), _p(Cm))
    return Cm


def block_sub(Q, Cm, W):
    Q, Cm, W = _f64(Q), _f64(Cm), _f64(W).copy()
    _load().or_block_sub(W.shape[0], Q.shape[1], _p(Q), W.shape[1], _p(Cm), _p(W))
    return W


def msdo_direction(part, t, r, P_prev, V_prev, z=None):
    """MSDO-CG direction (Algorithm 2 lines 6-7): returns (P, beta) with
    beta = -V_prev^T z (z = r unless given, e.g. M^{-1} r) and
    P = [T(r)] + P_prev diag(beta); T = T^t when P_prev has t columns,
    T^{t/2} when it has t/2.  The solver builds its MSDO blocks with the same
    C function."""
    P_prev, V_prev, r = _f64(P_prev), _f64(V_prev), _f64(r)
    z = r if z is None else _f64(z)
    n, w = P_prev.shape
    P = split(part, t, r) if w == t else split_half(part, t, r)
    beta = np.empty(w)
    _load().or_msdo_direction(n, w, _p(P_prev), _p(V_prev), _p(z), _p(beta), _p(P))
    return P, beta


def right_trsm(R, X):
    R, X = _f64(R), _f64(X).copy()
    _load().or_right_trsm(X.shape[0], X.shape[1], _p(R), _p(X))
    return X


def cholesky(G):
    """Upper R with G = R^T R; returns (R, status) with status 0 or j+1."""
    G = _f64(G)
    w = G.shape[0]
    R = np.empty((w, w))
    st = _load().or_cholesky(w, _p(G), _p(R))
    return R, st


def householder_qr(W):
    W = _f64(W)
    n, w = W.shape
    Q = np.empty((n, w))
    R = np.empty((w, w))
    st = _load().or_householder_qr(n, w, _p(W), _p(Q), _p(R))
    return Q, R, st


def dense_spd_solve(A, b):
    A, b = _f64(A), _f64(b)
    x = np.empty(len(b))
    st = _load().or_dense_spd_solve(len(b), _p(A), _p(b), _p(x))
    return x, st


def a_orthonormalize(A, W, mode=0):
    """Returns (W_k, A W_k, status)."""
    rp, ci, va, n = _csr(A)
    W = _f64(W).copy()
    V = np.empty_like(W)
    st = _load().or_a_orthonormalize(n, _p(rp), _p(ci), _p(va), W.shape[1], mode, _p(W), _p(V))
    return W, V, st


def cgs2(Qs, Vs, W):
    """Two passes of block CGS in the A-inner product against blocks Qs (with
    Vs = A Qs)."""
    W = _f64(W).copy()
    Qs = [_f64(q) for q in Qs]
    Vs = [_f64(v) for v in Vs]
    m = len(Qs)
    qp = (C.c_void_p * max(m, 1))(*[q.ctypes.data for q in Qs])
    vp = (C.c_void_p * max(m, 1))(*[v.ctypes.data for v in Vs])
    ws = np.array([q.shape[1] for q in Qs] or [0], dtype=np.int32)
    st = _load().or_cgs2(W.shape[0], m, C.cast(qp, C.c_void_p), C.cast(vp, C.c_void_p), _p(ws), W.shape[1], _p(W))
    return W, st


@dataclass
class OracleResult:
    x: np.ndarray
    iters: int
    switch_it: int
    status: int
    mem_vectors: int
    relres: float
    relres_true: float
    history: np.ndarray
    xhist: np.ndarray | None = None
    basis: list | None = None
    restarts: int = 0


VARIANTS = {"sre": 0, "msdo": 1, "modmsdo": 2}


def ecg_solve(
    A,
    part,
    t,
    b,
    x0=None,
    tol=1e-8,
    maxit=1000,
    variant="sre",
    trunc=0,
    switch_tol=0.0,
    ortho=0,
    keep_x=False,
    keep_basis=False,
    restart_every=0,
    restart_tol=0.0,
    restart_max=0,
    restart_at_switch=False,
    prec=None,
):
    """Enlarged CG (Algorithms 1-4, their truncated and restarted forms of
    Section 3, and with ``prec`` a ``BlockJacobi`` the preconditioned forms
    of Section 3 and Algorithm 5).  ``maxit`` is the paper's k_max: at most
    maxit - 1 iterations run."""
    rp, ci, va, n = _csr(A)
    part = np.ascontiguousarray(part, dtype=np.int32)
    b = _f64(b)
    x0a = None if x0 is None else _f64(x0)
    x = np.empty(n)
    hist = np.zeros(max(maxit, 1))
    xh = np.zeros((max(maxit - 1, 1), n)) if keep_x else None
    cap = n * t * max(maxit - 1, 1) if keep_basis else 0
    basis = np.zeros(cap) if keep_basis else None
    widths = np.zeros(max(maxit, 1), dtype=np.int32)
    res = _Res()
    rs = _Restart(int(restart_every), float(restart_tol), int(restart_max), 1 if restart_at_switch else 0)
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _load().or_ecg_solve(
        n, _p(rp), _p(ci), _p(va), _p(part), t, v, trunc, switch_tol, ortho, _p(b), _p(x0a), tol, maxit,
        _p(x), _p(hist), _p(xh), _p(basis), cap, _p(widths), C.byref(rs),
        None if prec is None else prec._h, C.byref(res),
    )
    blocks = None
    if keep_basis:
        blocks, off = [], 0
        for k in range(res.iters):
            w = int(widths[k])
            blocks.append(basis[off : off + n * w].reshape(n, w).copy())
            off += n * w
    return OracleResult(
        x=x,
        iters=res.iters,
        switch_it=res.switch_it,
        status=res.status,
        mem_vectors=res.mem_vectors,
        relres=res.relres,
        relres_true=res.relres_true,
        history=hist[: res.iters + 1].copy(),
        xhist=None if xh is None else xh[: res.iters].copy(),
        basis=blocks,
        restarts=res.restarts,
    )


def becg_solve(A, part, t, b, x0=None, tol=1e-8, maxit=1000, trunc=0, ortho=0, keep_x=False):
    """Block-residual enlarged CG (Section 1): SRE-CG's direction blocks,
    t x t coefficients alpha_k = W_k^T R_{k-1}, x = x_0 + X_k 1.  Returns an
    OracleResult whose ``basis`` holds the final n x t block solution X."""
    rp, ci, va, n = _csr(A)
    part = np.ascontiguousarray(part, dtype=np.int32)
    b = _f64(b)
    x0a = None if x0 is None else _f64(x0)
    x = np.empty(n)
    hist = np.zeros(max(maxit, 1))
    xh = np.zeros((max(maxit - 1, 1), n)) if keep_x else None
    Xb = np.zeros((n, t))
    res = _Res()
    _load().or_becg_solve(
        n, _p(rp), _p(ci), _p(va), _p(part), t, trunc, ortho, _p(b), _p(x0a), tol, maxit, _p(x), _p(hist), _p(xh),
        _p(Xb), C.byref(res),
    )
    return OracleResult(
        x=x,
        iters=res.iters,
        switch_it=0,
        status=res.status,
        mem_vectors=res.mem_vectors,
        relres=res.relres,
        relres_true=res.relres_true,
        history=hist[: res.iters + 1].copy(),
        xhist=None if xh is None else xh[: res.iters].copy(),
        basis=[Xb],
    )


def cg_solve(A, b, x0=None, tol=1e-8, maxit=1000, keep_x=False):
    rp, ci, va, n = _csr(A)
    b = _f64(b)
    x0a = None if x0 is None else _f64(x0)
    x = np.empty(n)
    hist = np.zeros(max(maxit, 1))
    xh = np.zeros((max(maxit - 1, 1), n)) if keep_x else None
    res = _Res()
    _load().or_cg_solve(n, _p(rp), _p(ci), _p(va), _p(b), _p(x0a), tol, maxit, _p(x), _p(hist), _p(xh), C.byref(res))
    return OracleResult(
        x=x,
        iters=res.iters,
        switch_it=0,
        status=res.status,
        mem_vectors=0,
        relres=res.relres,
        relres_true=res.relres_true,
        history=hist[: res.iters + 1].copy(),
        xhist=None if xh is None else xh[: res.iters].copy(),
    )


def mem_flexible(t, iters, switch_it):
    return int(_load().or_mem_flexible(t, iters, switch_it))


PREC_CHOL, PREC_IC0 = 0, 1


class BlockJacobi:
    """Block Jacobi preconditioner M = L L^T, L = diag(L_1, ..., L_nb)
    (Section 3 "Preconditioned versions"; eq. (cholprec), Section 5).
    ``pblock[i]`` is the diagonal block of row i; ``kind`` is PREC_CHOL (the
    exact Cholesky factor of each diagonal block) or PREC_IC0 (incomplete
    Cholesky with zero fill)."""

    def __init__(self, A, pblock, nb, kind=PREC_IC0):
        rp, ci, va, n = _csr(A)
        self.n = n
        self._keep = (rp, ci, va)
        pb = np.ascontiguousarray(pblock, dtype=np.int32)
        h = C.c_void_p()
        rc = _load().or_prec_setup(n, _p(rp), _p(ci), _p(va), _p(pb), int(nb), int(kind), C.byref(h))
        if rc != OK:
            raise ValueError(f"or_prec_setup failed: {rc}")
        self._h = h
        self.status = rc

    def __del__(self):
        try:
            if self._h:
                _load().or_prec_free(self._h)
                self._h = None
        except Exception:
            pass

    def factor(self):
        """L in global coordinates as (I, J, V) triplets."""
        nnz = _load().or_prec_nnz(self._h)
        I = np.zeros(nnz, dtype=np.int64)
        J = np.zeros(nnz, dtype=np.int64)
        V = np.zeros(nnz)
        _load().or_prec_export(self._h, _p(I), _p(J), _p(V))
        return I, J, V

    def _run(self, name, X):
        X = _f64(X).copy()
        w = 1 if X.ndim == 1 else X.shape[1]
        getattr(_load(), name)(self._h, w, _p(X))
        return X

    def lsolve(self, X):
        """L^{-1} X."""
        return self._run("or_prec_lsolve", X)

    def ltsolve(self, X):
        """L^{-T} X."""
        return self._run("or_prec_ltsolve", X)

    def apply(self, X):
        """M^{-1} X = L^{-T} L^{-1} X."""
        return self._run("or_prec_apply", X)
