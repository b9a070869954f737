"""The OpenMP build of the oracle against its single-threaded build.

Both builds come from the same C source; every sum over rows is taken in
fixed chunks of rows added in chunk order, so the number of threads cannot
change a result.  These cases have several chunks and a ragged last one
(10,000 rows), and cover every function the full-size parity tests and the
benchmark's CPU baseline run through threads: the products, the Householder
QR, both Pre-CholQR readings, the solvers (SRE, MSDO, flexible, truncated)
and the block Jacobi
preconditioner (setup, substitutions, preconditioned solve).  CPU only.
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_19013_gb300 import workloads as W

pytestmark = pytest.mark.skipif(not O.have_threads(), reason="the compiler has no OpenMP")


def both(fn, nthreads=4):
    O.threads(1)
    a = fn()
    try:
        assert O.threads(nthreads) == nthreads
        b = fn()
    finally:
        O.threads(1)
    return a, b


def test_products_and_qr_bitwise_equal():
    p = W.random_spd_grid(100, 8, seed=11)
    A = p.scipy()
    rng = np.random.default_rng(3)
    X = rng.standard_normal((p.n, 16))
    Y = rng.standard_normal((p.n, 8))
    a, b = both(lambda: (O.spmm(A, X), O.block_tdot(X, Y), O.householder_qr(X), O.a_orthonormalize(A, X, 0),
                         O.a_orthonormalize(A, X, 2)))
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    for k in (2, 3, 4):
        for u, v in zip(a[k], b[k]):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("variant,trunc,switch,ortho", [("sre", 2, 0.0, 0), ("msdo", 3, 0.0, 0), ("sre", 0, 1e-4, 0),
                                                        ("sre", 2, 0.0, 2)])
def test_solves_bitwise_equal(variant, trunc, switch, ortho):
    p = W.random_spd_grid(100, 8, seed=12)
    A = p.scipy()

    def run():
        return O.ecg_solve(A, p.part, p.t, p.b, tol=1e-8, maxit=60, variant=variant, trunc=trunc, switch_tol=switch,
                           ortho=ortho)

    a, b = both(run)
    assert a.iters == b.iters and a.status == b.status and a.switch_it == b.switch_it
    assert np.array_equal(a.x, b.x)
    assert np.array_equal(a.history, b.history)


def test_preconditioner_bitwise_equal():
    p = W.blocky_diffusion2d(100, 4, blocks=4, seed=13)
    A = p.scipy()
    pb = W.jacobi_blocks(p, 16)

    def run():
        M = O.BlockJacobi(A, pb, 16, O.PREC_IC0)
        Z = M.apply(np.ascontiguousarray(np.eye(p.n, 4)))
        r = O.ecg_solve(A, p.part, p.t, p.b, tol=1e-8, maxit=80, trunc=2, prec=M)
        return M.factor()[2], Z, r

    a, b = both(run)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert a[2].iters == b[2].iters
    assert np.array_equal(a[2].x, b[2].x)
    assert np.array_equal(a[2].history, b[2].history)
