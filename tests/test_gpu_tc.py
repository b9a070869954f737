"""The FP64 CGS products on the tensor cores (ecg_tc.cuh) against the oracle.

The tensor-core update W -= Q C (ecg_op_block_sub with tensor_cores on,
block width 16, window of 16 or 32 columns) is compared entry by entry with
the oracle's block_sub.  Its error bound is FP64's: |got - ref| <= 1e-12 x
(|W| + sum_a |Q_a| |C_a|) entry by entry, the tolerance of the other block
products.  The inputs span rows of very different magnitude, rows whose
entries span many binades, zero rows, ragged row counts (several 128-row
tiles per CTA and a partial last tile), and a C with one tiny column.
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_19013_gb300 import ecg

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    ecg.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def inputs(n, widths, seed, spread):
    rng = np.random.default_rng(seed)
    Qs = [rng.standard_normal((n, w)) for w in widths]
    X = rng.standard_normal((n, 16))
    if spread:
        rows = 10.0 ** rng.uniform(-8, 8, n)  # rows of very different size
        Qs = [q * rows[:, None] * 10.0 ** rng.uniform(-5, 5, q.shape) for q in Qs]  # binades within a row
        X = X * rows[:, None]
        for q in Qs:
            q[::97] = 0.0  # zero rows
    tot = sum(widths)
    Cm = rng.standard_normal((tot, 16))
    Cm[:, 3] *= 1e-9
    return Qs, Cm, X


@pytest.mark.parametrize("n,widths,spread", [(1296, [16, 16], False), (1296, [16], False),
                                             (100_003, [16, 16], True), (5000, [16, 16], True),
                                             (777, [8, 8, 16], False)])
def test_tensor_core_block_sub_matches_oracle(n, widths, spread):
    Qs, Cm, X = inputs(n, widths, seed=n + len(widths), spread=spread)
    ref = O.block_sub(np.hstack(Qs), Cm, X)
    bound = 1e-12 * (np.abs(X) + np.abs(np.hstack(Qs)) @ np.abs(Cm))
    part = np.zeros(n, dtype=np.int32)
    rowptr = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    val = np.ones(n)
    for tcores in (True, False):
        with ecg.Solver(rowptr, col, val, part, 1, tensor_cores=tcores) as s:
            got = s.block_sub([dev(q) for q in Qs], dev(Cm), dev(X)).cpu().numpy()
        assert np.all(np.abs(got - ref) <= bound), (tcores, np.max(np.abs(got - ref) / np.maximum(bound, 1e-300)))


def test_tensor_core_block_sub_propagates_nan():
    n = 300
    Qs, Cm, X = inputs(n, [16, 16], seed=5, spread=False)
    Qs[0][17, 3] = np.nan
    rowptr = np.arange(n + 1, dtype=np.int64)
    with ecg.Solver(rowptr, np.arange(n, dtype=np.int32), np.ones(n), np.zeros(n, np.int32), 1) as s:
        got = s.block_sub([dev(q) for q in Qs], dev(Cm), dev(X)).cpu().numpy()
    assert np.all(np.isnan(got[17]))
    ref = O.block_sub(np.hstack(Qs), Cm, X)
    ok = np.ones(n, bool)
    ok[17] = False
    assert np.allclose(got[ok], ref[ok], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n,widths,spread", [(1296, [16, 16], False), (1296, [16], False),
                                             (100_003, [16, 16], True), (40_000, [8, 8, 16], False)])
def test_tensor_core_tdot_matches_oracle(n, widths, spread):
    """C = [V_0 .. V_{m-1}]^T Y (ecg_op_tdot, Y of width 16) against the
    oracle's block_tdot: |got - ref| <= 1e-12 sum |v||y| entry by entry."""
    Vs, _, Y = inputs(n, widths, seed=7 * n + len(widths), spread=spread)
    V = np.hstack(Vs)
    ref = O.block_tdot(V, Y)
    bound = 1e-12 * (np.abs(V).T @ np.abs(Y))
    rowptr = np.arange(n + 1, dtype=np.int64)
    for tcores in (True, False):
        with ecg.Solver(rowptr, np.arange(n, dtype=np.int32), np.ones(n), np.zeros(n, np.int32), 1,
                        tensor_cores=tcores) as s:
            got = s.tdot([dev(v) for v in Vs], dev(Y)).cpu().numpy()
        assert np.all(np.abs(got - ref) <= bound), (tcores, np.max(np.abs(got - ref) / np.maximum(bound, 1e-300)))


def test_tensor_core_solve_matches_cuda_core_solve():
    """A whole truncated SRE-CG solve (t = 16, window of 2 blocks, both
    CGS products on the tensor cores) against the oracle, and against the
    same solve on CUDA-core FP64 FMAs: same iteration count within the
    envelope of parity_util, x within the oracle's spread."""
    from paper_2305_19013_gb300 import workloads as Wk
    from parity_util import envelope_check

    p = Wk.blocky_diffusion2d(64, 16, blocks=8, seed=17)
    res = {}
    for tcores in (True, False):
        with ecg.Solver.from_problem(p, trunc=2, tensor_cores=tcores) as s:
            g = s.solve(dev(p.b), tol=1e-8, maxit=3000)
        res[tcores] = g
        envelope_check(p, g.iters, g.history, g.x.cpu().numpy(), dict(trunc=2), 3000)
    assert abs(res[True].iters - res[False].iters) <= max(2, res[False].iters // 50)
