"""The allocation-free block inner product, ecg_tdot_noalloc.

Some callers cannot let a library allocate device memory when they need a
result: a service that has already reserved the whole GPU for its own pool
allocator (a cudaMalloc from the library would fail or fragment that pool),
or a latency-critical loop that must not enter cudaMalloc/cudaFree, which can
block or synchronise the device.  ecg_tdot_noalloc serves them: it keeps its
scratch in a static device array inside the library.

This file is collected last, so that a run stopping at the first failure has
already run every other test.  It passes alone in a fresh process and after
the other tests: the first call on the device sets up the array's address,
and every later call reuses the same array.  One test runs the call in a
new Python process before any solver context exists.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle as O
from paper_2305_19013_gb300 import ecg
from paper_2305_19013_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def bound(Xs, Y):
    # the block-product tolerance of the parity tests: 1e-12 sum |x||y|
    return 1e-12 * (np.abs(np.hstack(Xs)).T @ np.abs(Y))


def test_noalloc_tdot_matches_context_tdot_and_oracle_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    p = W.random_spd_grid(36, 16, seed=41)  # 1296 rows: ragged row tiles
    rng = np.random.default_rng(42)
    calls = [([16, 16, 8, 3], 16), ([64, 32, 5], 4), ([128, 100], 64), ([16, 16], 32)]
    with ecg.Solver.from_problem(p) as s:
        for widths, wy in calls:
            Xs = [rng.standard_normal((p.n, w)) for w in widths]
            Y = rng.standard_normal((p.n, wy))
            ref = s.tdot([dev(x) for x in Xs], dev(Y)).cpu().numpy()
            orc = O.block_tdot(np.hstack(Xs), Y)
            rc, got = ecg.tdot_noalloc([dev(x) for x in Xs], dev(Y))
            assert rc == ecg.OK
            got = got.cpu().numpy()
            assert got.shape == ref.shape == orc.shape
            assert np.all(np.abs(got - ref) <= bound(Xs, Y))
            assert np.all(np.abs(got - orc) <= bound(Xs, Y))


def test_noalloc_tdot_in_a_fresh_process_before_any_context():
    """Widths 1, 2, 8 and 32 (32 needs more than 48 KiB of shared memory),
    each called twice, in a process that never creates a solver context;
    compared with the oracle."""
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    code = textwrap.dedent(
        """
        import sys
        sys.path.insert(0, %r)
        import numpy as np, torch
        import oracle as O
        from paper_2305_19013_gb300 import ecg
        rng = np.random.default_rng(7)
        n = 5000
        for wy in (1, 2, 8, 32, 32, 1):
            Xs = [rng.standard_normal((n, w)) for w in (16, 16, 7)]
            Y = rng.standard_normal((n, wy))
            rc, got = ecg.tdot_noalloc([torch.from_numpy(x).cuda() for x in Xs], torch.from_numpy(Y).cuda())
            assert rc == ecg.OK, rc
            ref = O.block_tdot(np.hstack(Xs), Y)
            tol = 1e-12 * (np.abs(np.hstack(Xs)).T @ np.abs(Y))
            assert np.all(np.abs(got.cpu().numpy() - ref) <= tol), wy
        print("fresh-process noalloc ok")
        """
        % ROOT
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process noalloc ok" in r.stdout


def test_noalloc_tdot_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    n = 100
    Y = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    too_wide = [torch.zeros((n, 128), dtype=torch.float64, device="cuda") for _ in range(3)]  # 384 columns
    rc, _ = ecg.tdot_noalloc(too_wide, Y)
    assert rc == ecg.EINVAL
    rc, _ = ecg.tdot_noalloc([torch.zeros((n, 129), dtype=torch.float64, device="cuda")], Y)
    assert rc == ecg.EINVAL
    with pytest.raises(ValueError):
        ecg.tdot_noalloc([torch.zeros((n, 4), dtype=torch.float64, device="cuda")], Y,
                         out=torch.zeros((3, 4), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        ecg.tdot_noalloc([], Y)
