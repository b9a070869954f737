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
and every later call reuses the same array.
"""
import numpy as np
import pytest

from paper_2305_19013_gb300 import ecg
from paper_2305_19013_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_noalloc_tdot_matches_context_tdot_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    p = W.random_spd_grid(36, 16, seed=41)  # 1296 rows: ragged row tiles
    rng = np.random.default_rng(42)
    calls = [([16, 16, 8, 3], 16), ([64, 32, 5], 4), ([128, 100], 64)]
    with ecg.Solver.from_problem(p) as s:
        for widths, wy in calls:
            Xs = [rng.standard_normal((p.n, w)) for w in widths]
            Y = rng.standard_normal((p.n, wy))
            ref = s.tdot([dev(x) for x in Xs], dev(Y)).cpu().numpy()
            rc, got = ecg.tdot_noalloc([dev(x) for x in Xs], dev(Y))
            assert rc == ecg.OK
            got = got.cpu().numpy()
            Xc = np.hstack(Xs)
            bound = 1e-12 * (np.abs(Xc).T @ np.abs(Y))  # the block-product tolerance of the parity tests
            assert got.shape == ref.shape
            assert np.all(np.abs(got - ref) <= bound)


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
