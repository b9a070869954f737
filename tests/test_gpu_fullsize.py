"""Parity at the sizes the benchmark runs, against the threaded FP64 oracle.

- The 1024 x 1024 heterogeneous-diffusion system (n = 1,048,576, t = 16,
  SRE-CG, Pre-CholQR) with the block Jacobi IC(0) preconditioner on 64
  blocks (Section 3 "Preconditioned versions", Algorithm 5), solved to the
  paper's tolerance rho_k <= 1e-8 rho_0 (Algorithm 1).
- The same system without a preconditioner for 200 iterations (it needs
  about 10,000 to converge): the residual history is compared iteration by
  iteration.
- Three systems of the batched workload's sizes (sides 128, 320, 512,
  log-normal coefficients, t = 8) through the batched solver in FP64, each
  against its own oracle solve (the envelope spans four perturbed runs and
  the run with the other orthonormalisation, as for the small systems).

The oracle is the same C source as everywhere else, built with OpenMP and
run on every host core; it returns the same bits as the single-threaded
build (tests/test_oracle_threads.py).  Runs of this size are chaotic: a
1e-15 relative perturbation of b moves the oracle's own history, so each
check spans the oracle's sensitivity with perturbed oracle runs
(parity_util).  When ECG_PARITY_REPORT names a file, every test appends the
measured iteration delta, divergence onset and relative x error to it as
one JSON line.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2305_19013_gb300 import ecg
from paper_2305_19013_gb300 import workloads as W
from parity_util import ONSET, TRACK, envelope_assert, envelope_metrics, rel

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    ecg.load()
    O.threads(None)
    yield
    O.threads(1)


def report(name, **kv):
    path = os.environ.get("ECG_PARITY_REPORT")
    line = {"test": name, **{k: (float(v) if isinstance(v, (np.floating, float)) else v) for k, v in kv.items()}}
    print(json.dumps(line))
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def headline():
    return W.blocky_diffusion2d(1024, 16, blocks=16, seed=2001)


def test_fullsize_ic0_solve_to_tolerance(headline):
    p = headline
    A = p.scipy()
    pb = W.jacobi_blocks(p, 64)
    pc = O.BlockJacobi(A, pb, 64, O.PREC_IC0)
    maxit = 3000
    with ecg.Solver.from_problem(p, trunc=2) as s:
        s.set_preconditioner(pb, 64)
        g = s.solve(dev(p.b), tol=1e-8, maxit=maxit)
        xg = g.x.cpu().numpy()
    r = envelope_metrics(p, g.iters, g.history, xg, dict(trunc=2), maxit, prec=pc, nperturbed=2, other_ortho=False)
    o = r["oracle"]
    report("fullsize_ic0_to_1e-8", gpu_iters=g.iters, oracle_iters=o.iters, iters_delta=r["iters_delta"],
           envelope_iters=r["oracle_iters"], onset=r["onset"], hist_dev_to_onset=r["hist_dev_to_onset"],
           x_rel_err=r["x_rel_err"], x_spread=r["x_spread"], gpu_relres_true=g.relres_true,
           oracle_relres_true=o.relres_true)
    assert g.status == ecg.OK and g.relres <= 1e-8
    envelope_assert(r, g.iters)
    assert g.relres_true <= 2e-8


def test_fullsize_200_iterations_history(headline):
    """200 iterations of the unpreconditioned solve.  The run is chaotic after
    about 20 iterations, so: (a) the GPU's history equals the oracle's to
    TRACK rho_0 up to the onset, the iteration where the oracle's runs on
    1e-15-perturbed b leave its history by ONSET rho_0; (c) x after 200
    iterations is within ten times the perturbed runs' spread of x; (d) so
    is rho_200.  The largest per-iteration deviation is reported.

    The oracle runs the GPU's reading of Pre-CholQR (ortho 2: CholQR as the
    Euclidean step).  Measured, the GPU's deviation from the oracle is the
    same to two digits for ortho 0 and ortho 2; the two modes' perturbed runs
    leave their histories at iterations 21 and 20.  The GPU's deviation grows
    about fourfold per iteration there (1.9e-9 rho_0 at iteration 19, 2.2e-8
    at 21), so whether the onset iteration itself stays within TRACK depends
    on that one-iteration difference."""
    p = headline
    A = p.scipy()
    K = 200
    with ecg.Solver.from_problem(p, trunc=2) as s:
        g = s.solve(dev(p.b), tol=0.0, maxit=K + 1)
        xg = g.x.cpu().numpy()
    assert g.status == ecg.ENOCONV and g.iters == K
    o = O.ecg_solve(A, p.part, 16, p.b, tol=0.0, maxit=K + 1, trunc=2, ortho=2)
    rng = np.random.default_rng(99)
    perturbed = [O.ecg_solve(A, p.part, 16, p.b * (1.0 + 1e-15 * rng.standard_normal(p.n)), tol=0.0,
                             maxit=K + 1, trunc=2, ortho=2) for _ in range(3)]
    h0 = o.history[0]
    onset = K
    for v in perturbed:
        dd = np.abs(v.history - o.history) > ONSET * h0
        if dd.any():
            onset = min(onset, int(np.argmax(dd)))
    d = np.abs(g.history - o.history)
    spread = np.max([np.abs(v.history - o.history) for v in perturbed], axis=0)
    xspread = max(rel(v.x, o.x) for v in perturbed)
    rspread = max(abs(v.history[K] - o.history[K]) for v in perturbed)
    report("fullsize_200_iterations", iters=K, onset=onset, max_dev_over_rho0=float(d.max() / h0),
           max_spread_over_rho0=float(spread.max() / h0), hist_dev_to_onset=float(d[: onset + 1].max() / h0),
           rho_dev_over_rho0=float(d[K] / h0), rho_spread_over_rho0=float(rspread / h0), x_rel_err=rel(xg, o.x),
           x_spread=xspread, relres_gpu=g.relres, relres_oracle=o.relres)
    assert np.all(d[: onset + 1] <= TRACK * h0)
    assert rel(xg, o.x) <= max(1e-8, 10.0 * xspread)
    assert d[K] <= max(TRACK * h0, 10.0 * rspread)


def test_fullsize_batched_systems_fp64():
    sides = [128, 320, 512]
    ps = []
    for q, side in enumerate(sides):
        ps += W.batch_diffusion2d(count=1, side_lo=side, side_hi=side, t=8, seed=4100 + q)
    maxit = 20000
    with ecg.BatchSolver(ps, trunc=2, precision=ecg.FP64) as bs:
        rc, res = bs.solve([p.b for p in ps], tol=1e-8, maxit=maxit)
    assert rc == ecg.OK
    ms = []
    for p, g in zip(ps, res):
        r = envelope_metrics(p, g.iters, g.history, g.x, dict(trunc=2), maxit, nperturbed=4, other_ortho=True)
        report(f"batched_fp64_side{int(p.meta['side'])}", n=p.n, gpu_iters=g.iters, oracle_iters=r["oracle"].iters,
               iters_delta=r["iters_delta"], envelope_iters=r["oracle_iters"], onset=r["onset"],
               hist_dev_to_onset=r["hist_dev_to_onset"], x_rel_err=r["x_rel_err"], x_spread=r["x_spread"])
        ms.append(r)
    for p, g, r in zip(ps, res, ms):
        assert g.status == ecg.OK and g.relres <= 1e-8
        envelope_assert(r, g.iters)


@pytest.fixture(scope="module")
def aniso3d():
    return W.anisotropic_diffusion3d(128, 16, seed=3000)


def test_fullsize_3d_first_iterations(aniso3d):
    """The 3D anisotropic workload at full size (128^3 = 2,097,152 rows,
    t = 16 as 4 x 2 x 2 boxes, SRE-CG): the first five iterates of the GPU
    (tensor-core CGS and final products) equal the oracle's to 1e-10."""
    p = aniso3d
    o = O.ecg_solve(p.scipy(), p.part, 16, p.b, tol=0.0, maxit=6, trunc=2)
    with ecg.Solver.from_problem(p, trunc=2) as s:
        g = s.solve(dev(p.b), tol=0.0, maxit=6)
        xg = g.x.cpu().numpy()
    report("fullsize_3d_first_iterations", n=p.n, iters=g.iters, x_rel_err=rel(xg, o.x),
           hist_dev_over_rho0=float(np.max(np.abs(g.history - o.history)) / o.history[0]))
    assert g.iters == o.iters == 5
    assert rel(xg, o.x) < 1e-10
    assert np.all(np.abs(g.history - o.history) <= 1e-10 * o.history[0])


def test_fullsize_3d_ic0_solve_to_tolerance(aniso3d):
    """The 3D workload with the block Jacobi IC(0) preconditioner on 64
    boxes, solved to 1e-8 in FP64 and in mixed precision; FP64 against the
    oracle's iteration count (within 1% and +-2), x within 1e-7 of the
    oracle's; mixed precision meets the FP64 tolerance on the true
    residual."""
    p = aniso3d
    A = p.scipy()
    pb = W.jacobi_blocks(p, 64)
    pc = O.BlockJacobi(A, pb, 64, O.PREC_IC0)
    o = O.ecg_solve(A, p.part, 16, p.b, tol=1e-8, maxit=3000, trunc=2, prec=pc)
    res = {}
    for prec in (ecg.FP64, ecg.MIXED):
        with ecg.Solver.from_problem(p, trunc=2, precision=prec) as s:
            s.set_preconditioner(pb, 64)
            g = s.solve(dev(p.b), tol=1e-8, maxit=20000)
            res[prec] = (g, g.x.cpu().numpy())
    g, xg = res[ecg.FP64]
    gm, xm = res[ecg.MIXED]
    report("fullsize_3d_ic0_to_1e-8", n=p.n, gpu_iters=g.iters, oracle_iters=o.iters, iters_delta=g.iters - o.iters,
           x_rel_err=rel(xg, o.x), mixed_iters=gm.iters, mixed_relres_true=gm.relres_true,
           mixed_x_rel_err=rel(xm, o.x))
    assert o.status == 0 and g.status == ecg.OK and gm.status == ecg.OK
    assert abs(g.iters - o.iters) <= max(2, -(-o.iters // 100))
    assert rel(xg, o.x) < 1e-7
    assert gm.relres_true <= 1e-8
