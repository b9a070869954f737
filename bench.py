"""Benchmark of the GB300 enlarged CG path.

One "step" is one ECG iteration (every row of the hot path: block
generation, CGS2 against the window, Pre-CholQR A-orthonormalisation with
the SpMM, the t x t Cholesky factorisations, and the x/r updates) on the
1024 x 1024 heterogeneous-diffusion system with t = 16 (n = 1,048,576),
SRE-CG (SRE-CG2 truncated to a window of 2 blocks) in FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank solves its own
replica of the system (weak scaling); the time is the maximum over ranks.

value    iterations per second of the whole job with a full window, inputs
         resident in HBM: CUDA events on the solver's stream around one
         ecg_solve call of trunc + K iterations and one of trunc iterations;
         the K steps take the difference (the first trunc iterations, whose
         window is still filling, are not counted).
e2e      the same metric through the C ABI with host buffers (b copied in,
         x and the residual history copied out inside the timed call of K
         iterations, window start-up included).
roofline the kernel class with the largest share of the iteration, from a
         second, profiled run (CUDA events on the solver's stream around
         every kernel class).
time_to_tol  wall time to the paper's tolerance rho_k <= 1e-8 rho_0
         (Algorithm 1) for plain FP64 SRE-CG, for FP64 with the block Jacobi
         IC(0) preconditioner (64 blocks; Section 3, Algorithm 5) and for the
         mixed-precision method with the same preconditioner.
--impl reference times the FP64 CPU oracle (the reference implementation of
this build) at the full size on every host core; so does cpu_baseline, on a
bounded number of iterations.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ECG time-to-1e-8 residual & iterations/sec (n≈1M, t=16), HBM GB/s vs peak"
UNIT = "iterations/s"
WORKLOAD = "diffusion2d_1024_t16"
# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per full-window launch of a kernel class, averaged
# over the two CGS passes of one iteration (the first pass of an SRE
# iteration reads V_{k-1} as both a window block and the block), from one ncu
# capture of the kernels as they stand; n = 1,048,576, t = 16, window of 2
# blocks.  Any other shape reports null.
MEASURED_TRAFFIC = {
    # CUDA-core kernels (--no-tensor-cores)
    ("cgs_tdot", 16, 2, "alu"): ((268.72e6 + 3.75e6) + (402.95e6 + 4.84e6)) / 2,
    ("cgs_update", 16, 2, "alu"): ((403.09e6 + 115.24e6) + (403.00e6 + 108.42e6)) / 2,
    # tensor-core kernels (profiles/cgs_final_tc_kernels_diffusion2d_1024_t16.md)
    ("cgs_tdot", 16, 2, "hbm"): ((268.50e6 + 4.38e6) + (402.86e6 + 4.42e6)) / 2,
    ("cgs_update", 16, 2, "hbm"): ((407.02e6 + 113.51e6) + (402.75e6 + 99.93e6)) / 2,
    ("final", 16, 2, "alu"): 287.18e6 + 236.88e6,
}


# Roofline denominators when the driver's measured peaks are absent: the
# profiling recipe's fallback figures for a GB300 (HBM copy, dense bf16).
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def peaks():
    """The measured peaks (MEASURED_PEAKS.json), else the fallback; the
    returned dict says which in "source"."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = dict(json.load(f))
        d["source"] = "measured (MEASURED_PEAKS.json)"
        return d
    except Exception:
        d = dict(FALLBACK_PEAKS)
        d["source"] = "fallback (no MEASURED_PEAKS.json on this box)"
        return d


class ClockSampler:
    """nvidia-smi samples (every 100 ms) of SM clock and throttle reasons,
    stamped with host time, so that the samples of a region can be picked
    out afterwards (summary(t0, t1))."""

    FIELDS = (
        "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, index=0, period_ms=100):
        self.index = index
        self.period_ms = period_ms
        self.rows = []  # (host time, fields)
        self._proc = None
        self._thr = None

    def _read(self):
        for line in self._proc.stdout:
            line = line.strip()
            if line:
                self.rows.append((time.perf_counter(), [c.strip() for c in line.split(",")]))

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms={self.period_ms}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
            self._thr = threading.Thread(target=self._read, daemon=True)
            self._thr.start()
            time.sleep(0.5)  # first samples before the region starts
        except Exception:
            self._proc = None
        return self

    def __exit__(self, *a):
        if self._proc is not None:
            time.sleep(0.3)
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._thr:
            self._thr.join(timeout=5)

    def summary(self, t0=None, t1=None, pad=0.25):
        """Samples taken in [t0 - pad, t1 + pad] (all samples when t0 is
        None); at least the two nearest samples."""
        rows = self.rows
        if t0 is not None and rows:
            sel = [r for r in rows if t0 - pad <= r[0] <= t1 + pad]
            if len(sel) < 2:
                mid = 0.5 * (t0 + t1)
                sel = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
            rows = sel
        rows = [r for _, r in rows]
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 4 + i and r[4 + i] == "Active"})
        return {
            "sm_mhz": float(np.median(sm)) if sm else None,
            "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons,
            "samples": len(rows),
            "window": f"samples within {pad} s of the timed region, every {self.period_ms} ms",
        }


def algorithmic_counts(n, nnz, t, trunc, K, sre=True):
    """FP64 flops and algorithmic DRAM bytes per kernel class, summed over
    iterations 1..K (the window holds m = min(k-1, trunc) blocks at
    iteration k).  Flops count every multiply-add the method's definition
    needs (2 flops); symmetric Grams count their upper triangle.  Bytes count
    each distinct n x t block a class must read or write once per launch
    (B = 8 n t bytes):
      cgs_tdot    pass 1 of an SRE iteration reads the m window blocks V_j
                  (the block itself is V_{k-1}, one of them); pass 2 reads
                  the m blocks and X: (2m + 1) B per iteration
      cgs_update  each pass reads the m blocks Q_j and its source, writes X:
                  2 (m + 2) B
      gram_e      X^T X reads X; q = X R_e^{-1} in place reads and writes
                  it: 3 B
      spmm_gram   Y = A q with q^T Y and q^T r: reads q and A (12 nnz +
                  4 (n + 1)) and r, writes Y: 2 B + 12 nnz + 4 (n + 1) + 8 n
      final       reads X, Y, x, r, writes W_k, V_k, x, r: 4 B + 32 n
    (the FP64 Pre-CholQR form, which materialises q before the SpMM)."""
    tri = t * (t + 1) // 2
    fl = {"cgs_tdot": 0.0, "cgs_update": 0.0, "gram_e": 0.0, "spmm_gram": 0.0, "final": 0.0}
    by = {k: 0.0 for k in fl}
    B = 8.0 * n * t
    for k in range(1, K + 1):
        m = min(k - 1, trunc)
        fl["cgs_tdot"] += 2 * 2.0 * (m * t) * t * n
        fl["cgs_update"] += 2 * 2.0 * (m * t) * t * n
        fl["gram_e"] += 2.0 * 2 * tri * n
        fl["spmm_gram"] += 2.0 * (nnz * t + tri * n + t * n)
        fl["final"] += 2.0 * (2 * tri * n + 2 * t * n)
        if m > 0:
            by["cgs_tdot"] += ((2 * m + 1) if sre else (2 * m + 2)) * B
            by["cgs_update"] += 2 * (m + 2) * B
        by["gram_e"] += 3 * B
        by["spmm_gram"] += 2 * B + 12.0 * nnz + 4.0 * (n + 1) + 8.0 * n
        by["final"] += 4 * B + 32.0 * n
    return fl, by


# Algorithmic DRAM bytes of one row-iteration of the batched kernel (FP32,
# t = 8, window of 2, Pre-CholQR): P1 96, P2 192, P3 128, P4 64, P5 112,
# P6 144 (each n x 8 FP32 row is 32 B; P5 counts the SELL entries and each
# gathered row once).
BATCH_BYTES_PER_ROW_ITER = 736


def batch_run(torch):
    """The batched workload: 64 independent 2D diffusion systems, sides
    uniform in {128, ..., 512}, log-normal coefficients, t = 8, FP32 inner
    solves with FP64 refinement to 1e-8, one persistent launch per round.
    Timed after one untimed solve, device resident right-hand sides."""
    from paper_2305_19013_gb300 import ecg
    from paper_2305_19013_gb300 import workloads as Wk

    ps = Wk.batch_diffusion2d(64)
    t0 = time.perf_counter()
    bs = ecg.BatchSolver(ps, precision=ecg.MIXED)
    t_create = time.perf_counter() - t0
    bd = [torch.from_numpy(p.b).cuda() for p in ps]
    bs.solve(bd, tol=1e-8, maxit=30000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, res = bs.solve(bd, tol=1e-8, maxit=30000)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    row_iters = sum(p.n * g.iters for p, g in zip(ps, res))
    achieved = BATCH_BYTES_PER_ROW_ITER * row_iters / dt / 1e9
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    out = {
        "workload": "64 x 2D diffusion, sides 128..512, t=8, FP32 inner + FP64 refinement, tol 1e-8",
        "status": rc,
        "seconds": dt,
        "systems_per_s": len(ps) / dt,
        "rows": sum(p.n for p in ps),
        "iters_min": min(g.iters for g in res),
        "iters_max": max(g.iters for g in res),
        "max_relres_true": max(g.relres_true for g in res),
        "layout": bs.layout(),
        "create_seconds": t_create,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if hbm else None,
                     "algorithmic_bytes_per_row_iteration": BATCH_BYTES_PER_ROW_ITER,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs" if hbm else None},
    }
    bs.close()
    return out



def warmstart_run(torch, side=64, ntrain=256, nheld=8, epochs=30, width=16, batch=8, lr=3e-3):
    """The learned warm start at a reduced scale: GRF diffusion problems
    (side x side, correlation length 0.1, sigma 1, t = 16), ntrain training
    solves, the U-Net trained with the energy-norm loss, and held-out solves
    from x_0 = 0 against the smoothed proposal (16 Jacobi sweeps, fallback
    to x_0 = 0), stopping rule ||r|| <= 1e-8 ||b||, SRE-CG (trunc 2)."""
    from paper_2305_19013_gb300 import warmstart as WS

    t0 = time.perf_counter()
    train = WS.make_dataset(ntrain, side=side, t=16, seed0=7000, prec_blocks=16 if side <= 64 else 64)
    t1 = time.perf_counter()
    held = WS.make_dataset(nheld, side=side, t=16, seed0=9000, solve=False)
    net = WS.WarmStartNet(side=side, batch=batch, seed=2, width=width)
    hist = WS.train(net, train, epochs=epochs, lr=lr)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rows = WS.evaluate(net, held, tol=1e-8, trunc=2, sweeps=16)
    it0 = np.array([r["iters_zero"] for r in rows], dtype=float)
    it1 = np.array([r["iters_net"] for r in rows], dtype=float)
    return {
        "saving_iters_median": float(np.median(1.0 - it1 / it0)),
        "raw_relres_mean": float(np.mean([r["raw_relres"] for r in rows])),
        "workload": f"GRF diffusion {side}x{side}, t=16, {ntrain} training solves, {nheld} held-out problems",
        "params": net.n_params(),
        "data_seconds": t1 - t0,
        "train_seconds": t2 - t1,
        "energy_loss_first_last": [hist[0], hist[-1]],
        "iters_zero_mean": float(np.mean([r["iters_zero"] for r in rows])),
        "iters_warm_mean": float(np.mean([r["iters_net"] for r in rows])),
        "seconds_zero_mean": float(np.mean([r["s_zero"] for r in rows])),
        "seconds_warm_mean": float(np.mean([r["s_net"] for r in rows])),
        "x0_relres_mean": float(np.mean([r["x0_relres"] for r in rows])),
        "proposals_used": int(sum(r["used"] for r in rows)),
    }



def headline_problem(seed=2001):
    from paper_2305_19013_gb300 import workloads as Wk

    return Wk.blocky_diffusion2d(1024, 16, blocks=16, seed=seed)


def oracle_rate(p, K, W, trunc):
    """The FP64 CPU oracle at the full size on every host core (its OpenMP
    build; the same bits as the single-threaded one): after W untimed
    iterations, a solve of trunc iterations and one of trunc + K iterations
    are timed; the K steps take the difference, like the GPU's value."""
    import oracle as O

    A = p.scipy()
    cores = O.threads(None)
    try:
        if W > 0:
            O.ecg_solve(A, p.part, p.t, p.b, tol=0.0, maxit=W + 1, trunc=trunc)
        t0 = time.perf_counter()
        O.ecg_solve(A, p.part, p.t, p.b, tol=0.0, maxit=trunc + 1, trunc=trunc)
        t1 = time.perf_counter()
        r = O.ecg_solve(A, p.part, p.t, p.b, tol=0.0, maxit=trunc + K + 1, trunc=trunc)
        t2 = time.perf_counter()
    finally:
        O.threads(1)
    assert r.iters == trunc + K
    dt = (t2 - t1) - (t1 - t0)
    return {
        "value": K / dt,
        "unit": UNIT,
        "cores": cores,
        "kind": "oracle",
        "sample": f"{K} full-window iterations of SRE-CG (trunc={trunc}, Pre-CholQR) on the full {p.n}-row system "
        f"after {W} warm-up iterations: the oracle's OpenMP build on {cores} host threads, timed as a "
        f"{trunc + K}-iteration solve minus a {trunc}-iteration solve ({dt:.1f} s)",
        "seconds": dt,
    }


def reference_arm(args, rank):
    if rank != 0:
        return
    p = headline_problem()
    cb = oracle_rate(p, args.steps, args.warmup, args.trunc)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": cb["value"],
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 / cb["value"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": p.n, "nnz": p.nnz, "t": 16,
                   "method": f"SRE-CG2 truncated to {args.trunc} blocks (SRE-CG)", "ortho": "Pre-CholQR",
                   "parallelism": "single"},
        "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_to_tol_runs(torch, p, stream, args, names):
    """Solves to the paper's tolerance (rho_k <= 1e-8 rho_0, Algorithm 1),
    device-resident b, wall time of the solve call (the preconditioner's
    setup is timed separately)."""
    from paper_2305_19013_gb300 import ecg
    from paper_2305_19013_gb300 import workloads as Wk

    out = {}
    pb = None
    specs = {"fp64": (ecg.FP64, False), "mixed": (ecg.MIXED, False),
             f"fp64_ic0_{args.prec_blocks}": (ecg.FP64, True), f"mixed_ic0_{args.prec_blocks}": (ecg.MIXED, True)}
    b_dev = torch.from_numpy(p.b).cuda()
    x_dev = torch.empty_like(b_dev)
    for name in names:
        prec, pre = specs[name]
        if pre and pb is None:
            pb = Wk.jacobi_blocks(p, args.prec_blocks)
        with ecg.Solver.from_problem(p, trunc=args.trunc, ortho=args.ortho, precision=prec,
                                     tensor_cores=args.tensor_cores, stream=stream.cuda_stream) as sv:
            ts = time.perf_counter()
            if pre:  # block Jacobi IC(0) (Section 3, Algorithm 5)
                sv.set_preconditioner(pb, args.prec_blocks)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - ts
            t0 = time.perf_counter()
            r = sv.solve(b_dev, tol=1e-8, maxit=args.time_to_tol_maxit, x_out=x_dev, raise_on_error=False)
            torch.cuda.synchronize()
            out[name] = {"seconds": time.perf_counter() - t0, "iters": r.iters, "status": r.status,
                         "relres_true": r.relres_true, "device_ms": r.device_ms}
            if pre:
                out[name]["setup_seconds"] = t_setup
    return out


def other_configs_run(torch, stream, args, K=20):
    """The other workloads of the measurement plan, each at its full size:
    the 1024 x 1024 diffusion system with t = 8 and t = 32, and the 3D
    anisotropic 128^3 system with t = 16 (SRE-CG, trunc 2, Pre-CholQR).
    Per workload: FP64 iterations/s over K full-window iterations (as the
    headline value), and time to 1e-8 with the block Jacobi IC(0)
    preconditioner on 64 blocks, FP64 and mixed precision."""
    from paper_2305_19013_gb300 import ecg
    from paper_2305_19013_gb300 import workloads as Wk

    cases = [
        ("diffusion2d_1024_t8", lambda: Wk.blocky_diffusion2d(1024, 8, blocks=16, seed=2001)),
        ("diffusion2d_1024_t32", lambda: Wk.blocky_diffusion2d(1024, 32, blocks=16, seed=2001)),
        ("aniso3d_128_t16", lambda: Wk.anisotropic_diffusion3d(128, 16, seed=3000)),
    ]
    out = {}
    for name, make in cases:
        p = make()
        b_dev = torch.from_numpy(p.b).cuda()
        x_dev = torch.empty_like(b_dev)
        entry = {"n": p.n, "nnz": p.nnz, "t": p.t}
        with ecg.Solver.from_problem(p, trunc=args.trunc, ortho=args.ortho, tensor_cores=args.tensor_cores,
                                     stream=stream.cuda_stream) as sv:
            sv.solve(b_dev, tol=0.0, maxit=4, x_out=x_dev)
            ms, _, _, _ = full_window_ms(sv, b_dev, x_dev, K, args.trunc, stream, lambda: None, torch)
            entry["fp64_iterations_per_s"] = K / (ms / 1000.0)
            entry["fp64_ms_per_iteration"] = ms / K
        pb = Wk.jacobi_blocks(p, args.prec_blocks)
        for label, prec in (("fp64", ecg.FP64), ("mixed", ecg.MIXED)):
            with ecg.Solver.from_problem(p, trunc=args.trunc, ortho=args.ortho, precision=prec,
                                         tensor_cores=args.tensor_cores, stream=stream.cuda_stream) as sv:
                sv.set_preconditioner(pb, args.prec_blocks)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = sv.solve(b_dev, tol=1e-8, maxit=args.time_to_tol_maxit, x_out=x_dev, raise_on_error=False)
                torch.cuda.synchronize()
                entry[f"time_to_tol_{label}_ic0_{args.prec_blocks}"] = {
                    "seconds": time.perf_counter() - t0, "iters": r.iters, "status": r.status,
                    "relres_true": r.relres_true}
        out[name] = entry
    return out


def mixed_profile(torch, p, stream, args, K=40):
    """Per-class device time of the mixed method's FP32 inner iterations on
    the headline system (K inner iterations, tol = 0, CUDA events around each
    kernel class), with the FP32 CGS coefficient Grams on the tensor cores
    (tensor_cores = 2) and on CUDA cores (the default, 1)."""
    from paper_2305_19013_gb300 import ecg

    b_dev = torch.from_numpy(p.b).cuda()
    out = {}
    for tcores in (2, 1):
        with ecg.Solver.from_problem(p, trunc=args.trunc, ortho=args.ortho, precision=ecg.MIXED,
                                     tensor_cores=tcores, stream=stream.cuda_stream) as sv:
            sv.solve(b_dev, tol=0.0, maxit=6)
            sv.profile(True)
            r = sv.solve(b_dev, tol=0.0, maxit=K + 1)
            prof = sv.profile_read()
            sv.profile(False)
        tot = sum(v[0] for v in prof.values())
        out["tensor_core_grams" if tcores == 2 else "cuda_core_grams"] = {
            "inner_iterations": r.iters, "ms_per_inner_iteration": tot / max(r.iters, 1),
            "profile_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]}}
    return out


def full_window_ms(solver, b_dev, x_dev, K, trunc, stream, barrier, torch):
    """CUDA-event time of K full-window iterations: a solve of trunc + K
    iterations minus a solve of trunc iterations, each bracketed by a barrier
    and a device synchronisation."""
    def one(iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        res = solver.solve(b_dev, tol=0.0, maxit=iters + 1, x_out=x_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        assert res.iters == iters, (res.iters, iters)
        return e0.elapsed_time(e1)

    short = one(trunc)
    t0 = time.perf_counter()
    long_ = one(trunc + K)
    t1 = time.perf_counter()
    return long_ - short, long_, short, (t0, t1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--trunc", type=int, default=2)
    ap.add_argument("--ortho", type=int, default=0)
    ap.add_argument("--no-tensor-cores", dest="tensor_cores", action="store_false",
                    help="run the FP64 CGS products on CUDA-core FMAs instead of the tensor cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-tol", action="store_true", help="skip the solves to 1e-8")
    ap.add_argument("--time-to-tol-maxit", type=int, default=60000)
    ap.add_argument("--time-to-tol-all", action="store_true",
                    help="also run mixed precision without a preconditioner (it stalls on this problem)")
    ap.add_argument("--prec-blocks", type=int, default=64, help="block Jacobi blocks for the preconditioned runs")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (t = 8, t = 32, the 3D anisotropic system)")
    ap.add_argument("--warmstart", action="store_true",
                    help="also train the warm-start network on GRF diffusion problems and compare solves")
    ap.add_argument("--ws-side", type=int, default=64, help="warm start: grid side")
    ap.add_argument("--ws-train", type=int, default=256, help="warm start: training solves")
    ap.add_argument("--ws-held", type=int, default=8, help="warm start: held-out problems")
    ap.add_argument("--ws-epochs", type=int, default=30, help="warm start: epochs")
    ap.add_argument("--ws-width", type=int, default=16, help="warm start: U-Net width (16: 118K, 20: 184K parameters)")
    ap.add_argument("--batch", action="store_true",
                    help="also solve the batched workload (64 uneven 2D diffusion systems, t=8) and report it")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch

    from paper_2305_19013_gb300 import ecg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    K, Wm = args.steps, args.warmup
    assert Wm >= 3, "at least 3 warm-up steps"
    p = headline_problem(seed=2001 + rank)
    stream = torch.cuda.current_stream()
    solver = ecg.Solver.from_problem(p, trunc=args.trunc, ortho=args.ortho, tensor_cores=args.tensor_cores,
                                     stream=stream.cuda_stream)
    b_dev = torch.from_numpy(p.b).cuda()
    x_dev = torch.empty_like(b_dev)

    # warm-up: W iterations
    solver.solve(b_dev, tol=0.0, maxit=Wm + 1, x_out=x_dev)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- timed region: K full-window iterations, inputs resident in HBM
    with ClockSampler(local) as clk:
        ms, ms_long, ms_short, (tw0, tw1) = full_window_ms(solver, b_dev, x_dev, K, args.trunc, stream, barrier,
                                                           torch)
    assert ms > 0.0, (ms_long, ms_short)
    # kernels of one iteration: generate, 2 x (coefficients, reduce, update),
    # [Euclidean Gram, reduce, factor] for Pre-CholQR, A-Gram, reduce, factor,
    # final update, finish
    launches_per_iter = 15 if args.ortho == 0 else 12
    t_all = torch.tensor([ms], device="cuda")
    if dist is not None:
        dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
    ms_max = float(t_all.item())
    value = world * K / (ms_max / 1000.0)

    # ---- end to end through the C ABI with host buffers (K iterations)
    b_host = p.b.copy()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    solver.solve(b_host, tol=0.0, maxit=K + 1)
    t_e2e = time.perf_counter() - t0
    t_e = torch.tensor([t_e2e], device="cuda")
    if dist is not None:
        dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
    e2e_value = world * K / float(t_e.item())

    # ---- per-kernel-class profile (same trunc + K iterations, events on the stream)
    solver.profile(True)
    solver.solve(b_dev, tol=0.0, maxit=args.trunc + K + 1, x_out=x_dev)
    prof = solver.profile_read()
    solver.profile(False)
    fl, by = algorithmic_counts(p.n, p.nnz, 16, args.trunc, args.trunc + K)
    bytes_total = sum(by.values())
    tot_ms = sum(v[0] for v in prof.values())
    pk = peaks()
    hbm = pk["hbm_gbs"]
    # the CGS classes run on the tensor cores (t = 16, window <= 32 columns),
    # bound by HBM; the other block classes are FP64 FMA-bound
    tc_classes = {"cgs_tdot", "cgs_update"} if (args.tensor_cores and args.trunc * 16 <= 32) else set()
    classes = {}
    for k in fl:
        if k not in prof or not prof[k][1]:
            continue
        ms_k, n_k = prof[k]
        if k in tc_classes:
            ach = by[k] / (ms_k / 1000.0) / 1e9
            classes[k] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                          "ms": ms_k, "launches": n_k, "algorithmic_bytes": by[k]}
        else:
            ach = fl[k] / (ms_k / 1000.0) / 1e12
            classes[k] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": ach / FP64_PEAK_TFLOPS, "ms": ms_k, "launches": n_k,
                          "hbm_gbs": by[k] / (ms_k / 1000.0) / 1e9}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    dc = classes[dom]
    probe = None
    if world == 1:
        try:
            probe = ecg.probe_fp64()
        except Exception:
            probe = None
    roofline = {
        "bound": dc["bound"],
        "kernel": dom,
        "achieved": dc["achieved"],
        "peak": dc["peak"],
        "unit": dc["unit"],
        "frac": dc["frac"],
        "traffic": MEASURED_TRAFFIC.get((dom, 16, args.trunc, dc["bound"])),
        "traffic_note": "DRAM bytes (read + write) per launch of this class from one ncu capture of the current "
        "kernels (null when none was taken since they changed)",
        "peak_source": (pk["source"] + " HBM copy bandwidth") if dc["bound"] == "hbm" else
        "derived FP64 FMA issue rate: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
        "fp64_probe_tflops": probe,
        "probe_note": "FP64 FMA rate measured in this run by ecg_probe_fp64 (8 independent chains per thread, "
        "8 CTAs x 256 threads per SM)",
        "launches": dc["launches"],
        "share": dc["ms"] / tot_ms,
        "algorithmic": "bytes or flops per class as bench.algorithmic_counts states them, over the profiled "
        "trunc + K iterations",
    }
    prof_ms_total = tot_ms
    total_fl = sum(fl.values())
    iter_tflops = total_fl / (prof_ms_total / 1000.0) / 1e12
    hbm_gbs = bytes_total / (prof_ms_total / 1000.0) / 1e9

    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": ms_max / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "n": p.n,
            "nnz": p.nnz,
            "t": 16,
            "method": f"SRE-CG2 truncated to {args.trunc} blocks (SRE-CG)",
            "ortho": "Pre-CholQR" if args.ortho == 0 else "A-CholQR",
            "parallelism": "replicas" if world > 1 else "single",
            "timing": f"full window: CUDA events, ({args.trunc}+K)-iteration solve minus {args.trunc}-iteration solve",
            "l2": "no flush: the iteration streams ~3 GB of blocks, far above the 129 MB L2",
        },
        "gpu_launches": K * launches_per_iter,
        "e2e": {
            "value": e2e_value,
            "unit": UNIT,
            "h2d_bytes_per_step": 8 * p.n / K,
            "d2h_bytes_per_step": (8 * p.n + 8 * (K + 1)) / K,
        },
        "roofline": roofline,
        "iteration": {
            "fp64_tflops": iter_tflops,
            "fp64_frac": iter_tflops / FP64_PEAK_TFLOPS,
            "hbm_gbs": hbm_gbs,
            "hbm_frac": hbm_gbs / hbm,
            "hbm_peak": hbm,
            "hbm_peak_source": pk["source"],
            "profile_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
            "classes": classes,
            "note": "profiled run of trunc + K iterations (window start-up included); algorithmic bytes and flops "
            "counted for the same iterations",
        },
        "clocks": clk.summary(tw0, tw1),
    }
    solver.close()
    if world == 1 and not args.no_time_to_tol:
        names = ["fp64", f"fp64_ic0_{args.prec_blocks}", f"mixed_ic0_{args.prec_blocks}"]
        if args.time_to_tol_all:
            names.insert(1, "mixed")
        line["time_to_tol"] = time_to_tol_runs(torch, p, stream, args, names)
    if world == 1 and not args.no_configs:
        line["mixed_inner_profile"] = mixed_profile(torch, p, stream, args)
        line["other_configs"] = other_configs_run(torch, stream, args)
    if args.batch:
        line["batch"] = batch_run(torch)
    if args.warmstart:
        line["warmstart"] = warmstart_run(torch, side=args.ws_side, ntrain=args.ws_train, nheld=args.ws_held,
                                          epochs=args.ws_epochs, width=args.ws_width)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_rate(p, 8, 0, args.trunc)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
