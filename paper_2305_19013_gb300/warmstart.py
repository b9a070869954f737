"""Learned warm start: a small U-Net that proposes the initial iterate x_0 of
an enlarged CG solve from (log coefficient, right-hand side) on a 2D grid.

The paper has no such component (its solves start from x_0 = 0); it sits
beside the method.  A solve started from the proposal uses the stopping
rule ||r_k|| <= tol ||b|| (ECG_STOP_B), so a good x_0 shortens it, and the
x_0 = 0 solve under the same rule is both the fallback and the measure of
the proposal.

This module only orchestrates: device memory comes from PyTorch tensors,
and every arithmetic step (convolutions, their gradients, pooling,
upsampling, the loss, Adam, input packing) runs in the kernels of
libecg.so (include/ecg_nn.h).  Activations are bf16 NHWC, weights bf16 with
FP32 master copies, gradients FP32.

Network (width 16: 118,129 parameters; width 20: 184,381): two 3x3 conv +
ReLU layers per level at side^2 (width channels), (side/2)^2 (2 width) and
(side/4)^2 (4 width), 2x2 average
pooling down, nearest upsampling up with skip connections concatenated,
and a 1x1 head.  Targets are the ECG solutions scaled by 1 / std(b) (the
problem is linear in b), so the proposal is x_0 = std(b) * net(...).  The
training loss is the relative energy-norm error e^T A e / x^T A x, the
quantity CG reduces: an MSE loss leaves high-frequency error that A
amplifies, and such proposals made the solves longer, not shorter.
"""
from __future__ import annotations

import ctypes as C
import time
from dataclasses import dataclass

import numpy as np

from . import ecg
from . import workloads as Wk

_P = C.c_void_p
_I = C.c_int
_I64 = C.c_int64
_F = C.c_float
_D = C.c_double

SIGNATURES = {
    "ecg_nn_conv": (_I, [_P, _I, _P, _I, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _P]),
    "ecg_nn_conv_dgrad": (_I, [_P, _P, _P, _I, _P, _I, _I, _I, _I, _I, _I, _I, _P]),
    "ecg_nn_wgrad_scratch": (C.c_size_t, [_I, _I, _I]),
    "ecg_nn_conv_wgrad": (_I, [_P, _I, _P, _I, _P, _P, _P, _P, _I, _I, _I, _I, _I, _P]),
    "ecg_nn_relu_bwd": (_I, [_P, _P, _I64, _P]),
    "ecg_nn_pool2": (_I, [_P, _P, _I, _I, _I, _I, _P]),
    "ecg_nn_pool2_bwd": (_I, [_P, _P, _I, _I, _I, _I, _P]),
    "ecg_nn_up2": (_I, [_P, _P, _I, _I, _I, _I, _P]),
    "ecg_nn_up2_bwd": (_I, [_P, _P, _I, _I, _I, _I, _P]),
    "ecg_nn_mse": (_I, [_P, _P, _P, _P, _I64, _P]),
    "ecg_nn_energy_loss": (_I, [_P, _P, _P, _P, _P, _P, _I, _I, _P]),
    "ecg_nn_adam": (_I, [_P, _P, _P, _P, _P, _I64, _F, _F, _F, _F, _I, _P]),
    "ecg_nn_to_bf16": (_I, [_P, _P, _I64, _P]),
    "ecg_nn_pack": (_I, [_P, _P, _D, _D, _D, _P, _I, _P]),
    "ecg_nn_unpack": (_I, [_P, _P, _D, _P, _I, _P]),
}

_nn = None


def lib():
    global _nn
    if _nn is None:
        L = ecg.load()
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _nn = L
    return _nn


def _p(t):
    return None if t is None else t.data_ptr()


def _ok(rc, what):
    if rc != 0:
        raise ecg.EcgError(rc, what)


def layers(width: int = 16):
    """(name, input A channels, input B channels (skip), output channels, K,
    relu) of the U-Net with `width`, 2 `width` and 4 `width` channels at its
    three levels (width 16: 118,129 parameters; 20: 184,381)."""
    w1, w2, w4 = width, 2 * width, 4 * width
    return [
        ("enc0a", 2, 0, w1, 3, 1),
        ("enc0b", w1, 0, w1, 3, 1),
        ("enc1a", w1, 0, w2, 3, 1),
        ("enc1b", w2, 0, w2, 3, 1),
        ("mid_a", w2, 0, w4, 3, 1),
        ("mid_b", w4, 0, w4, 3, 1),
        ("dec1a", w4, w2, w2, 3, 1),
        ("dec1b", w2, 0, w2, 3, 1),
        ("dec0a", w2, w1, w1, 3, 1),
        ("dec0b", w1, 0, w1, 3, 1),
        ("head", w1, 0, 1, 1, 0),
    ]


LAYERS = layers(16)


class WarmStartNet:
    def __init__(self, side: int = 256, batch: int = 8, seed: int = 0, device="cuda", width: int = 16):
        import torch

        if side % 4:
            raise ValueError("side must be a multiple of 4")
        self.side, self.batch, self.dev = side, batch, device
        self.w1, self.w2, self.w4 = width, 2 * width, 4 * width
        self.layers = layers(width)
        self.t = torch
        self.L = lib()
        g = torch.Generator().manual_seed(seed)
        self.params = {}
        for name, ca, cb, co, k, _ in self.layers:
            fan_in = k * k * (ca + cb)
            w = torch.randn(k, k, ca + cb, co, generator=g) * np.sqrt(2.0 / fan_in)
            if name == "head":
                w *= 0.1
            w32 = w.float().to(device).contiguous()
            b32 = torch.zeros(co, device=device)
            self.params[name] = {
                "w32": w32,
                "w16": w32.to(torch.bfloat16).contiguous(),
                "b": b32,
                "gw": torch.zeros_like(w32),
                "gb": torch.zeros_like(b32),
                "mw": torch.zeros_like(w32),
                "vw": torch.zeros_like(w32),
                "mb": torch.zeros_like(b32),
                "vb": torch.zeros_like(b32),
            }
        self.step_count = 0
        smax = max(self.L.ecg_nn_wgrad_scratch(ca + cb, co, k) for _, ca, cb, co, k, _ in self.layers)
        self.scratch = torch.empty(int(smax), dtype=torch.float32, device=device)
        self.loss_buf = torch.zeros(257, dtype=torch.float64, device=device)
        self._acts = None

    def n_params(self) -> int:
        return sum(p["w32"].numel() + p["b"].numel() for p in self.params.values())

    # ---------------------------------------------------------- forward
    def _alloc(self, N):
        t = self.t
        s = self.side
        bf = t.bfloat16

        def A(h, c, dt=bf):
            return t.empty(N, h, h, c, dtype=dt, device=self.dev)

        a = {
            "x": A(s, 2), "a0a": A(s, self.w1), "s0": A(s, self.w1), "p0": A(s // 2, self.w1), "a1a": A(s // 2, self.w2),
            "s1": A(s // 2, self.w2), "p1": A(s // 4, self.w2), "ma": A(s // 4, self.w4), "mb": A(s // 4, self.w4),
            "u1": A(s // 2, self.w4), "d1a": A(s // 2, self.w2), "d1b": A(s // 2, self.w2), "u0": A(s, self.w2), "d0a": A(s, self.w1),
            "d0b": A(s, self.w1), "out": A(s, 1, t.float32),
        }
        return a

    def _conv(self, name, inA, inB, out, N, H, out32=False):
        _, ca, cb, co, k, relu = next(l for l in self.layers if l[0] == name)
        p = self.params[name]
        _ok(self.L.ecg_nn_conv(_p(inA), ca, _p(inB), cb, _p(p["w16"]), _p(p["b"]), _p(out), 1 if out32 else 0, N, H,
                               H, co, k, relu, None), name)

    def forward(self, x):
        """x: N x side x side x 2 bf16 (packed inputs).  Returns the FP32
        N x side x side x 1 output; keeps the activations for backward."""
        N = x.shape[0]
        s = self.side
        if self._acts is None or self._acts["x"].shape[0] != N:
            self._acts = self._alloc(N)
        a = self._acts
        a["x"].copy_(x)
        L = self.L
        self._conv("enc0a", a["x"], None, a["a0a"], N, s)
        self._conv("enc0b", a["a0a"], None, a["s0"], N, s)
        _ok(L.ecg_nn_pool2(_p(a["s0"]), _p(a["p0"]), N, s, s, self.w1, None), "pool0")
        self._conv("enc1a", a["p0"], None, a["a1a"], N, s // 2)
        self._conv("enc1b", a["a1a"], None, a["s1"], N, s // 2)
        _ok(L.ecg_nn_pool2(_p(a["s1"]), _p(a["p1"]), N, s // 2, s // 2, self.w2, None), "pool1")
        self._conv("mid_a", a["p1"], None, a["ma"], N, s // 4)
        self._conv("mid_b", a["ma"], None, a["mb"], N, s // 4)
        _ok(L.ecg_nn_up2(_p(a["mb"]), _p(a["u1"]), N, s // 4, s // 4, self.w4, None), "up1")
        self._conv("dec1a", a["u1"], a["s1"], a["d1a"], N, s // 2)
        self._conv("dec1b", a["d1a"], None, a["d1b"], N, s // 2)
        _ok(L.ecg_nn_up2(_p(a["d1b"]), _p(a["u0"]), N, s // 2, s // 2, self.w2, None), "up0")
        self._conv("dec0a", a["u0"], a["s0"], a["d0a"], N, s)
        self._conv("dec0b", a["d0a"], None, a["d0b"], N, s)
        self._conv("head", a["d0b"], None, a["out"], N, s, out32=True)
        return a["out"]

    # --------------------------------------------------------- backward
    def _grads(self, name, inA, inB, dout, N, H, dA=None, dB=None, accumulate=0):
        """Weight/bias gradients of layer `name` and (when dA is given) its
        input gradients; dout already masked by the ReLU derivative."""
        _, ca, cb, co, k, _ = next(l for l in self.layers if l[0] == name)
        p = self.params[name]
        _ok(self.L.ecg_nn_conv_wgrad(_p(inA), ca, _p(inB), cb, _p(dout), _p(p["gw"]), _p(p["gb"]), _p(self.scratch),
                                     N, H, H, co, k, None), name + " wgrad")
        if dA is not None:
            _ok(self.L.ecg_nn_conv_dgrad(_p(dout), _p(p["w16"]), _p(dA), ca, _p(dB), cb, N, H, H, co, k, accumulate,
                                         None), name + " dgrad")

    def _relu_bwd(self, act, d):
        _ok(self.L.ecg_nn_relu_bwd(_p(act), _p(d), d.numel(), None), "relu_bwd")

    def backward(self, dout):
        """dout: FP32 gradient of the loss with respect to the output."""
        t = self.t
        a = self._acts
        N = dout.shape[0]
        s = self.side
        L = self.L

        def G(h, c):
            return t.empty(N, h, h, c, dtype=t.float32, device=self.dev)

        d_d0b = G(s, self.w1)
        self._grads("head", a["d0b"], None, dout, N, s, d_d0b)
        self._relu_bwd(a["d0b"], d_d0b)
        d_d0a = G(s, self.w1)
        self._grads("dec0b", a["d0a"], None, d_d0b, N, s, d_d0a)
        self._relu_bwd(a["d0a"], d_d0a)
        d_u0, d_s0 = G(s, self.w2), G(s, self.w1)
        self._grads("dec0a", a["u0"], a["s0"], d_d0a, N, s, d_u0, d_s0)
        d_d1b = G(s // 2, self.w2)
        _ok(L.ecg_nn_up2_bwd(_p(d_u0), _p(d_d1b), N, s // 2, s // 2, self.w2, None), "up0 bwd")
        self._relu_bwd(a["d1b"], d_d1b)
        d_d1a = G(s // 2, self.w2)
        self._grads("dec1b", a["d1a"], None, d_d1b, N, s // 2, d_d1a)
        self._relu_bwd(a["d1a"], d_d1a)
        d_u1, d_s1 = G(s // 2, self.w4), G(s // 2, self.w2)
        self._grads("dec1a", a["u1"], a["s1"], d_d1a, N, s // 2, d_u1, d_s1)
        d_mb = G(s // 4, self.w4)
        _ok(L.ecg_nn_up2_bwd(_p(d_u1), _p(d_mb), N, s // 4, s // 4, self.w4, None), "up1 bwd")
        self._relu_bwd(a["mb"], d_mb)
        d_ma = G(s // 4, self.w4)
        self._grads("mid_b", a["ma"], None, d_mb, N, s // 4, d_ma)
        self._relu_bwd(a["ma"], d_ma)
        d_p1 = G(s // 4, self.w2)
        self._grads("mid_a", a["p1"], None, d_ma, N, s // 4, d_p1)
        _ok(L.ecg_nn_pool2_bwd(_p(d_p1), _p(d_s1), N, s // 2, s // 2, self.w2, None), "pool1 bwd")
        self._relu_bwd(a["s1"], d_s1)
        d_a1a = G(s // 2, self.w2)
        self._grads("enc1b", a["a1a"], None, d_s1, N, s // 2, d_a1a)
        self._relu_bwd(a["a1a"], d_a1a)
        d_p0 = G(s // 2, self.w1)
        self._grads("enc1a", a["p0"], None, d_a1a, N, s // 2, d_p0)
        _ok(L.ecg_nn_pool2_bwd(_p(d_p0), _p(d_s0), N, s, s, self.w1, None), "pool0 bwd")
        self._relu_bwd(a["s0"], d_s0)
        d_a0a = G(s, self.w1)
        self._grads("enc0b", a["a0a"], None, d_s0, N, s, d_a0a)
        self._relu_bwd(a["a0a"], d_a0a)
        self._grads("enc0a", a["x"], None, d_a0a, N, s)

    def loss_and_grad(self, out, target, kappa=None, weights=None):
        """Loss (device scalar in loss_buf[0]) and its gradient: the energy
        norm of the error when the batch's coefficients (kappa, N x side x
        side FP32) and per-image weights are given, else the MSE."""
        dout = self.t.empty_like(out)
        if kappa is not None:
            _ok(self.L.ecg_nn_energy_loss(_p(out), _p(target), _p(kappa), _p(weights), _p(dout), _p(self.loss_buf),
                                          out.shape[0], self.side, None), "energy loss")
        else:
            _ok(self.L.ecg_nn_mse(_p(out), _p(target), _p(dout), _p(self.loss_buf), out.numel(), None), "mse")
        return dout

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        for p in self.params.values():
            _ok(self.L.ecg_nn_adam(_p(p["w32"]), _p(p["w16"]), _p(p["gw"]), _p(p["mw"]), _p(p["vw"]), p["w32"].numel(),
                                   lr, beta1, beta2, eps, self.step_count, None), "adam w")
            _ok(self.L.ecg_nn_adam(_p(p["b"]), None, _p(p["gb"]), _p(p["mb"]), _p(p["vb"]), p["b"].numel(), lr, beta1,
                                   beta2, eps, self.step_count, None), "adam b")


# ------------------------------------------------------------------ data


@dataclass
class Sample:
    problem: object  # workloads.Problem
    x_grid: np.ndarray | None  # ECG solution in grid order (None for held-out problems)
    scale: float  # std(b)


def pack_inputs(samples, device="cuda"):
    """N x side x side x 2 bf16 network inputs, packed by ecg_nn_pack."""
    import torch

    L = lib()
    side = samples[0].problem.meta["side"]
    out = torch.empty(len(samples), side, side, 2, dtype=torch.bfloat16, device=device)
    for i, s in enumerate(samples):
        logk = torch.from_numpy(np.ascontiguousarray(s.problem.meta["logk"].ravel())).to(device)
        bg = torch.from_numpy(np.ascontiguousarray(s.problem.meta["b_grid"])).to(device)
        _ok(L.ecg_nn_pack(_p(logk), _p(bg), 0.0, 1.0, float(s.scale), out[i].data_ptr(), side, None), "pack")
    return out


def make_dataset(count, side=256, t=16, seed0=100000, tol=1e-8, prec_blocks=64, solve=True):
    """count GRF diffusion problems with their ECG solutions (grid order)
    from GPU solves (FP64 SRE-CG with the block Jacobi IC(0) preconditioner,
    tol 1e-8)."""
    import torch

    out = []
    for i in range(count):
        p = Wk.grf_diffusion2d(side, t, seed=seed0 + i)
        scale = float(np.std(p.b))
        xg = None
        if solve:
            with ecg.Solver.from_problem(p, trunc=2) as sv:
                sv.set_preconditioner(Wk.jacobi_blocks(p, prec_blocks), prec_blocks)
                r = sv.solve(torch.from_numpy(p.b).cuda(), tol=tol, maxit=20000)
            x = r.x.cpu().numpy()
            xg = np.empty_like(x)
            xg[p.meta["perm"]] = x  # solver row r holds grid row perm[r]
        out.append(Sample(p, xg, scale))
    return out


def train(net, samples, epochs=10, lr=1e-3, seed=0, log=None):
    """Adam on the relative energy-norm error of the output against
    x_grid / scale, e^T A e / (x^T A x) per image (x^T A x = x^T b), with a
    cosine learning-rate decay.  Returns the per-epoch mean losses."""
    import torch

    X = pack_inputs(samples, net.dev)
    Y = torch.stack([torch.from_numpy((s.x_grid / s.scale).astype(np.float32)) for s in samples]).to(net.dev)
    Y = Y.reshape(len(samples), net.side, net.side, 1).contiguous()
    K = torch.stack([torch.from_numpy(np.exp(s.problem.meta["logk"]).astype(np.float32)) for s in samples]).to(net.dev)
    # x^T A x = x^T b in the scaled units (x / scale, b / scale)
    energy = np.array([float(s.x_grid @ s.problem.meta["b_grid"]) / s.scale**2 for s in samples])
    rng = np.random.default_rng(seed)
    hist = []
    B = net.batch
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        tot, nb = 0.0, 0
        lr_ep = lr * 0.5 * (1.0 + np.cos(np.pi * ep / max(epochs, 1)))
        for j in range(0, len(order) - B + 1, B):
            sel = order[j : j + B]
            idx = torch.from_numpy(sel).to(net.dev)
            w = torch.from_numpy((1.0 / (B * energy[sel])).astype(np.float32)).to(net.dev)
            out = net.forward(X[idx])
            dout = net.loss_and_grad(out, Y[idx], K[idx].contiguous(), w)
            net.backward(dout)
            net.adam(lr=float(lr_ep))
            tot += float(net.loss_buf[0].item())
            nb += 1
        hist.append(tot / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def propose(net, sample, device="cuda"):
    """x_0 in the solver's row order (FP64 device tensor)."""
    import torch

    X = pack_inputs([sample], device)
    out = net.forward(X)
    p = sample.problem
    perm = torch.from_numpy(p.meta["perm"].astype(np.int32)).to(device)
    x0 = torch.empty(p.n, dtype=torch.float64, device=device)
    _ok(lib().ecg_nn_unpack(out.data_ptr(), perm.data_ptr(), float(sample.scale), x0.data_ptr(), p.n, None), "unpack")
    return x0


def evaluate(net, samples, tol=1e-8, trunc=2, prec_blocks=0, maxit=60000, sweeps=4, omega=0.8, device="cuda"):
    """Solve every held-out problem from x_0 = 0 and from the smoothed
    proposal (the network's output after `sweeps` damped Jacobi sweeps,
    which remove the high-frequency error that A amplifies), both with the
    stopping rule ||r_k|| <= tol ||b||; the proposal falls back to x_0 = 0
    when its residual is not below ||b||.  Returns per-problem rows
    (iterations, seconds; the proposal's seconds include inference,
    smoothing and the fallback test)."""
    import torch

    rows = []
    for s in samples:
        p = s.problem
        b = torch.from_numpy(p.b).to(device)
        nb = float(torch.linalg.norm(b).item())
        with ecg.Solver.from_problem(p, trunc=trunc, stop_rule=ecg.STOP_B) as sv:
            if prec_blocks:
                sv.set_preconditioner(Wk.jacobi_blocks(p, prec_blocks), prec_blocks)
            sv.solve(b, tol=tol, maxit=maxit)  # warm the context
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r0 = sv.solve(b, tol=tol, maxit=maxit)
            torch.cuda.synchronize()
            t_zero = time.perf_counter() - t0
            t0 = time.perf_counter()
            x0 = propose(net, s, device)
            raw = x0.clone()
            sv.smooth(b, x0, sweeps, omega)
            r1 = sv.solve(b, x0=x0, tol=tol, maxit=maxit)
            used = float(r1.history[0]) < nb
            if not used:  # fallback: the proposal did not beat x_0 = 0
                r1 = sv.solve(b, tol=tol, maxit=maxit)
            torch.cuda.synchronize()
            t_net = time.perf_counter() - t0
            # the raw proposal's residual (0 iterations: history[0] = ||b - A x0||)
            raw_rho = float(sv.solve(b, x0=raw, tol=tol, maxit=1, raise_on_error=False).history[0])
            rows.append({
                "iters_zero": r0.iters, "iters_net": r1.iters, "s_zero": t_zero, "s_net": t_net,
                "status_zero": r0.status, "status_net": r1.status,
                "relres_true_zero": r0.relres_true, "relres_true_net": r1.relres_true,
                "x0_relres": float(r1.history[0]) / nb if used else 1.0,
                "raw_relres": raw_rho / nb,
                "used": used,
            })
    return rows
