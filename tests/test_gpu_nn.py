"""Kernels of the warm-start network (include/ecg_nn.h) against plain
PyTorch FP32 references on the CPU, with the bf16 rounding of activations and
weights applied to the reference's inputs; the training loop and the warm
start itself are checked end to end on small problems."""
import numpy as np
import pytest

from paper_2305_19013_gb300 import ecg
from paper_2305_19013_gb300 import warmstart as WS
from paper_2305_19013_gb300 import workloads as W

torch = pytest.importorskip("torch")
F = torch.nn.functional

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    WS.lib()


def _bf(x):
    return x.to(torch.bfloat16)


def _ref_conv(a, b, w, bias, K):
    """NHWC inputs, [K][K][Cin][Cout] weights -> NHWC output (FP32 CPU)."""
    x = a.float() if b is None else torch.cat([a.float(), b.float()], dim=3)
    wt = w.float().permute(3, 2, 0, 1)  # Cout, Cin, K, K
    y = F.conv2d(x.permute(0, 3, 1, 2), wt, bias, padding=K // 2)
    return y.permute(0, 2, 3, 1)


@pytest.mark.parametrize("K,Ca,Cb,Cout,H", [(3, 5, 3, 20, 20), (3, 2, 0, 16, 32), (1, 16, 0, 1, 24), (3, 64, 32, 32, 16)])
@pytest.mark.parametrize("out32", [0, 1])
def test_conv_forward(K, Ca, Cb, Cout, H, out32):
    g = torch.Generator().manual_seed(K * 100 + Ca)
    N = 2
    a = _bf(torch.randn(N, H, H, Ca, generator=g))
    b = _bf(torch.randn(N, H, H, Cb, generator=g)) if Cb else None
    w = _bf(torch.randn(K, K, Ca + Cb, Cout, generator=g) / np.sqrt(K * K * (Ca + Cb)))
    bias = torch.randn(Cout, generator=g)
    ref = F.relu(_ref_conv(a, b, w, bias, K))
    ad, wd, biasd = a.cuda(), w.cuda(), bias.cuda()
    bd = b.cuda() if b is not None else None
    out = torch.empty(N, H, H, Cout, dtype=torch.float32 if out32 else torch.bfloat16, device="cuda")
    rc = WS.lib().ecg_nn_conv(ad.data_ptr(), Ca, None if bd is None else bd.data_ptr(), Cb, wd.data_ptr(),
                              biasd.data_ptr(), out.data_ptr(), out32, N, H, H, Cout, K, 1, None)
    assert rc == 0
    got = out.float().cpu()
    tol = (1e-5 if out32 else 8e-3) * ref.abs().max().item()
    assert (got - ref).abs().max().item() <= tol


@pytest.mark.parametrize("K,Ca,Cb,Cout,H", [(3, 5, 3, 20, 20), (1, 16, 0, 1, 24), (3, 32, 16, 16, 32)])
def test_conv_gradients(K, Ca, Cb, Cout, H):
    g = torch.Generator().manual_seed(7 * K + Cout)
    N = 2
    a = _bf(torch.randn(N, H, H, Ca, generator=g))
    b = _bf(torch.randn(N, H, H, Cb, generator=g)) if Cb else None
    w = _bf(torch.randn(K, K, Ca + Cb, Cout, generator=g) / np.sqrt(K * K * (Ca + Cb)))
    dout = torch.randn(N, H, H, Cout, generator=g)
    # reference gradients by autograd
    af = a.float().requires_grad_()
    bf_ = b.float().requires_grad_() if b is not None else None
    wf = w.float().requires_grad_()
    bias = torch.zeros(Cout, requires_grad=True)
    y = _ref_conv(af, bf_, wf, bias, K)
    (y * dout).sum().backward()
    L = WS.lib()
    ad, wd, dd = a.cuda(), w.cuda(), dout.cuda()
    bd = b.cuda() if b is not None else None
    dA = torch.full((N, H, H, Ca), 0.5, device="cuda")
    dB = torch.full((N, H, H, Cb), 0.5, device="cuda") if Cb else None
    assert L.ecg_nn_conv_dgrad(dd.data_ptr(), wd.data_ptr(), dA.data_ptr(), Ca, None if dB is None else dB.data_ptr(),
                               Cb, N, H, H, Cout, K, 1, None) == 0  # accumulate onto 0.5
    scale = max(af.grad.abs().max().item(), 1.0)
    assert (dA.cpu() - 0.5 - af.grad).abs().max().item() <= 1e-4 * scale
    if Cb:
        assert (dB.cpu() - 0.5 - bf_.grad).abs().max().item() <= 1e-4 * scale
    dw = torch.empty(K, K, Ca + Cb, Cout, device="cuda")
    db = torch.empty(Cout, device="cuda")
    scratch = torch.empty(int(L.ecg_nn_wgrad_scratch(Ca + Cb, Cout, K)), device="cuda")
    assert L.ecg_nn_conv_wgrad(ad.data_ptr(), Ca, None if bd is None else bd.data_ptr(), Cb, dd.data_ptr(),
                               dw.data_ptr(), db.data_ptr(), scratch.data_ptr(), N, H, H, Cout, K, None) == 0
    sw = wf.grad.abs().max().item()
    assert (dw.cpu() - wf.grad).abs().max().item() <= 1e-4 * sw
    assert (db.cpu() - bias.grad).abs().max().item() <= 1e-4 * bias.grad.abs().max().item()


def test_pool_up_relu_mse_adam():
    g = torch.Generator().manual_seed(3)
    L = WS.lib()
    N, H, C = 2, 8, 6
    x = _bf(torch.randn(N, H, H, C, generator=g))
    xd = x.cuda()
    p = torch.empty(N, H // 2, H // 2, C, dtype=torch.bfloat16, device="cuda")
    assert L.ecg_nn_pool2(xd.data_ptr(), p.data_ptr(), N, H, H, C, None) == 0
    ref = F.avg_pool2d(x.float().permute(0, 3, 1, 2), 2).permute(0, 2, 3, 1)
    assert (p.float().cpu() - ref).abs().max().item() <= 1e-2
    dp = torch.randn(N, H // 2, H // 2, C, generator=g)
    dx = torch.zeros(N, H, H, C, device="cuda")
    assert L.ecg_nn_pool2_bwd(dp.cuda().data_ptr(), dx.data_ptr(), N, H, H, C, None) == 0
    assert torch.allclose(dx.cpu(), 0.25 * dp.repeat_interleave(2, 1).repeat_interleave(2, 2))
    u = torch.empty(N, 2 * H, 2 * H, C, dtype=torch.bfloat16, device="cuda")
    assert L.ecg_nn_up2(xd.data_ptr(), u.data_ptr(), N, H, H, C, None) == 0
    assert torch.equal(u.cpu(), x.repeat_interleave(2, 1).repeat_interleave(2, 2))
    du = torch.randn(N, 2 * H, 2 * H, C, generator=g)
    dxx = torch.empty(N, H, H, C, device="cuda")
    assert L.ecg_nn_up2_bwd(du.cuda().data_ptr(), dxx.data_ptr(), N, H, H, C, None) == 0
    ref_up = du.reshape(N, H, 2, H, 2, C).sum(dim=(2, 4))
    assert torch.allclose(dxx.cpu(), ref_up, atol=1e-5)
    d = torch.randn(N, H, H, C, generator=g)
    dd = d.cuda()
    assert L.ecg_nn_relu_bwd(xd.data_ptr(), dd.data_ptr(), d.numel(), None) == 0
    assert torch.equal(dd.cpu(), torch.where(x.float() > 0, d, torch.zeros_like(d)))
    pred, target = torch.randn(1000, generator=g), torch.randn(1000, generator=g)
    dpred = torch.empty(1000, device="cuda")
    loss = torch.zeros(257, dtype=torch.float64, device="cuda")
    assert L.ecg_nn_mse(pred.cuda().data_ptr(), target.cuda().data_ptr(), dpred.data_ptr(), loss.data_ptr(), 1000,
                        None) == 0
    assert abs(loss[0].item() - ((pred - target).double() ** 2).mean().item()) <= 1e-6
    assert torch.allclose(dpred.cpu(), 2 * (pred - target) / 1000, atol=1e-7)
    w = torch.randn(50, generator=g)
    gr = torch.randn(50, generator=g)
    m = torch.zeros(50)
    v = torch.zeros(50)
    wd_, gd, md, vd = w.cuda(), gr.cuda(), m.cuda(), v.cuda()
    w16 = torch.empty(50, dtype=torch.bfloat16, device="cuda")
    assert L.ecg_nn_adam(wd_.data_ptr(), w16.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), 50, 1e-2, 0.9,
                         0.999, 1e-8, 1, None) == 0
    m1 = 0.1 * gr
    v1 = 0.001 * gr * gr
    ref_w = w - 1e-2 * (m1 / 0.1) / (torch.sqrt(v1 / 0.001) + 1e-8)
    assert torch.allclose(wd_.cpu(), ref_w, atol=1e-6)
    assert torch.equal(w16.cpu(), ref_w.to(torch.bfloat16)) or (w16.float().cpu() - ref_w).abs().max() < 1e-2


def test_energy_loss_matches_the_sparse_matrix():
    # e^T A e and A e against workloads.diffusion2d's CSR matrix
    g = np.random.default_rng(5)
    side, N = 12, 2
    kap = np.exp(g.standard_normal((N, side, side)))
    pred = g.standard_normal((N, side, side)).astype(np.float32)
    targ = g.standard_normal((N, side, side)).astype(np.float32)
    w = np.array([0.7, 1.3], dtype=np.float32)
    dpred = torch.empty(N, side, side, device="cuda")
    loss = torch.zeros(257, dtype=torch.float64, device="cuda")
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    assert WS.lib().ecg_nn_energy_loss(td(pred).data_ptr(), td(targ).data_ptr(), td(kap).data_ptr(), td(w).data_ptr(),
                                       dpred.data_ptr(), loss.data_ptr(), N, side, None) == 0
    tot = 0.0
    for n in range(N):
        A = W.diffusion2d(kap[n].astype(np.float32).astype(np.float64))
        e = (pred[n] - targ[n]).astype(np.float64).ravel()
        Ae = A @ e
        tot += w[n] * e @ Ae
        np.testing.assert_allclose(dpred[n].cpu().numpy().ravel(), 2 * w[n] * Ae, rtol=1e-4, atol=1e-4 * np.abs(Ae).max())
    assert abs(loss[0].item() - tot) <= 1e-4 * abs(tot)


def _ref_network(net, x, round_acts):
    """The network in plain PyTorch FP32 on the CPU with the GPU's bf16
    weights; round_acts rounds every stored activation to bf16 as the GPU
    does."""
    R = (lambda t: t.to(torch.bfloat16).float()) if round_acts else (lambda t: t)
    P = {k: (v["w16"].float().cpu().requires_grad_(), v["b"].cpu().requires_grad_()) for k, v in net.params.items()}

    def c(name, xs, relu=True, K=3):
        x_ = torch.cat(xs, dim=3) if len(xs) > 1 else xs[0]
        y = F.conv2d(x_.permute(0, 3, 1, 2), P[name][0].permute(3, 2, 0, 1), P[name][1], padding=K // 2)
        y = y.permute(0, 2, 3, 1)
        return F.relu(y) if relu else y

    def pool(t):
        return F.avg_pool2d(t.permute(0, 3, 1, 2), 2).permute(0, 2, 3, 1)

    def up(t):
        return t.repeat_interleave(2, 1).repeat_interleave(2, 2)

    x = x.float().cpu()
    a0a = R(c("enc0a", [x]))
    s0 = R(c("enc0b", [a0a]))
    p0 = R(pool(s0))
    a1a = R(c("enc1a", [p0]))
    s1 = R(c("enc1b", [a1a]))
    p1 = R(pool(s1))
    mb = R(c("mid_b", [R(c("mid_a", [p1]))]))
    d1b = R(c("dec1b", [R(c("dec1a", [up(mb), s1]))]))
    d0b = R(c("dec0b", [R(c("dec0a", [up(d1b), s0]))]))
    return c("head", [d0b], relu=False, K=1), P


def test_network_forward_and_gradients_match_pytorch():
    # forward against the reference with bf16-rounded activations; the
    # gradients of every layer against autograd of the unrounded reference
    # (the GPU backward reads the bf16 activations, so a few percent)
    net = WS.WarmStartNet(side=32, batch=2, seed=1)
    g = torch.Generator().manual_seed(9)
    x = torch.randn(2, 32, 32, 2, generator=g).to(torch.bfloat16).cuda()
    y = torch.randn(2, 32, 32, 1, generator=g).cuda()
    out = net.forward(x)
    ref, _ = _ref_network(net, x, True)
    assert (out.cpu() - ref.detach()).abs().max().item() <= 1e-2 * ref.abs().max().item()
    dout = net.loss_and_grad(out, y)
    # the loss squares FP32 differences in FP64
    assert abs(net.loss_buf[0].item() - ((out - y).double() ** 2).mean().item()) <= 1e-12
    net.backward(dout)
    ref2, P = _ref_network(net, x, False)
    ((ref2 - y.cpu()) ** 2).mean().backward()
    for name, _, _, _, _, _ in WS.LAYERS:
        gw, gref = net.params[name]["gw"].cpu(), P[name][0].grad
        assert ((gw - gref).norm() / gref.norm()).item() <= 0.15, name
        gb, gbref = net.params[name]["gb"].cpu(), P[name][1].grad
        assert ((gb - gbref).norm() / gbref.norm()).item() <= 0.15, name


def test_stop_rule_b_matches_oracle_with_scaled_tolerance():
    import oracle as O

    p = W.poisson2d(64, 4, seed=1001)
    x0 = 0.5 * p.x_star
    r0 = np.linalg.norm(p.b - p.scipy() @ x0)
    tol = 1e-8
    o = O.ecg_solve(p.scipy(), p.part, 4, p.b, x0=x0, tol=tol * np.linalg.norm(p.b) / r0, maxit=3000)
    with ecg.Solver.from_problem(p, stop_rule=ecg.STOP_B) as s:
        g = s.solve(torch.from_numpy(p.b).cuda(), x0=torch.from_numpy(x0).cuda(), tol=tol, maxit=3000)
    assert g.status == ecg.OK
    assert abs(g.iters - o.iters) <= 1
    assert g.history[g.iters] <= tol * np.linalg.norm(p.b) * (1 + 1e-12)


def test_training_and_warm_started_solves():
    # a small version of the workload: 48 training solves on 64 x 64 grids;
    # the energy-norm loss must fall, every warm-started solve must reach
    # the tolerance, and the smoothed proposal must start below ||b||
    # (whether it saves iterations is measured by bench.py --warmstart; at
    # these training scales it does not; a warm start must not cost more than
    # 5 % extra iterations)
    train = WS.make_dataset(48, side=64, t=16, seed0=7000, prec_blocks=16)
    held = WS.make_dataset(4, side=64, t=16, seed0=9000, solve=False)
    net = WS.WarmStartNet(side=64, batch=8, seed=2)
    hist = WS.train(net, train, epochs=30, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    rows = WS.evaluate(net, held, tol=1e-8, trunc=2, sweeps=16)
    for r in rows:
        assert r["status_zero"] == 0 and r["status_net"] == 0, r
        assert r["relres_true_net"] <= 1.0000001e-8, r
        assert r["used"] and r["x0_relres"] < 1.0, r
        assert r["iters_net"] <= 1.05 * r["iters_zero"], r
