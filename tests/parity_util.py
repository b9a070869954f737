"""Solve-level parity criterion shared by GPU tests: the GPU run is compared
with the oracle inside the oracle's own sensitivity to rounding.

The oracle is run on b and on four copies of b perturbed by 1e-15
relative, and once with the other orthonormalisation.  The GPU run must
  (a) track the oracle's residual history to 1e-8 rho_0 for as long as the
      oracle tracks its own perturbed runs to 1e-12 rho_0 (the whole run
      when the problem is stable).  The GPU's rounding enters at every
      iteration, the perturbation of b only once, so the GPU leaves the
      oracle an iteration or two before the perturbed runs do; once a run
      is chaotic a deviation grows about 100x per iteration, and the
      1e-12 onset leaves those iterations' margin against the 1e-8 bar,
  (b) converge within the iteration range of those runs widened by its
      width (at least +-2), and
  (c) end within ten times the oracle's own spread of x (at least 1e-8).
"""
import numpy as np

import oracle as O


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def envelope_check(p, g_iters, g_hist, g_x, okw, maxit, prec=None, tol=1e-8):
    A = p.scipy()
    o = O.ecg_solve(A, p.part, p.t, p.b, tol=tol, maxit=maxit, prec=prec, **okw)
    assert o.status == 0, o.status
    rng = np.random.default_rng(99)
    variants = []
    for _ in range(4):
        bp = p.b * (1.0 + 1e-15 * rng.standard_normal(p.n))
        variants.append(O.ecg_solve(A, p.part, p.t, bp, tol=tol, maxit=maxit, prec=prec, **okw))
    kw2 = dict(okw)
    kw2["ortho"] = 1 - kw2.get("ortho", 0)
    variants.append(O.ecg_solve(A, p.part, p.t, p.b, tol=tol, maxit=maxit, prec=prec, **kw2))
    assert all(v.status == 0 for v in variants)
    its = [o.iters] + [v.iters for v in variants]
    lo, hi = min(its), max(its)
    width = max(2, hi - lo)
    assert lo - width <= g_iters <= hi + width, (g_iters, its)
    h0 = o.history[0]
    kdiv = min(g_iters, o.iters)
    for v in variants[:4]:
        k = min(kdiv, v.iters)
        d = np.abs(v.history[: k + 1] - o.history[: k + 1]) > 1e-12 * h0
        if np.any(d):
            kdiv = min(kdiv, int(np.argmax(d)))
    assert np.all(np.abs(g_hist[: kdiv + 1] - o.history[: kdiv + 1]) <= 1e-8 * h0), kdiv
    xspread = max(rel(v.x, o.x) for v in variants)
    assert rel(g_x, o.x) <= max(1e-8, 10.0 * xspread), (rel(g_x, o.x), xspread)
    return o
