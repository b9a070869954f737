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
      width (at least +-2 and +-1% of the count: the perturbed runs inject
      rounding once, in b, while the GPU's arithmetic differs from the
      oracle's at every iteration), and
  (c) end within ten times the oracle's own spread of x (at least 1e-8).
"""
import numpy as np

import oracle as O


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# The oracle's runs count as tracking each other while their residual
# histories agree to ONSET rho_0; the GPU is held to TRACK rho_0 up to there.
ONSET = 1e-12
TRACK = 1e-8


def envelope_metrics(p, g_iters, g_hist, g_x, okw, maxit, prec=None, tol=1e-8, o=None, nperturbed=4,
                     other_ortho=True):
    """The quantities criteria (a)-(c) above compare, for a GPU run
    (iterations, residual history, final x) of problem p with oracle options
    okw, without asserting anything.  o is the oracle's own run on p.b when
    already computed.  nperturbed and other_ortho choose the oracle runs that
    span the envelope (fewer for problems too large to solve six times)."""
    A = p.scipy()
    if o is None:
        o = O.ecg_solve(A, p.part, p.t, p.b, tol=tol, maxit=maxit, prec=prec, **okw)
    rng = np.random.default_rng(99)
    variants = []
    for _ in range(nperturbed):
        bp = p.b * (1.0 + 1e-15 * rng.standard_normal(p.n))
        variants.append(O.ecg_solve(A, p.part, p.t, bp, tol=tol, maxit=maxit, prec=prec, **okw))
    perturbed = list(variants)
    if other_ortho:
        kw2 = dict(okw)
        kw2["ortho"] = 1 - kw2.get("ortho", 0)
        variants.append(O.ecg_solve(A, p.part, p.t, p.b, tol=tol, maxit=maxit, prec=prec, **kw2))
    its = [o.iters] + [v.iters for v in variants]
    h0 = o.history[0]
    kdiv = min(g_iters, o.iters)
    for v in perturbed:
        k = min(kdiv, v.iters)
        d = np.abs(v.history[: k + 1] - o.history[: k + 1]) > ONSET * h0
        if np.any(d):
            kdiv = min(kdiv, int(np.argmax(d)))
    hist_dev = float(np.max(np.abs(g_hist[: kdiv + 1] - o.history[: kdiv + 1])) / h0)
    xspread = max(rel(v.x, o.x) for v in variants)
    return {"oracle": o, "variants": variants, "oracle_iters": its, "iters_delta": g_iters - o.iters,
            "onset": kdiv, "hist_dev_to_onset": hist_dev, "x_rel_err": rel(g_x, o.x), "x_spread": xspread}


def envelope_assert(m, g_iters):
    """Assert criteria (a)-(c) on the output of envelope_metrics."""
    assert m["oracle"].status == 0, m["oracle"].status
    assert all(v.status == 0 for v in m["variants"])
    its = m["oracle_iters"]
    lo, hi = min(its), max(its)
    # the perturbed runs inject rounding once (in b); a different FP64
    # implementation injects it at every iteration, which moves long
    # truncated runs by a few tenths of a percent more: at least 1%
    width = max(2, hi - lo, -(-hi // 100))
    assert lo - width <= g_iters <= hi + width, (g_iters, its)
    assert m["hist_dev_to_onset"] <= TRACK, (m["onset"], m["hist_dev_to_onset"])
    assert m["x_rel_err"] <= max(1e-8, 10.0 * m["x_spread"]), (m["x_rel_err"], m["x_spread"])


def envelope_check(p, g_iters, g_hist, g_x, okw, maxit, **kw):
    """envelope_metrics, then envelope_assert; returns the metrics."""
    m = envelope_metrics(p, g_iters, g_hist, g_x, okw, maxit, **kw)
    envelope_assert(m, g_iters)
    return m
