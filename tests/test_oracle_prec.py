"""Pins of the oracle's block Jacobi preconditioner and of the preconditioned
enlarged CG methods (Section 3 "Preconditioned versions", eq. (zsre2),
(zmsd2), Algorithm 5; the block Jacobi preconditioner of Section 5).

Each check is against something other than the oracle itself:
- the factors against numpy's dense Cholesky and against the defining
  property of IC(0);
- the substitutions against scipy's dense triangular solves;
- the preconditioned solver against textbook PCG (t = 1), against the
  unpreconditioned oracle run on L^{-1} A L^{-T} (the paper's first option,
  which Section 3 shows equal to the second), and against the one-step
  convergence that M = A forces.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from paper_2305_19013_gb300 import workloads as W


def _dense_factor(pc, n):
    I, J, V = pc.factor()
    return sp.csr_matrix((V, (I, J)), shape=(n, n)).toarray()


def _same_block(pb):
    return np.equal.outer(pb, pb)


def test_exact_block_cholesky_matches_numpy():
    p = W.random_spd_grid(12, 4, seed=5)
    A = p.scipy().toarray()
    pb = p.part
    pc = O.BlockJacobi(p.scipy(), pb, 4, O.PREC_CHOL)
    L = _dense_factor(pc, p.n)
    for blk in range(4):
        idx = np.nonzero(pb == blk)[0]
        ref = np.linalg.cholesky(A[np.ix_(idx, idx)])
        np.testing.assert_allclose(L[np.ix_(idx, idx)], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    # nothing outside the diagonal blocks
    assert np.all(L[~_same_block(pb)] == 0.0)


def test_ic0_equals_cholesky_without_fill():
    # a 1D chain (tridiagonal) has a Cholesky factor with no fill, so IC(0)
    # must be the exact factor
    n = 40
    rng = np.random.default_rng(3)
    off = -rng.uniform(0.5, 1.5, n - 1)
    d = np.zeros(n)
    d[:-1] -= off
    d[1:] -= off
    d += rng.uniform(0.1, 1.0, n)
    A = sp.diags([off, d, off], [-1, 0, 1]).tocsr()
    pb = (np.arange(n) * 3 // n).astype(np.int32)
    L_ic = _dense_factor(O.BlockJacobi(A, pb, 3, O.PREC_IC0), n)
    L_ch = _dense_factor(O.BlockJacobi(A, pb, 3, O.PREC_CHOL), n)
    np.testing.assert_allclose(L_ic, L_ch, rtol=0, atol=1e-14)


def test_ic0_defining_property_2d():
    # IC(0): L has the pattern of tril(A_i) and (L L^T)_ij = a_ij on that
    # pattern; off the pattern L L^T differs (the dropped fill)
    p = W.random_spd_grid(16, 4, seed=9)
    A = p.scipy().toarray()
    pb = W.jacobi_blocks(p, 16)
    L = _dense_factor(O.BlockJacobi(p.scipy(), pb, 16, O.PREC_IC0), p.n)
    pat = (A != 0) & _same_block(pb)
    assert np.all((L != 0) <= np.tril(pat))
    assert np.all(np.diag(L) > 0)
    M = L @ L.T
    np.testing.assert_allclose(M[pat], A[pat], rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.abs(M[~pat]).max() > 1e-3  # fill was dropped


@pytest.mark.parametrize("kind", [O.PREC_CHOL, O.PREC_IC0])
def test_substitutions_match_scipy(kind):
    p = W.random_spd_grid(12, 4, seed=2)
    pb = W.jacobi_blocks(p, 16)
    pc = O.BlockJacobi(p.scipy(), pb, 16, kind)
    L = _dense_factor(pc, p.n)
    X = np.random.default_rng(0).standard_normal((p.n, 3))
    y = sla.solve_triangular(L, X, lower=True)
    z = sla.solve_triangular(L.T, X, lower=False)
    np.testing.assert_allclose(pc.lsolve(X), y, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pc.ltsolve(X), z, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pc.apply(X), np.linalg.solve(L @ L.T, X), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(pc.apply(X[:, 0]), np.linalg.solve(L @ L.T, X[:, 0]), rtol=1e-10, atol=1e-12)


def test_aligned_blocks_split_commutes():
    # Section 3: with diagonal blocks inside the subdomains,
    # L^{-T}[T(L^{-1} r)] = [T(M^{-1} r)] (the form the GPU path uses)
    p = W.random_spd_grid(16, 4, seed=4)
    pb = W.jacobi_blocks(p, 16)
    pc = O.BlockJacobi(p.scipy(), pb, 16, O.PREC_IC0)
    r = p.b
    lhs = pc.ltsolve(O.split(p.part, 4, pc.lsolve(r)))
    rhs = O.split(p.part, 4, pc.apply(r))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-14)
    lhs2 = pc.ltsolve(O.split_half(p.part, 4, pc.lsolve(r)))
    rhs2 = O.split_half(p.part, 4, pc.apply(r))
    np.testing.assert_allclose(lhs2, rhs2, rtol=1e-12, atol=1e-14)


def _pcg(A, b, Minv, iters):
    """Textbook preconditioned CG (Hestenes-Stiefel with z = M^{-1} r)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = Minv(r)
    pdir = z.copy()
    rz = r @ z
    xs = []
    for _ in range(iters):
        q = A @ pdir
        a = rz / (pdir @ q)
        x = x + a * pdir
        r = r - a * q
        z = Minv(r)
        rz_new = r @ z
        pdir = z + (rz_new / rz) * pdir
        rz = rz_new
        xs.append(x.copy())
    return xs


@pytest.mark.parametrize("kind", [O.PREC_CHOL, O.PREC_IC0])
def test_t1_preconditioned_is_pcg(kind):
    p = W.random_spd_grid(14, 4, seed=8)
    A = p.scipy()
    pb = W.jacobi_blocks(p, 16)
    pc = O.BlockJacobi(A, pb, 16, kind)
    L = _dense_factor(pc, p.n)
    M = L @ L.T
    iters = 25
    ref = _pcg(A, p.b, lambda v: np.linalg.solve(M, v), iters)
    part1 = np.zeros(p.n, dtype=np.int32)
    o = O.ecg_solve(A, part1, 1, p.b, tol=0.0, maxit=iters + 1, trunc=0, keep_x=True, prec=pc)
    assert o.iters == iters
    for k in range(iters):
        np.testing.assert_allclose(o.xhist[k], ref[k], rtol=0, atol=1e-9 * np.linalg.norm(ref[k]))


@pytest.mark.parametrize(
    "variant,trunc,ortho",
    [("sre", 0, 0), ("sre", 2, 0), ("sre", 2, 1), ("msdo", 1, 0), ("msdo", 2, 1), ("modmsdo", 3, 0)],
)
def test_split_preconditioning_equals_transformed_system(variant, trunc, ortho):
    """Section 3: running the method on A^ = L^{-1} A L^{-T}, b^ = L^{-1} b
    and mapping x = L^{-T} x^ gives the iterates of the preconditioned form."""
    p = W.random_spd_grid(12, 4, seed=6)
    A = p.scipy()
    pb = W.jacobi_blocks(p, 16)
    pc = O.BlockJacobi(A, pb, 16, O.PREC_IC0)
    L = _dense_factor(pc, p.n)
    Li = np.linalg.inv(L)
    Ah = Li @ A.toarray() @ Li.T
    Ah = 0.5 * (Ah + Ah.T)
    bh = Li @ p.b
    iters = 8
    kw = dict(tol=0.0, maxit=iters + 1, trunc=trunc, variant=variant, ortho=ortho, keep_x=True)
    o_hat = O.ecg_solve(sp.csr_matrix(Ah), p.part, 4, bh, **kw)
    o = O.ecg_solve(A, p.part, 4, p.b, prec=pc, **kw)
    assert o.iters == o_hat.iters == iters
    for k in range(iters):
        ref = Li.T @ o_hat.xhist[k]
        np.testing.assert_allclose(o.xhist[k], ref, rtol=0, atol=1e-8 * np.linalg.norm(ref))


@pytest.mark.parametrize("t", [2, 4])
def test_exact_single_block_converges_in_one_step(t):
    # one diagonal block with its exact Cholesky factor: M = A, and
    # L^{-T}[T(L^{-1} r_0)] sums to A^{-1} r_0, so x_1 is the solution
    p = W.random_spd_grid(10, t, seed=12)
    A = p.scipy()
    pc = O.BlockJacobi(A, np.zeros(p.n, dtype=np.int32), 1, O.PREC_CHOL)
    o = O.ecg_solve(A, p.part, t, p.b, tol=1e-12, maxit=20, prec=pc)
    assert o.iters == 1
    np.testing.assert_allclose(o.x, p.x_star, rtol=0, atol=1e-10)


def test_preconditioning_cuts_iterations():
    # Section 5, Tables 10-13: block Jacobi cuts the iteration counts
    p = W.blocky_diffusion2d(64, 4, blocks=8, seed=21)
    A = p.scipy()
    pb = W.jacobi_blocks(p, 16)
    plain = O.ecg_solve(A, p.part, 4, p.b, tol=1e-8, maxit=3000, trunc=2)
    for kind in (O.PREC_CHOL, O.PREC_IC0):
        pc = O.BlockJacobi(A, pb, 16, kind)
        o = O.ecg_solve(A, p.part, 4, p.b, tol=1e-8, maxit=3000, trunc=2, prec=pc)
        assert o.status == O.OK and o.relres_true < 1e-7
        assert o.iters < 0.6 * plain.iters, (kind, o.iters, plain.iters)


def test_prec_setup_rejects_bad_blocks():
    p = W.random_spd_grid(8, 2, seed=1)
    bad = np.zeros(p.n, dtype=np.int32)
    with pytest.raises(ValueError):
        O.BlockJacobi(p.scipy(), bad, 2, O.PREC_IC0)  # block 1 empty
    bad[0] = 5
    with pytest.raises(ValueError):
        O.BlockJacobi(p.scipy(), bad, 2, O.PREC_IC0)  # id out of range


# ------------------------------------------------- block-residual ECG (Section 1)


@pytest.mark.parametrize("trunc", [0, 2])
def test_block_residual_sum_equals_sre(trunc):
    # alpha_k 1 = W_k^T R_{k-1} 1 = W_k^T r_{k-1}: summing the block solution's
    # columns gives the vector SRE-CG2 iterates (the same direction blocks)
    p = W.random_spd_grid(14, 4, seed=31)
    A = p.scipy()
    ob = O.becg_solve(A, p.part, 4, p.b, tol=0.0, maxit=15, trunc=trunc, keep_x=True)
    ov = O.ecg_solve(A, p.part, 4, p.b, tol=0.0, maxit=15, trunc=trunc, keep_x=True)
    assert ob.iters == ov.iters == 14
    for k in range(14):
        np.testing.assert_allclose(ob.xhist[k], ov.xhist[k], rtol=0, atol=1e-10 * np.linalg.norm(ov.xhist[k]))


def test_block_residual_columns_solve_their_subdomain_rhs():
    # with the full window the method is block CG on A X = [T^t(r_0)]: at
    # convergence column j solves A X_j = T_j(r_0), and the residual block is
    # A-Galerkin-orthogonal per column (checked against a dense solve)
    p = W.random_spd_grid(10, 4, seed=32)
    A = p.scipy()
    ob = O.becg_solve(A, p.part, 4, p.b, tol=1e-12, maxit=200, trunc=0)
    assert ob.status == O.OK
    X = ob.basis[0]
    Ad = A.toarray()
    for j in range(4):
        rhs = np.where(p.part == j, p.b, 0.0)
        ref = np.linalg.solve(Ad, rhs)
        np.testing.assert_allclose(X[:, j], ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose(ob.x, np.linalg.solve(Ad, p.b), rtol=0, atol=1e-9)


def test_block_residual_t1_is_cg():
    # t = 1: block CG with one column is CG (compared over the iterations
    # before CG's own loss of orthogonality sets in on this 144-row system)
    p = W.random_spd_grid(12, 1, seed=33)
    A = p.scipy()
    ob = O.becg_solve(A, np.zeros(p.n, dtype=np.int32), 1, p.b, tol=0.0, maxit=11, trunc=0, keep_x=True)
    oc = O.cg_solve(A, p.b, tol=0.0, maxit=11, keep_x=True)
    for k in range(10):
        np.testing.assert_allclose(ob.xhist[k], oc.xhist[k], rtol=0, atol=1e-9 * np.linalg.norm(oc.xhist[k]))
