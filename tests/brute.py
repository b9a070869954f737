"""Extended-precision brute force for tiny problems (test helper).

Builds an explicit basis of the search space a method is supposed to use and
solves the Galerkin system in mpmath.  For any basis V of the space S,
x = x0 + V (V^T A V)^{-1} V^T r0 is the unique iterate with x - x0 in S and
b - A x orthogonal to S (Section 2: subspace and orthogonality conditions).
This file shares nothing with the oracle or the CUDA path.
"""
import mpmath as mp
import numpy as np


def to_mp_dense(A):
    Ad = A.toarray()
    return mp.matrix(Ad.tolist())


def mp_vec(v):
    return mp.matrix([[mp.mpf(float(x))] for x in v])


def split_cols(part, w, r, half=False):
    """Columns of [T^w(r)] built from the definition: r restricted to each
    subdomain (merged pairs when half=True)."""
    n = len(part)
    cols = []
    for j in range(w):
        c = mp.matrix(n, 1)
        for i in range(n):
            d = part[i] // 2 if half else part[i]
            if d == j:
                c[i] = r[i]
        cols.append(c)
    return cols


def galerkin(A, x0, r0, cols):
    n = A.rows
    m = len(cols)
    V = mp.matrix(n, m)
    for j, c in enumerate(cols):
        for i in range(n):
            V[i, j] = c[i]
    G = V.T * A * V
    y = mp.lu_solve(G, V.T * r0)
    return x0 + V * y


def to_np(v):
    return np.array([float(v[i]) for i in range(v.rows)])


def krylov_block(A, start_cols, k):
    """Columns of A^j C for j = 0..k-1 and C = start_cols."""
    out = []
    cur = list(start_cols)
    for j in range(k):
        out.extend(cur)
        cur = [A * c for c in cur]
    return out


def a_orthonormal_basis(A, cols):
    """A-orthonormal basis of span(cols) by Gram-Schmidt (twice) in mpmath."""
    Q = []
    for c in cols:
        v = c.copy()
        for _ in range(2):
            for q in Q:
                v = v - q * (q.T * (A * v))[0]
        nrm = mp.sqrt((v.T * (A * v))[0])
        Q.append(v / nrm)
    return Q


def project_out(A, Q, cols):
    """Remove from each column its A-orthogonal projection onto span(Q),
    Q A-orthonormal."""
    out = []
    for c in cols:
        v = c.copy()
        for q in Q:
            v = v - q * (q.T * (A * c))[0]
        out.append(v)
    return out


def flexible_sre_iterates(A, b, part, t, kF, K):
    """Exact-arithmetic iterates of flexibly SRE-CG2 (Algorithm 3) with the
    switch after iteration kF: blocks B_1 = [T^t(r_0)], B_k = A B~_{k-1}
    (B~ = block after its A-orthogonal projection against all earlier
    blocks), except B_{kF+1} = [T^{t/2}(r_kF)].  x_k is the Galerkin iterate
    over span(B_1..B_k).  kF = 0 means no switch."""
    n = A.rows
    x0 = mp.matrix(n, 1)
    cols = []
    xs = []
    prev = None
    xk = x0
    for k in range(1, K + 1):
        if k == 1:
            B = split_cols(part, t, b)
        elif kF and k == kF + 1:
            B = split_cols(part, t // 2, b - A * xk, half=True)
        else:
            B = [A * c for c in prev]
        Qb = a_orthonormal_basis(A, cols) if cols else []
        Bt = project_out(A, Qb, B)
        cols = cols + Bt
        prev = Bt
        xk = galerkin(A, x0, b, cols)
        xs.append(xk)
    return xs
