"""Seeded synthetic inputs for the enlarged CG solvers.

This module builds problems only: sparse SPD matrices in CSR form, subdomain
partitions, right-hand sides and exact solutions.  It holds none of the
solver's arithmetic and imports nothing from the CUDA path or the oracle, so
both the tests and the benchmark may draw inputs from it.

The matrices stand in for the paper's FreeFem++ test matrices (Section 5,
Table 1), which are not available: Dirichlet-eliminated 5-point (2D) and
7-point (3D) finite-difference diffusion stencils with cell-wise coefficients
and harmonic-mean face coefficients.  At 100x100 (2D) and 20^3 (3D) they have
exactly the sizes and nonzero counts of Table 1 (n=10000, nnz=49600 and
n=8000, nnz=53600).

As in the paper's setup (Section 5: METIS k-way partitioning, then a
reordering so that every subdomain is a contiguous index range), rows are by
default renumbered so that subdomain 0 comes first, then subdomain 1, etc.,
keeping the lexicographic order inside each subdomain.  Subdomain ids are
numbered so that merging the pairs {2j, 2j+1} (the halving of Section 4,
eq. (Tt)) merges two geometrically adjacent blocks.

All random draws use numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """One linear system A x = b with a subdomain partition of its rows."""

    name: str
    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    part: np.ndarray  # int32[n], subdomain id of each row, values in [0, t)
    t: int
    b: np.ndarray  # float64[n]
    x_star: np.ndarray | None  # float64[n] when b = A x_star, else None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _harmonic(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return 2.0 * a * b / (a + b)


def diffusion2d(kappa: np.ndarray) -> sp.csr_matrix:
    """5-point stencil of -div(kappa grad u) on an ny x nx cell grid.

    kappa has shape (ny, nx).  Interior faces take the harmonic mean of the
    two cell coefficients; a face on the (eliminated) Dirichlet boundary takes
    the cell's own coefficient.  Row index = y*nx + x.  With kappa == 1 this
    is the classical (4, -1, -1, -1, -1) Laplacian.
    """
    ny, nx = kappa.shape
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    diag = np.zeros((ny, nx))
    rows, cols, vals = [], [], []
    # x-faces
    fx = _harmonic(kappa[:, :-1], kappa[:, 1:])
    diag[:, :-1] += fx
    diag[:, 1:] += fx
    diag[:, 0] += kappa[:, 0]
    diag[:, -1] += kappa[:, -1]
    rows += [idx[:, :-1].ravel(), idx[:, 1:].ravel()]
    cols += [idx[:, 1:].ravel(), idx[:, :-1].ravel()]
    vals += [-fx.ravel(), -fx.ravel()]
    # y-faces
    fy = _harmonic(kappa[:-1, :], kappa[1:, :])
    diag[:-1, :] += fy
    diag[1:, :] += fy
    diag[0, :] += kappa[0, :]
    diag[-1, :] += kappa[-1, :]
    rows += [idx[:-1, :].ravel(), idx[1:, :].ravel()]
    cols += [idx[1:, :].ravel(), idx[:-1, :].ravel()]
    vals += [-fy.ravel(), -fy.ravel()]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)
    ).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def diffusion3d(kx: np.ndarray, ky: np.ndarray, kz: np.ndarray) -> sp.csr_matrix:
    """7-point stencil of -div(K grad u), K = diag(kx, ky, kz) per cell.

    Arrays have shape (nz, ny, nx); row index = (z*ny + y)*nx + x.  Faces
    normal to axis a take the harmonic mean of the two cells' k_a; boundary
    faces take the cell's own k_a.
    """
    nz, ny, nx = kx.shape
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    diag = np.zeros((nz, ny, nx))
    rows, cols, vals = [], [], []
    for axis, k in ((2, kx), (1, ky), (0, kz)):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(None, -1)
        hi[axis] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        f = _harmonic(k[lo], k[hi])
        diag[lo] += f
        diag[hi] += f
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[axis] = 0
        last[axis] = -1
        diag[tuple(first)] += k[tuple(first)]
        diag[tuple(last)] += k[tuple(last)]
        rows += [idx[lo].ravel(), idx[hi].ravel()]
        cols += [idx[hi].ravel(), idx[lo].ravel()]
        vals += [-f.ravel(), -f.ravel()]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)
    ).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def block_partition2d(nx: int, ny: int, px: int, py: int) -> np.ndarray:
    """Rectangular px x py block partition of an ny x nx grid.

    Subdomain id = by*px + bx, so pairs {2j, 2j+1} are horizontally adjacent
    blocks when px is even (and vertically adjacent strips when px == 1).
    Block bx covers the columns x with floor(x*px/nx) = bx (equal blocks
    when px divides nx).
    """
    if px > nx or py > ny:
        raise ValueError("more blocks than grid lines")
    y, x = np.divmod(np.arange(nx * ny), nx)
    return ((y * py // ny) * px + (x * px // nx)).astype(np.int32)


def block_partition3d(nx: int, ny: int, nz: int, px: int, py: int, pz: int) -> np.ndarray:
    """Rectangular px x py x pz block partition; id = (bz*py + by)*px + bx."""
    if px > nx or py > ny or pz > nz:
        raise ValueError("more blocks than grid lines")
    i = np.arange(nx * ny * nz)
    z, rem = np.divmod(i, nx * ny)
    y, x = np.divmod(rem, nx)
    return (((z * pz // nz) * py + (y * py // ny)) * px + (x * px // nx)).astype(np.int32)


def reorder_by_subdomain(A: sp.csr_matrix, part: np.ndarray):
    """Symmetric permutation making every subdomain a contiguous row range.

    Returns (A_perm, part_perm, perm) with A_perm = A[perm][:, perm]; new row
    r is old row perm[r].  Stable, so the lexicographic order inside each
    subdomain is kept.
    """
    perm = np.argsort(part, kind="stable")
    Ap = A[perm][:, perm].tocsr()
    Ap.sort_indices()
    return Ap, part[perm].astype(np.int32), perm


def _finish(name, A, part, t, b, x_star, meta, reorder):
    if reorder:
        A, part, perm = reorder_by_subdomain(A, part)
        b = b[perm]
        x_star = None if x_star is None else x_star[perm]
        meta = dict(meta, perm=perm)
    A = A.tocsr()
    return Problem(
        name=name,
        n=A.shape[0],
        rowptr=A.indptr.astype(np.int64),
        col=A.indices.astype(np.int32),
        val=A.data.astype(np.float64),
        part=np.ascontiguousarray(part, dtype=np.int32),
        t=int(t),
        b=np.ascontiguousarray(b, dtype=np.float64),
        x_star=None if x_star is None else np.ascontiguousarray(x_star, dtype=np.float64),
        meta=meta,
    )


def poisson2d(side: int = 64, strips: int = 4, seed: int = 1000, reorder: bool = True) -> Problem:
    """2D Poisson 5-point on side x side, t row strips, x* ~ U[-1,1], b = A x*.

    At side=64, strips=4 this is the 4096-unknown workload with 4 strips of
    16 grid rows.
    """
    rng = _rng(seed)
    A = diffusion2d(np.ones((side, side)))
    part = block_partition2d(side, side, 1, strips)
    x_star = rng.uniform(-1.0, 1.0, side * side)
    b = A @ x_star
    return _finish(f"poisson2d_{side}", A, part, strips, b, x_star, {"side": side}, reorder)


def blocky_diffusion2d(
    side: int = 1024,
    t: int = 16,
    blocks: int = 16,
    seed: int = 2000,
    reorder: bool = True,
    rhs: str = "uniform",
) -> Problem:
    """2D heterogeneous diffusion: kappa piecewise constant on blocks x blocks
    tiles, each tile log-uniform in [1, 1e3]; t rectangular subdomains
    (8 = 4x2, 16 = 4x4, 32 = 8x4, otherwise a near-square power-of-two split).

    rhs="uniform": b ~ U[-1,1] (x* unknown); rhs="manufactured": x* ~ U[-1,1],
    b = A x*.
    """
    rng = _rng(seed)
    tile = side // blocks
    logk = rng.uniform(0.0, 3.0, (blocks, blocks))
    kappa = np.repeat(np.repeat(10.0**logk, tile, axis=0), tile, axis=1)
    A = diffusion2d(kappa)
    px, py = _split2(t)
    part = block_partition2d(side, side, px, py)
    if rhs == "uniform":
        b = rng.uniform(-1.0, 1.0, side * side)
        x_star = None
    else:
        x_star = rng.uniform(-1.0, 1.0, side * side)
        b = A @ x_star
    return _finish(f"diffusion2d_{side}_t{t}", A, part, t, b, x_star, {"side": side}, reorder)


def anisotropic_diffusion3d(side: int = 128, t: int = 16, seed: int = 3000, reorder: bool = True) -> Problem:
    """3D anisotropic diffusion, 7-point on side^3.  Diagonal tensor with one
    axis weakened to 1e-2; the weak axis is chosen per octant (octant
    o = ox + 2*oy + 4*oz has its weak axis o mod 3).  t=16 subdomains are
    4x2x2 boxes.  x* ~ U[-1,1], b = A x*.
    """
    rng = _rng(seed)
    h = side // 2
    k = [np.ones((side, side, side)) for _ in range(3)]  # kx, ky, kz
    for oz in range(2):
        for oy in range(2):
            for ox in range(2):
                o = ox + 2 * oy + 4 * oz
                sl = (slice(oz * h, (oz + 1) * h), slice(oy * h, (oy + 1) * h), slice(ox * h, (ox + 1) * h))
                k[o % 3][sl] = 1e-2
    A = diffusion3d(k[0], k[1], k[2])
    px, py, pz = _split3(t)
    part = block_partition3d(side, side, side, px, py, pz)
    x_star = rng.uniform(-1.0, 1.0, side**3)
    b = A @ x_star
    return _finish(f"aniso3d_{side}_t{t}", A, part, t, b, x_star, {"side": side}, reorder)


def random_spd_grid(side: int, t: int, seed: int, px: int | None = None, reorder: bool = True) -> Problem:
    """Small 2D diffusion with iid log-normal cell coefficients; x* ~ U[-1,1].

    Used for tiny brute-force and invariant checks.
    """
    rng = _rng(seed)
    kappa = np.exp(rng.standard_normal((side, side)))
    A = diffusion2d(kappa)
    if px is None:
        px, py = _split2(t)
    else:
        py = t // px
    part = block_partition2d(side, side, px, py)
    x_star = rng.uniform(-1.0, 1.0, side * side)
    b = A @ x_star
    return _finish(f"rand2d_{side}_t{t}", A, part, t, b, x_star, {"side": side}, reorder)


def paper_setup_rhs(A: sp.csr_matrix, seed: int = 5489):
    """Section 5 setup: x* uniform in [0, 4), b = A x*.  (The paper draws x*
    with MATLAB's Mersenne twister; PCG64 stands in for it.)"""
    x_star = 4.0 * _rng(seed).random(A.shape[0])
    return A @ x_star, x_star


def _split2(t: int):
    table = {1: (1, 1), 2: (2, 1), 4: (2, 2), 8: (4, 2), 16: (4, 4), 32: (8, 4), 64: (8, 8)}
    if t not in table:
        raise ValueError(f"unsupported t={t}")
    return table[t]


def _split3(t: int):
    table = {1: (1, 1, 1), 2: (2, 1, 1), 4: (2, 2, 1), 8: (2, 2, 2), 16: (4, 2, 2), 32: (4, 4, 2), 64: (4, 4, 4)}
    if t not in table:
        raise ValueError(f"unsupported t={t}")
    return table[t]


def jacobi_blocks(p: Problem, nb: int) -> np.ndarray:
    """Diagonal blocks of a block Jacobi preconditioner for a grid problem:
    nb rectangular (2D) or box (3D) blocks of the grid, split like the
    subdomains (_split2 / _split3), returned in the problem's row order.

    As in Section 5 (64 blocks for every t, each subdomain the union of 64/t
    consecutive blocks), every block must lie inside one subdomain; a
    ValueError says when nb does not refine the subdomain partition.
    """
    side = int(p.meta["side"])
    perm = p.meta.get("perm", np.arange(p.n))
    if side * side == p.n:
        qx, qy = _split2(nb)
        pb = block_partition2d(side, side, qx, qy)[perm]
    elif side**3 == p.n:
        qx, qy, qz = _split3(nb)
        pb = block_partition3d(side, side, side, qx, qy, qz)[perm]
    else:
        raise ValueError("not a square or cubic grid problem")
    pb = np.ascontiguousarray(pb, dtype=np.int32)
    pairs = np.unique(pb.astype(np.int64) * p.t + p.part)
    if len(np.unique(pairs // p.t)) != len(pairs):
        raise ValueError(f"{nb} blocks do not refine the {p.t} subdomains")
    return pb


def batch_diffusion2d(count: int = 64, side_lo: int = 128, side_hi: int = 512, t: int = 8, seed: int = 4000,
                      sigma: float = 1.0) -> list[Problem]:
    """A batch of independent 2D diffusion systems of uneven size: system q
    has a side drawn uniformly from {side_lo, ..., side_hi}, iid log-normal
    cell coefficients exp(sigma * N(0, 1)), t rectangular subdomains and
    b ~ U[-1, 1].  At the defaults: 64 systems with n from 16K to 262K."""
    rng = _rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, count)
    out = []
    for q, side in enumerate(sides):
        side = int(side)
        kappa = np.exp(sigma * rng.standard_normal((side, side)))
        A = diffusion2d(kappa)
        px, py = _split2(t)
        part = block_partition2d(side, side, px, py)
        b = rng.uniform(-1.0, 1.0, side * side)
        out.append(_finish(f"batch{q}_2d_{side}_t{t}", A, part, t, b, None, {"side": side}, True))
    return out


def gaussian_field(side: int, corr: float, rng: np.random.Generator) -> np.ndarray:
    """Stationary Gaussian random field on the periodic unit square (side x
    side cells), squared-exponential covariance exp(-d^2 / (2 corr^2)),
    zero mean and unit variance, by spectral synthesis: white noise
    filtered by the square root of the covariance's spectral density."""
    k = np.fft.fftfreq(side, d=1.0 / side)  # integer wave numbers
    kx, ky = np.meshgrid(k, k, indexing="xy")
    spec = np.exp(-0.5 * (2.0 * np.pi * corr) ** 2 * (kx**2 + ky**2))
    g = np.real(np.fft.ifft2(np.fft.fft2(rng.standard_normal((side, side))) * np.sqrt(spec)))
    g -= g.mean()
    return g / g.std()


def grf_diffusion2d(side: int = 256, t: int = 16, seed: int = 5000, corr: float = 0.1, sigma: float = 1.0,
                    b_corr: float = 0.2) -> Problem:
    """2D diffusion whose coefficient is exp(sigma g), g a Gaussian random
    field with correlation length corr (unit square), and whose right-hand
    side is a smooth random field (correlation length b_corr, unit
    variance); t rectangular subdomains, rows reordered by subdomain.  The
    grid-ordered fields ride along in meta (logk, b_grid) for the warm-start
    network."""
    rng = _rng(seed)
    logk = sigma * gaussian_field(side, corr, rng)
    b = gaussian_field(side, b_corr, rng).ravel()
    A = diffusion2d(np.exp(logk))
    px, py = _split2(t)
    part = block_partition2d(side, side, px, py)
    meta = {"side": side, "logk": logk, "b_grid": b.copy()}
    return _finish(f"grf2d_{side}_t{t}", A, part, t, b, None, meta, True)


# Named workloads: the small parity case and the two large single-GPU cases.
WORKLOADS = {
    "poisson2d_64_t4": lambda seed=1001: poisson2d(64, 4, seed),
    "diffusion2d_1024_t16": lambda seed=2001: blocky_diffusion2d(1024, 16, seed=seed),
    "diffusion2d_1024_t8": lambda seed=2001: blocky_diffusion2d(1024, 8, seed=seed),
    "diffusion2d_1024_t32": lambda seed=2001: blocky_diffusion2d(1024, 32, seed=seed),
    "aniso3d_128_t16": lambda seed=3001: anisotropic_diffusion3d(128, 16, seed=seed),
}


def make(name: str, seed: int | None = None) -> Problem:
    f = WORKLOADS[name]
    return f() if seed is None else f(seed)
