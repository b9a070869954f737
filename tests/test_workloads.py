"""Pins of the synthetic input generators (CPU only)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2305_19013_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_table1_sizes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, n, nnz, dim = line.split()
        rows.append((name, int(n), int(nnz), int(dim)))
    return rows


@pytest.mark.parametrize("row", _table1(), ids=lambda r: r[0])
def test_stencil_sizes_match_table1(row):
    """Table 1: the paper's 2D matrices have n=10000, nnz=49600 and its 3D ones
    n=8000, nnz=53600 -- exactly a 100^2 5-point and a 20^3 7-point grid."""
    name, n, nnz, dim = row
    if dim == 2:
        A = W.diffusion2d(np.ones((100, 100)))
    else:
        A = W.diffusion3d(np.ones((20, 20, 20)), np.ones((20, 20, 20)), np.ones((20, 20, 20)))
    assert A.shape == (n, n)
    assert A.nnz == nnz


def test_poisson_is_classical_laplacian():
    A = W.diffusion2d(np.ones((5, 7))).toarray()
    assert np.all(np.diag(A) == 4.0)
    off = A - np.diag(np.diag(A))
    assert set(np.unique(off)) <= {0.0, -1.0}
    # interior row has 4 neighbours
    i = 2 * 7 + 3
    assert (off[i] == -1.0).sum() == 4


def test_config_nnz_closed_form():
    """Dirichlet-eliminated stencils: nnz = 5n - 4*side (2D), 7n - 6*side^2 (3D)."""
    for side in (16, 64):
        A = W.diffusion2d(np.ones((side, side)))
        assert A.nnz == 5 * side * side - 4 * side
    for side in (6, 10):
        o = np.ones((side, side, side))
        A = W.diffusion3d(o, o, o)
        assert A.nnz == 7 * side**3 - 6 * side**2


@pytest.mark.parametrize("maker", ["poisson", "blocky", "aniso", "rand"])
def test_generated_matrices_are_spd_and_symmetric(maker):
    if maker == "poisson":
        p = W.poisson2d(12, 4, seed=1)
    elif maker == "blocky":
        p = W.blocky_diffusion2d(32, 16, blocks=4, seed=2)
    elif maker == "aniso":
        p = W.anisotropic_diffusion3d(8, 16, seed=3)
    else:
        p = W.random_spd_grid(10, 4, seed=4)
    A = p.scipy()
    assert abs(A - A.T).max() == 0.0
    ev = np.linalg.eigvalsh(A.toarray())
    assert ev.min() > 0.0
    # weak diagonal dominance with strict dominance on boundary rows
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=1)).ravel() - d
    assert np.all(d >= off - 1e-12 * d)
    assert np.any(d > off + 1e-12 * d)


def test_partition_contiguous_and_balanced():
    p = W.blocky_diffusion2d(64, 16, blocks=4, seed=5)
    assert p.part.min() == 0 and p.part.max() == 15
    assert np.all(np.diff(p.part) >= 0), "rows must be ordered subdomain by subdomain"
    counts = np.bincount(p.part)
    assert np.all(counts == 64 * 64 // 16)


def test_pair_merge_is_geometrically_adjacent():
    """Halving merges {2j, 2j+1}; with the block numbering these are
    neighbouring blocks, so the merged subdomains stay connected."""
    part = W.block_partition2d(16, 16, 4, 4)
    grid = part.reshape(16, 16)
    for j in range(8):
        mask = (grid // 2) == j
        ys, xs = np.nonzero(mask)
        # merged subdomain is a rectangle
        assert mask.sum() == (ys.max() - ys.min() + 1) * (xs.max() - xs.min() + 1)


def test_reordering_is_a_symmetric_permutation():
    p0 = W.random_spd_grid(8, 4, seed=7, reorder=False)
    p1 = W.random_spd_grid(8, 4, seed=7, reorder=True)
    perm = p1.meta["perm"]
    A0, A1 = p0.scipy(), p1.scipy()
    assert abs(A0[perm][:, perm] - A1).max() == 0.0
    assert np.array_equal(p0.b[perm], p1.b)


def test_seeded_inputs_are_reproducible():
    a = W.blocky_diffusion2d(32, 8, blocks=4, seed=11)
    b = W.blocky_diffusion2d(32, 8, blocks=4, seed=11)
    c = W.blocky_diffusion2d(32, 8, blocks=4, seed=12)
    assert np.array_equal(a.val, b.val) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.b, c.b)


def test_blocky_coefficients_span_three_decades():
    p = W.blocky_diffusion2d(64, 16, blocks=16, seed=13)
    d = p.scipy().diagonal()
    assert d.max() / d.min() > 50.0


def test_manufactured_rhs():
    p = W.poisson2d(16, 4, seed=3)
    assert np.allclose(p.scipy() @ p.x_star, p.b, rtol=0, atol=1e-13)
    assert p.x_star.min() >= -1.0 and p.x_star.max() <= 1.0


@pytest.mark.parametrize("side,t,nb", [(64, 4, 16), (1024, 16, 64)])
def test_jacobi_blocks_are_rectangles_refining_the_subdomains(side, t, nb):
    """Section 5's layout: nb equal rectangular blocks of the grid, each inside
    one subdomain, each subdomain the union of nb / t blocks."""
    p = W.poisson2d(side, t, seed=1001) if side < 1024 else W.make("diffusion2d_1024_t16")
    pb = W.jacobi_blocks(p, nb)
    assert pb.shape == (p.n,) and pb.dtype == np.int32
    sizes = np.bincount(pb, minlength=nb)
    assert len(sizes) == nb and np.all(sizes == p.n // nb)
    cell = np.asarray(p.meta.get("perm", np.arange(p.n)))  # grid cell of each row
    y, x = np.divmod(cell, side)
    owners = np.empty(nb, dtype=np.int64)
    for b in range(nb):
        rows = pb == b
        assert len(np.unique(p.part[rows])) == 1
        owners[b] = p.part[rows][0]
        h = y[rows].max() - y[rows].min() + 1
        w = x[rows].max() - x[rows].min() + 1
        assert h * w == sizes[b]  # a full rectangle of cells
    assert np.all(np.bincount(owners, minlength=t) == nb // t)


@pytest.mark.parametrize("nb", [2, 4])
def test_jacobi_blocks_reject_a_partition_that_does_not_refine_the_subdomains(nb):
    # the 64^2 Poisson problem has 4 row-strip subdomains; with 2 or 4 blocks
    # some block holds rows of more than one strip
    p = W.poisson2d(64, 4, seed=1001)
    with pytest.raises(ValueError):
        W.jacobi_blocks(p, nb)
