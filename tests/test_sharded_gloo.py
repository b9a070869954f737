"""Row-sharded enlarged CG over torch.distributed (gloo, two CPU ranks).

This is the multi-GPU decomposition of the method, checked on the CPU: each
rank owns a contiguous range of whole subdomains (the paper's
subdomain-per-processor picture, Section 1 and Section 5), its rows of A and
of every n x t block.  Per iteration of SRE-CG2 (Algorithm 1) the ranks
exchange only
  - one halo of block rows before the product A W (the neighbour rows their
    matrix rows reference), and
  - sum-allreduces of t x t and t-sized partial results: the two CGS
    coefficient blocks, the Euclidean Gram of Pre-CholQR, [W^T A W | W^T r]
    and ||r||^2,
while the t x t factorisations are computed redundantly on every rank.  The
gathered iterates must equal the single-process oracle's to rounding.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _allreduce(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _chol_upper(G):
    return np.linalg.cholesky(0.5 * (G + G.T)).T


class Shard:
    """This rank's rows [lo, hi) and the halo exchange plan."""

    def __init__(self, A, lo, hi, rank, world, bounds):
        self.lo, self.hi, self.rank, self.world = lo, hi, rank, world
        self.A = A[lo:hi]  # local rows, global columns
        cols = np.unique(self.A.indices)
        self.remote = {}  # owner -> global rows this rank needs from it
        for q in range(world):
            if q == rank:
                continue
            qlo, qhi = bounds[q]
            need = cols[(cols >= qlo) & (cols < qhi)]
            self.remote[q] = need
        # tell every owner which of its rows we need
        self.send_rows = {}
        for q in range(world):
            if q == rank:
                continue
            n_out = torch.tensor([len(self.remote[q])], dtype=torch.int64)
            n_in = torch.zeros(1, dtype=torch.int64)
            if rank < q:
                dist.send(n_out, q)
                dist.recv(n_in, q)
            else:
                dist.recv(n_in, q)
                dist.send(n_out, q)
            want = torch.from_numpy(self.remote[q].astype(np.int64))
            got = torch.zeros(int(n_in.item()), dtype=torch.int64)
            if rank < q:
                dist.send(want, q)
                dist.recv(got, q)
            else:
                dist.recv(got, q)
                dist.send(want, q)
            self.send_rows[q] = got.numpy()
        self.n_global = A.shape[0]

    def spmm(self, X_local):
        """A W for the local rows: one halo exchange of block rows."""
        w = X_local.shape[1]
        full = np.zeros((self.n_global, w))
        full[self.lo : self.hi] = X_local
        for q in sorted(self.send_rows):
            out = torch.from_numpy(np.ascontiguousarray(X_local[self.send_rows[q] - self.lo]))
            inc = torch.zeros((len(self.remote[q]), w), dtype=torch.float64)
            if self.rank < q:
                dist.send(out, q)
                dist.recv(inc, q)
            else:
                dist.recv(inc, q)
                dist.send(out, q)
            full[self.remote[q]] = inc.numpy()
        return self.A @ full


def _sharded_sre(rank, world, port, out_path, iters, trunc):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2305_19013_gb300 import workloads as W

        p = W.random_spd_grid(24, 4, seed=71)  # rows ordered subdomain by subdomain
        A = p.scipy()
        t = p.t
        # whole subdomains per rank
        sub_per_rank = t // world
        bounds = []
        for q in range(world):
            rows = np.nonzero((p.part >= q * sub_per_rank) & (p.part < (q + 1) * sub_per_rank))[0]
            bounds.append((int(rows.min()), int(rows.max()) + 1))
        lo, hi = bounds[rank]
        sh = Shard(A, lo, hi, rank, world, bounds)
        part = p.part[lo:hi]
        r = p.b[lo:hi].copy()
        x = np.zeros(hi - lo)
        rho0 = np.sqrt(_allreduce(np.array([r @ r]))[0])
        Qs, Vs = [], []
        Vprev = None
        xs = []
        for k in range(1, iters + 1):
            if k == 1:  # [T^t(r_0)]
                Wb = np.zeros((hi - lo, t))
                Wb[np.arange(hi - lo), part] = r
            else:
                Wb = Vprev.copy()
                for _ in range(2):  # CGS2: C = (AQ)^T W summed over ranks
                    Cs = [_allreduce(V.T @ Wb) for V in Vs]
                    for Q, Cm in zip(Qs, Cs):
                        Wb = Wb - Q @ Cm
            # Pre-CholQR: Euclidean Gram, then A-Gram of Q_e
            Re = _chol_upper(_allreduce(Wb.T @ Wb))
            Qe = np.linalg.solve(Re.T, Wb.T).T
            AQe = sh.spmm(Qe)
            S = _chol_upper(_allreduce(Qe.T @ AQe))
            Wk = np.linalg.solve(S.T, Qe.T).T
            Vk = np.linalg.solve(S.T, AQe.T).T
            alpha = _allreduce(Wk.T @ r)
            x = x + Wk @ alpha
            r = r - Vk @ alpha
            Qs.append(Wk)
            Vs.append(Vk)
            if trunc and len(Qs) > trunc:
                Qs.pop(0)
                Vs.pop(0)
            Vprev = Vk
            xs.append(x.copy())
        gathered = [torch.zeros(hi_ - lo_, iters, dtype=torch.float64) for (lo_, hi_) in bounds]
        dist.all_gather(gathered, torch.from_numpy(np.stack(xs, axis=1)))
        if rank == 0:
            np.save(out_path, np.concatenate([g.numpy() for g in gathered], axis=0))
        del rho0
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("trunc", [0, 2])
def test_row_sharded_sre_cg2_matches_oracle(tmp_path, trunc):
    import oracle as O
    from paper_2305_19013_gb300 import workloads as W

    iters = 12
    out = str(tmp_path / "x.npy")
    mp.start_processes(_sharded_sre, args=(2, _free_port(), out, iters, trunc), nprocs=2, join=True,
                       start_method="spawn")
    xs = np.load(out)  # n x iters, rows in global order
    p = W.random_spd_grid(24, 4, seed=71)
    o = O.ecg_solve(p.scipy(), p.part, 4, p.b, tol=0.0, maxit=iters + 1, trunc=trunc, keep_x=True)
    for k in range(iters):
        ref = o.xhist[k]
        assert np.linalg.norm(xs[:, k] - ref) <= 1e-10 * np.linalg.norm(ref), k
