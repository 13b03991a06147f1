"""The sharded form of Algorithm 1 (Sec. 4.2) on CPU ranks (gloo).

paper_1907_05420_gb300/sharded.py splits the periods over processes, reduces
the local Schur complements and right-hand-side parts to the root, factors S
there, broadcasts x_g and refines on the distributed K.  Here every process's
arithmetic is the oracle's (OracleShard below, the stand-in for the GPU
kernels), so the test checks the partition, the coupling windows and the
collectives: the root's reduced S and t equal the single-process oracle's,
and the gathered solution equals the oracle's solution within the parity
bound 10 kappa(K) max(eta, eps), with eta <= 1e-10.
"""
import os
import pickle
import socket

import numpy as np
import pytest

import oracle
from gen import CONFIGS, make_problem, make_scopf
from tests.kkt_dense import b_dense, dense_K

EPS = np.finfo(np.float64).eps


class OracleShard:
    """The backend interface of ShardedSolver with the oracle's FP64 CPU
    arithmetic on CPU tensors."""

    def __init__(self, sub):
        import torch

        self.torch, self.sub = torch, sub
        self.nb = sub.N * sub.nA
        self.perm = oracle.min_degree(sub.nA, sub.a_rowptr, sub.a_col, sub.nP)
        self.B = [b_dense(sub, i) for i in range(sub.N)]
        self.S_reduced = None
        self.t_first = None

    def _t(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))

    # buffers
    def empty(self, n):
        return self.torch.zeros(int(n), dtype=self.torch.float64)

    def upload(self, a):
        return self._t(np.array(a, dtype=np.float64, copy=True))

    def download(self, t):
        return t.numpy()

    def host_tensor(self, vals):
        return self.torch.tensor(vals, dtype=self.torch.float64)

    def to_list(self, t):
        return t.tolist()

    def slice(self, v, off, n):
        return v[off:off + n]

    def copy_from(self, v, other):
        return v

    def zero_tail(self, v, off):
        v[off:] = 0.0

    def _solve(self, i, b):
        s = self.sub
        return oracle.sparse_solve(s.nA, s.a_rowptr, s.a_col, s.a_vals[i], self.perm, b)

    # steps
    def factor(self, a, b, c):
        s = self.sub
        S = np.diag(s.c_vals) if s.c_kind == 0 else np.array(s.c_vals, dtype=np.float64).reshape(s.nC, s.nC)
        S = S.astype(np.float64)
        for i in range(s.N):
            Bi = self.B[i]
            for c_ in np.nonzero(np.any(Bi != 0.0, axis=0))[0]:
                y = self._solve(i, Bi[:, c_])
                S[:, c_] -= Bi.T @ y
        self.S = S

    def schur_part(self):
        return self._t(self.S.T.reshape(-1).copy())

    def add_schur(self, part, c0, nc):
        self.S[c0:c0 + nc, c0:c0 + nc] += part.numpy().reshape(nc, nc).T

    def factor_schur(self):
        self.S_reduced = self.S.copy()
        self.F, _ = oracle.dense_ldlt(self.S)

    def add_vec(self, dst, off, src):
        dst[off:off + src.numel()] += src

    def front(self, r):
        s, rr = self.sub, r.numpy()
        t = rr[self.nb:].copy()
        for i in range(s.N):
            y = self._solve(i, rr[i * s.nA:(i + 1) * s.nA])
            t -= self.B[i].T @ y
        self._r = rr.copy()
        return self._t(t)

    def coupling_solve(self, t):
        if self.t_first is None:
            self.t_first = t.numpy().copy()
        return self._t(oracle.dense_ldlt_solve(self.F, t.numpy()))

    def back(self, xg, c0, nc):
        s = self.sub
        w = xg.numpy()[c0:c0 + nc]
        x = np.empty(self.nb + nc)
        for i in range(s.N):
            x[i * s.nA:(i + 1) * s.nA] = self._solve(i, self._r[i * s.nA:(i + 1) * s.nA] - self.B[i] @ w)
        x[self.nb:] = w
        return self._t(x)

    def residual(self, r, x):
        return self._t(r.numpy() - oracle.kkt_matvec(self.sub, x.numpy()))

    def rowsums(self):
        return self._t(np.abs(dense_K(self.sub)).sum(axis=1))

    def norm(self, v, off, n):
        return float(np.max(np.abs(v.numpy()[off:off + n]))) if n > 0 else 0.0


PROBLEMS = {
    "small": lambda: make_problem(CONFIGS["small"]),
    "grid30_n24": lambda: make_problem(CONFIGS["grid30_n24"]),
    "grid30_n24_paper": lambda: make_problem(CONFIGS["grid30_n24"], coupling="paper"),
    "scopf_small": lambda: make_scopf(CONFIGS["small"], 3),
}


def _worker(rank, world, port, name, out_dir):
    import torch.distributed as dist

    from paper_1907_05420_gb300.sharded import ShardedSolver, TorchComm

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        p = PROBLEMS[name]()
        solver = ShardedSolver(p, OracleShard, TorchComm())
        solver.factor()
        x, eta, steps = solver.solve()
        res = {"rank": rank, "x": x.numpy().copy(), "lo": solver.sub.lo, "hi": solver.sub.hi,
               "c0": solver.sub.c0, "nc": solver.sub.nC, "eta": eta, "steps": steps, "knorm": solver.knorm}
        if rank == 0:
            res["S"] = solver.be.S_reduced
            res["t"] = solver.be.t_first
        with open(os.path.join(out_dir, f"r{rank}.pkl"), "wb") as f:
            pickle.dump(res, f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(name, world, tmp_path):
    import torch.multiprocessing as mp

    mp.start_processes(_worker, args=(world, _free_port(), name, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    return [pickle.load(open(tmp_path / f"r{r}.pkl", "rb")) for r in range(world)]


@pytest.mark.parametrize("name,world", [("small", 2), ("grid30_n24", 2), ("grid30_n24", 3),
                                        ("grid30_n24_paper", 2), ("scopf_small", 2)])
def test_sharded_solve_matches_single_process_oracle(name, world, tmp_path):
    pytest.importorskip("torch")
    p = PROBLEMS[name]()
    ref = oracle.kkt_solve(p, want_S=True)
    res = _run(name, world, tmp_path)
    # partition: contiguous, covering every period once
    assert [r["lo"] for r in res] == [0] + [r["hi"] for r in res[:-1]] and res[-1]["hi"] == p.N
    # the reduced S and t on the root equal the single-process ones
    root = res[0]
    scale = np.max(np.abs(ref["S"]))
    assert np.max(np.abs(root["S"] - ref["S"])) <= 1e-12 * scale
    assert np.max(np.abs(root["t"] - ref["t"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["t"])))
    # ||K||_inf over the processes equals the whole system's
    assert root["knorm"] == pytest.approx(oracle.kkt_norm_inf(p), rel=1e-14)
    # the gathered solution: every shard's block rows, then x_g from the root
    x = np.concatenate([r["x"][:(r["hi"] - r["lo"]) * p.nA] for r in res] + [root["x"][(root["hi"] - root["lo"]) * p.nA:]])
    for r in res[1:]:  # each process's window of x_g is the root's
        nb = (r["hi"] - r["lo"]) * p.nA
        assert np.array_equal(r["x"][nb:], x[p.N * p.nA + r["c0"]:p.N * p.nA + r["c0"] + r["nc"]])
    eta = oracle.backward_error(p, x)
    assert eta <= 1e-10
    assert all(r["eta"] == res[0]["eta"] for r in res)  # every process takes the same decision
    kappa = np.linalg.cond(dense_K(p))
    err = np.max(np.abs(x - ref["x"])) / np.max(np.abs(ref["x"]))
    assert err <= 10 * kappa * max(eta, oracle.backward_error(p, ref["x"]), EPS), err


def test_partition_and_windows():
    from paper_1907_05420_gb300.sharded import coupling_window, partition, shard_of

    assert partition(24, 5) == [(0, 5), (5, 10), (10, 15), (15, 20), (20, 24)]
    with pytest.raises(ValueError):
        partition(3, 4)
    p = make_problem(CONFIGS["grid30_n24"])
    ns = p.nC // p.N
    # adjacent coupling: periods lo..hi-1 touch the storage columns of periods lo-1..hi-1
    assert coupling_window(p, 8, 16, False) == (7 * ns, 9 * ns)
    assert coupling_window(p, 0, 8, False) == (0, 8 * ns)
    assert coupling_window(p, 0, 8, True) == (0, p.nC)
    sub = shard_of(p, 8, 16, False)
    assert sub.N == 8 and sub.nC == 9 * ns and sub.b_col.min() >= 0 and sub.b_col.max() < sub.nC
    assert np.all(sub.c_vals == 0.0) and np.all(sub.rhs[sub.N * sub.nA:] == 0.0)
    assert np.array_equal(sub.a_vals, np.asarray(p.a_vals)[8:16])
