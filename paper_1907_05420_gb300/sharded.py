"""Algorithm 1 (Sec. 4.2) over processes, one GPU each.

The N periods are split into contiguous shards, one per process (Algorithm 1:
the blocks are distributed evenly).  Process p holds the arrowhead system of
its own blocks and of the coupling columns they touch, c0_p .. c0_p + nc_p - 1
(re-indexed from 0); the root (rank 0) holds every coupling column, C and
r_g, the other processes a zero C and a zero r_g.  Then:

  every p   factor its blocks and form S_p = C_p - sum_{i in p} B_i^T A_i^{-1} B_i
  reduce    the root adds every S_p into the window (c0_p, c0_p) of its S
  root      factor S = L_s D_s L_s^T
  every p   t_p = r_g,p - sum_{i in p} B_i^T A_i^{-1} r_i
  reduce    the root adds every t_p into the window c0_p of its t
  root      x_g = S^{-1} t, broadcast to every process
  every p   x_i = A_i^{-1} (r_i - B_i x_g) with its window of x_g

With the adjacent-period coupling a shard of periods lo..hi-1 touches the
coupling columns of periods lo-1..hi-1, so the windows of neighbouring shards
overlap in one period's storage columns and the reduce is a gather of banded
windows.  FP64 refinement on the distributed K repeats the solve on the
residual r - K x: its block rows are local, its coupling rows are the sum of
every process's part (reduced like t), and the normwise backward error
eta = ||r - Kx||_inf / (||K||_inf ||x||_inf + ||r||_inf) takes maxima over
processes.

The arithmetic runs in a backend per process: ``GpuShard`` calls the C ABI
(include/kkt_schur.h, "the steps of Algorithm 1 one at a time"); any object
with the same methods can stand in (the CPU tests use the oracle).  The
collectives go through a ``comm`` object: ``TorchComm`` uses
torch.distributed point-to-point sends for the reduce, a broadcast for x_g
and an all-reduce for the norms.
"""
from __future__ import annotations

import types

import numpy as np


def partition(N: int, world: int) -> list[tuple[int, int]]:
    """Contiguous period ranges [lo, hi) of the `world` processes; sizes differ
    by at most one (the first processes take the extra periods)."""
    if world < 1 or N < world:
        raise ValueError(f"cannot split {N} periods over {world} processes")
    q, r = divmod(N, world)
    out, lo = [], 0
    for p in range(world):
        hi = lo + q + (1 if p < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


def coupling_window(prob, lo: int, hi: int, root: bool) -> tuple[int, int]:
    """(c0, nc): the coupling columns that blocks lo..hi-1 touch (all of them
    on the root)."""
    if root:
        return 0, int(prob.nC)
    bp = np.asarray(prob.b_blockptr)
    cols = np.asarray(prob.b_col)[bp[lo]:bp[hi]]
    if cols.size == 0:
        return 0, 0
    return int(cols.min()), int(cols.max()) - int(cols.min()) + 1


def shard_of(prob, lo: int, hi: int, root: bool):
    """The arrowhead system of blocks lo..hi-1 and their coupling window (a
    view of the problem's pattern and values; no arithmetic)."""
    c0, nc = coupling_window(prob, lo, hi, root)
    N = hi - lo
    bp = np.asarray(prob.b_blockptr, dtype=np.int64)
    e0, e1 = int(bp[lo]), int(bp[hi])
    a_vals = np.ascontiguousarray(np.asarray(prob.a_vals).reshape(prob.N, -1)[lo:hi])
    rhs = np.asarray(prob.rhs)
    nb = prob.N * prob.nA
    r_local = np.concatenate([rhs[lo * prob.nA:hi * prob.nA],
                              rhs[nb:nb + prob.nC] if root else np.zeros(nc)])
    if root:
        c_kind, c_vals = int(prob.c_kind), np.ascontiguousarray(prob.c_vals, dtype=np.float64)
    else:
        c_kind, c_vals = 0, np.zeros(nc)
    return types.SimpleNamespace(
        N=N, nA=int(prob.nA), nP=int(prob.nP), nC=nc, nK=N * int(prob.nA) + nc,
        a_rowptr=np.asarray(prob.a_rowptr, dtype=np.int32), a_col=np.asarray(prob.a_col, dtype=np.int32),
        a_vals=a_vals, b_blockptr=(bp[lo:hi + 1] - e0).astype(np.int32),
        b_row=np.ascontiguousarray(np.asarray(prob.b_row, dtype=np.int32)[e0:e1]),
        b_col=np.ascontiguousarray(np.asarray(prob.b_col, dtype=np.int32)[e0:e1] - c0),
        b_vals=np.ascontiguousarray(np.asarray(prob.b_vals, dtype=np.float64)[e0:e1]),
        c_kind=c_kind, c_vals=c_vals, rhs=r_local, c0=c0, lo=lo, hi=hi, root=root, nC_global=int(prob.nC))


class TorchComm:
    """The collectives of Algorithm 1 over torch.distributed (NCCL for CUDA
    tensors, gloo for CPU tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def send(self, t, dst):
        self.dist.send(t, dst, group=self.group)

    def recv(self, t, src):
        self.dist.recv(t, src, group=self.group)

    def broadcast(self, t, src):
        self.dist.broadcast(t, src, group=self.group)

    def allreduce_max(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)


class ShardedSolver:
    """One process's part of the sharded Schur-complement solve.

    prob: the whole system's pattern and values (every process reads the
    pattern; each takes its own blocks' values); backend(sub) builds this
    process's backend for its shard; comm: a TorchComm or equivalent."""

    def __init__(self, prob, backend, comm):
        self.comm = comm
        self.world, self.rank = comm.world, comm.rank
        self.parts = partition(int(prob.N), self.world)
        self.windows = [coupling_window(prob, lo, hi, p == 0) for p, (lo, hi) in enumerate(self.parts)]
        lo, hi = self.parts[self.rank]
        self.sub = shard_of(prob, lo, hi, self.rank == 0)
        self.be = backend(self.sub)
        self.nb = self.sub.N * self.sub.nA
        self.nc = self.sub.nC
        self.knorm = None

    # the reduce of Algorithm 1: the root adds every other process's part
    def _reduce_vec(self, v, off):
        """v: this process's vector; its coupling part v[off:off+nc] is added
        into the root's at the sender's window."""
        if self.rank == 0:
            for p in range(1, self.world):
                c0, nc = self.windows[p]
                if nc == 0:
                    continue
                buf = self.be.empty(nc)
                self.comm.recv(buf, p)
                self.be.add_vec(v, off + c0, buf)
        elif self.nc > 0:
            self.comm.send(self.be.slice(v, off, self.nc), 0)

    def factor(self, a_vals=None, b_vals=None, c_vals=None):
        """Block factors, the reduce of S, the root's factor of S, and ||K||_inf.
        Values default to the shard's own (host arrays)."""
        sub = self.sub
        self.be.factor(sub.a_vals if a_vals is None else a_vals, sub.b_vals if b_vals is None else b_vals,
                       sub.c_vals if c_vals is None else c_vals)
        if self.rank == 0:
            for p in range(1, self.world):
                c0, nc = self.windows[p]
                if nc == 0:
                    continue
                buf = self.be.empty(nc * nc)
                self.comm.recv(buf, p)
                self.be.add_schur(buf, c0, nc)
            self.be.factor_schur()
        elif self.nc > 0:
            self.comm.send(self.be.schur_part(), 0)
        # ||K||_inf: block rows are local; coupling rows add up over processes
        rs = self.be.rowsums()
        self._reduce_vec(rs, self.nb)
        m = self.be.norm(rs, 0, self.nb + (self.nc if self.rank == 0 else 0))
        self.knorm = self._max([m])[0]

    def _max(self, vals):
        t = self.be.host_tensor(vals)
        self.comm.allreduce_max(t)
        return [float(v) for v in self.be.to_list(t)]

    def apply(self, r):
        """x = K~^{-1} r for this process's part r (its block rows, and r_g on
        the root; the other processes' coupling part is ignored)."""
        t = self.be.front(r)
        if self.rank == 0:
            self._reduce_vec(t, 0)
            xg = self.be.coupling_solve(t)
        else:
            self._reduce_vec(t, 0)
            xg = self.be.empty(self.sub.nC_global)
        self.comm.broadcast(xg, 0)
        return self.be.back(xg, self.sub.c0, self.nc)

    def solve(self, r=None, tol=1e-10, max_refine=10):
        """Refined solve; returns (x of this process, eta, refinement steps).

        x holds this process's block rows and its window of x_g."""
        r = self.be.upload(self.sub.rhs) if r is None else r
        own = self.nb + (self.nc if self.rank == 0 else 0)  # the rows this process reports
        x = self.apply(r)
        steps, eta, eta_prev = 0, float("inf"), float("inf")
        rnorm = None
        while True:
            rho = self.be.residual(r, x)
            self._reduce_vec(rho, self.nb)
            if self.rank != 0:
                self.be.zero_tail(rho, self.nb)  # r_g,p = 0 off the root
            if rnorm is None:
                rnorm = self.be.norm(r, 0, own)
            nr, nx = self.be.norm(rho, 0, own), self.be.norm(x, 0, own)
            nr, nx, nrr = self._max([nr, nx, rnorm])
            if not (np.isfinite(nr) and np.isfinite(nx) and np.isfinite(nrr) and np.isfinite(self.knorm)):
                return x, float("nan"), steps
            eta = 0.0 if nr == 0.0 else nr / (self.knorm * nx + nrr)
            if eta <= tol or steps >= max_refine or (steps > 0 and not eta < 0.5 * eta_prev):
                return x, eta, steps
            eta_prev = eta
            dx = self.apply(rho)
            self.be.add_vec(x, 0, dx)
            steps += 1


def solve_in_process(prob, nshards, backend, tol=1e-10, max_refine=10):
    """The data flow of ShardedSolver for `nshards` shards held by one process
    (one GPU): the reduce and the broadcast become direct additions into the
    root's buffers.  Returns (x of the whole system as a host array, eta,
    steps)."""
    parts = partition(int(prob.N), nshards)
    subs = [shard_of(prob, lo, hi, p == 0) for p, (lo, hi) in enumerate(parts)]
    bes = [backend(s) for s in subs]
    root = bes[0]
    nbs = [s.N * s.nA for s in subs]
    for be, s in zip(bes, subs):
        be.factor(s.a_vals, s.b_vals, s.c_vals)
    for be, s in zip(bes[1:], subs[1:]):
        if s.nC:
            root.add_schur(be.schur_part(), s.c0, s.nC)
    root.factor_schur()

    def reduce_tail(vs, off0):
        for be, s, v, nb in zip(bes[1:], subs[1:], vs[1:], nbs[1:]):
            if s.nC:
                root.add_vec(vs[0], off0 + s.c0, be.slice(v, nb if off0 else 0, s.nC))

    rs = [be.rowsums() for be in bes]
    reduce_tail(rs, nbs[0])
    knorm = max(be.norm(v, 0, nb + (s.nC if i == 0 else 0))
                for i, (be, v, nb, s) in enumerate(zip(bes, rs, nbs, subs)))

    def apply(rr):
        ts = [be.front(v) for be, v in zip(bes, rr)]
        for be, s, t in zip(bes[1:], subs[1:], ts[1:]):
            if s.nC:
                root.add_vec(ts[0], s.c0, be.slice(t, 0, s.nC))
        xg = root.coupling_solve(ts[0])
        return [be.back(be.copy_from(xg, root), s.c0, s.nC) for be, s in zip(bes, subs)]

    r = [be.upload(s.rhs) for be, s in zip(bes, subs)]
    own = [nb + (s.nC if i == 0 else 0) for i, (nb, s) in enumerate(zip(nbs, subs))]
    x = apply(r)
    rnorm = max(be.norm(v, 0, o) for be, v, o in zip(bes, r, own))
    steps, eta_prev = 0, float("inf")
    while True:
        rho = [be.residual(v, xv) for be, v, xv in zip(bes, r, x)]
        for be, s, v, nb in zip(bes[1:], subs[1:], rho[1:], nbs[1:]):
            if s.nC:
                root.add_vec(rho[0], nbs[0] + s.c0, be.slice(v, nb, s.nC))
                be.zero_tail(v, nb)
        nr = max(be.norm(v, 0, o) for be, v, o in zip(bes, rho, own))
        nx = max(be.norm(v, 0, o) for be, v, o in zip(bes, x, own))
        eta = 0.0 if nr == 0.0 else nr / (knorm * nx + rnorm)
        if not np.isfinite(eta) or eta <= tol or steps >= max_refine or (steps > 0 and not eta < 0.5 * eta_prev):
            break
        eta_prev = eta
        dx = apply(rho)
        for be, xv, d in zip(bes, x, dx):
            be.add_vec(xv, 0, d)
        steps += 1
    # the whole x: every shard's block rows, then the root's x_g
    xs = [be.download(v) for be, v in zip(bes, x)]
    out = np.concatenate([xv[:nb] for xv, nb in zip(xs, nbs)] + [xs[0][nbs[0]:]])
    return out, eta, steps


class GpuShard:
    """A process's blocks on its GPU, through the C ABI (binding.py)."""

    def __init__(self, sub, opt=None, device=None):
        import torch

        from . import binding as B

        self.B, self.torch = B, torch
        self.dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.sub = sub
        self.h = B.kkt_analyze(sub, opt)
        self.nb = sub.N * sub.nA

    def close(self):
        if self.h:
            self.B.kkt_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass

    # buffers
    def empty(self, n):
        return self.torch.empty(int(n), dtype=self.torch.float64, device=self.dev)

    def upload(self, arr):
        return self.torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)).to(self.dev)

    def download(self, t):
        return t.cpu().numpy()

    def host_tensor(self, vals):
        return self.torch.tensor(vals, dtype=self.torch.float64, device=self.dev)

    def to_list(self, t):
        return t.cpu().tolist()

    def slice(self, v, off, n):
        return v[off:off + n]

    def copy_from(self, v, other):
        return v if other is self or v.device == self.dev else v.to(self.dev)

    def zero_tail(self, v, off):
        v[off:].zero_()

    # steps
    def factor(self, a, b, c):
        self.B.kkt_factor_blocks(self.h, np.ascontiguousarray(a), np.ascontiguousarray(b), np.ascontiguousarray(c))

    def schur_part(self):
        n = self.sub.nC
        out = self.empty(n * n)
        ptr, ld = self.B.kkt_schur_matrix(self.h)
        src = _DevView(ptr, n * n)
        self.B.kkt_accumulate(out.zero_(), n * n, src, n * n, n * n, 1)
        return out

    def add_schur(self, part, c0, nc):
        ptr, ld = self.B.kkt_schur_matrix(self.h)
        self.B.kkt_accumulate(ptr + 8 * (c0 + c0 * ld), ld, part, nc, nc, nc)

    def factor_schur(self):
        self.B.kkt_factor_schur(self.h)

    def add_vec(self, dst, off, src):
        n = src.numel()
        self.B.kkt_accumulate(dst.data_ptr() + 8 * off, n, src, n, n, 1)

    def front(self, r):
        t = self.empty(max(1, self.sub.nC))
        self.B.kkt_solve_front(self.h, r, t)
        return t[:self.sub.nC]

    def coupling_solve(self, t):
        xg = self.empty(max(1, self.sub.nC))
        self.B.kkt_solve_coupling(self.h, t.contiguous(), xg)
        return xg[:self.sub.nC]

    def back(self, xg, c0, nc):
        x = self.empty(self.nb + nc)
        w = xg[c0:c0 + nc].contiguous() if nc else self.empty(1)
        self.B.kkt_solve_back(self.h, w, x)
        return x

    def residual(self, r, x):
        rho = self.empty(self.nb + self.sub.nC)
        self.B.kkt_residual(self.h, r, x, rho)
        return rho

    def rowsums(self):
        out = self.empty(self.nb + self.sub.nC)
        self.B.kkt_abs_rowsums(self.h, out)
        return out

    def norm(self, v, off, n):
        return self.B.kkt_norm_inf(self.h, v[off:off + n].contiguous(), n) if n > 0 else 0.0


class _DevView:
    """A device address with the tensor interface the binding reads (no copy)."""

    is_cuda = True

    def __init__(self, ptr, n):
        self._p, self._n = ptr, n

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return self._p

    def numel(self):
        return self._n
