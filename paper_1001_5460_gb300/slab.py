"""Slab partition of the CG solve along mode 1, for one process per GPU.

The solve of (A^T A + lambda R) x = A^T b (Sec. 4.1, Fig. 2) splits into
contiguous runs of mode-1 planes ("slabs"), one per rank:

  - K couples mode-1 planes only through G_1 (7 bands: +-3 planes) and
    lambda L_1 (+-2), so K applied to a rank's planes needs its neighbours'
    three nearest planes of p: a halo exchange of p before each application;
  - a rank applies K to its extended slab (owned planes plus halo) with a
    plan whose factor 1 is A_1 restricted to the extended slab's columns:
    (A_1[:, lo:hi])^T A_1[:, lo:hi] is exactly G_1[lo:hi, lo:hi], so the owned
    planes of the result equal the global K p there; planes in the halo
    are not used.  The same restricted factor gives the rank's part of A^T b;
  - each iteration needs two inner products over all planes, <P, Q> and
    <R, R>: FP64 partial sums all-reduced across ranks.

This module is the host logic: the partition, the halo exchange and the CG
driver.  The local operator and the vector steps are passed in, so the same
driver runs on the library's kernels (GpuSlab: the slab plan's
tca_apply_normal, tca_vec_axpby and tca_vec_dot) or on any other backend
with the same interface.  Exchanges use torch.distributed point-to-point
copies into each rank's own buffer and all-reduces (NCCL on GPUs, gloo on
CPUs); no rank reads another's memory directly.
"""
from __future__ import annotations

import dataclasses

import numpy as np

HALO = 3  # planes of p a rank needs from each neighbour (G_1 reaches +-3, L_1 +-2)


@dataclasses.dataclass(frozen=True)
class Slab:
    rank: int
    start: int  # first owned plane (global mode-1 index)
    stop: int   # one past the last owned plane
    lo: int     # first plane of the extended slab (owned planes plus halo)
    hi: int

    @property
    def owned(self) -> slice:
        """Owned planes as a slice of the extended slab's planes."""
        return slice(self.start - self.lo, self.stop - self.lo)

    @property
    def planes(self) -> int:
        return self.hi - self.lo


class SlabPartition:
    """Contiguous, balanced split of mode 1 (n1 planes) over `world` ranks."""

    def __init__(self, n1: int, world: int, halo: int = HALO):
        if world < 1 or n1 < world * halo:
            raise ValueError(f"{n1} planes cannot give {world} ranks at least {halo} planes each")
        self.n1, self.world, self.halo = int(n1), int(world), int(halo)
        base, extra = divmod(self.n1, self.world)
        starts = [r * base + min(r, extra) for r in range(self.world + 1)]
        self.slabs = [Slab(r, starts[r], starts[r + 1], max(0, starts[r] - halo), min(self.n1, starts[r + 1] + halo))
                      for r in range(self.world)]

    def slab(self, rank: int) -> Slab:
        return self.slabs[rank]

    def sends(self, rank: int):
        """(peer, slice of this rank's extended planes) it sends to each neighbour: its owned
        planes that fall in the neighbour's halo."""
        s = self.slabs[rank]
        out = []
        for peer in (rank - 1, rank + 1):
            if 0 <= peer < self.world:
                t = self.slabs[peer]
                a, b = max(s.start, t.lo), min(s.stop, t.hi)
                if a < b:
                    out.append((peer, slice(a - s.lo, b - s.lo)))
        return out

    def recvs(self, rank: int):
        """(peer, slice of this rank's extended planes) it receives from each neighbour."""
        s = self.slabs[rank]
        out = []
        for peer in (rank - 1, rank + 1):
            if 0 <= peer < self.world:
                t = self.slabs[peer]
                a, b = max(t.start, s.lo), min(t.stop, s.hi)
                if a < b:
                    out.append((peer, slice(a - s.lo, b - s.lo)))
        return out


def exchange_halo(part: SlabPartition, rank: int, v, dist=None):
    """Fill the halo planes of the extended-slab tensor v (planes on dim 0) from the neighbours'
    owned planes.  Every rank calls it; sends and receives are posted together."""
    if part.world == 1:
        return v
    if dist is None:
        import torch.distributed as dist
    ops = []
    for peer, sl in part.sends(rank):
        ops.append(dist.P2POp(dist.isend, v[sl].contiguous(), peer))
    bufs = []
    for peer, sl in part.recvs(rank):
        buf = v[sl].new_empty(v[sl].shape)
        bufs.append((sl, buf))
        ops.append(dist.P2POp(dist.irecv, buf, peer))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    for sl, buf in bufs:
        v[sl].copy_(buf)
    return v


def allreduce_sum(values, dist=None, world: int = 1):
    """Sum FP64 scalars over all ranks (one all-reduce for the list)."""
    import torch

    vals = torch.tensor(list(values), dtype=torch.float64)
    if world > 1:
        if dist is None:
            import torch.distributed as dist
        backend = dist.get_backend()
        if backend == "nccl":
            vals = vals.cuda()
        dist.all_reduce(vals)
    return [float(v) for v in vals.cpu()]


class GpuSlab:
    """A rank's slab on the GPU: the slab plan (factor 1 restricted to the extended slab's
    columns) and the library's vector kernels."""

    def __init__(self, part: SlabPartition, rank: int, factors, shape, lam: float, precision: str = "f32"):
        import torch

        from . import tca

        self.part, self.rank = part, rank
        self.slab = part.slab(rank)
        f0 = factors[0]
        self.factor0 = restrict_columns(f0, self.slab.lo, self.slab.hi)
        self.shape = (self.slab.planes,) + tuple(shape[1:])
        self.plan = tca.Plan(self.shape, [self.factor0] + list(factors[1:]), lam=lam, precision=precision)
        self.tca = tca
        self.torch = torch
        self._dot = torch.zeros(1, dtype=torch.float64, device="cuda")

    # --- backend interface of slab_cg ---
    def zeros(self):
        return self.torch.zeros(self.shape, dtype=self.torch.float32, device="cuda")

    def apply_K(self, p_ext, q_ext):
        self.plan.apply_normal(p_ext, q_ext)

    def rhs(self, b):
        """This rank's part of A^T b on the extended slab (b: the full sample tensor on the device)."""
        out = self.zeros()
        self.plan.apply_T(b, out)
        return out

    def dot(self, a, b):
        self.tca.vec_dot(a, b, self._dot)
        return float(self._dot.item())

    def axpby(self, y, x, a, b):
        self.tca.vec_axpby(y, x, a, b)


def restrict_columns(f, lo: int, hi: int):
    """Factor f (synth.Factor or tca.Factor) restricted to its columns lo..hi-1, as a tca.Factor."""
    from . import tca

    if isinstance(f, tca.Factor):
        kind = "dense" if f.kind == tca.FACTOR_DENSE else "ell4"
        a = f.values.reshape(f.m, f.n) if kind == "dense" else None
        w = f.values.reshape(f.m, 4) if kind == "ell4" else None
        col0 = f.col0
        m = f.m
    else:
        kind, a, w, col0, m = f.kind, f.a, f.w, f.col0, f.m
    if kind == "dense":
        return tca.Factor(tca.FACTOR_DENSE, m, hi - lo, np.ascontiguousarray(np.asarray(a)[:, lo:hi]))
    c0 = np.asarray(col0, dtype=np.int64) - lo
    w = np.array(w, dtype=np.float64)
    cols = c0[:, None] + np.arange(4)[None, :]
    w[(cols < 0) | (cols >= hi - lo)] = 0.0  # entries outside the slab's columns
    return tca.Factor(tca.FACTOR_ELL4, m, hi - lo, w, np.clip(c0, -(2 ** 31), 2 ** 31 - 1).astype(np.int32))


def slab_cg(part: SlabPartition, rank: int, be, rhs_ext, rtol: float = 1e-6, max_iter: int = 10000,
            dist=None, history: list | None = None):
    """CG of Fig. 2 on this rank's slab, from x = 0.

    be: backend with zeros(), apply_K(p_ext, q_ext), dot(a, b) -> float (this rank's
    partial), axpby(y, x, a, b); rhs_ext: this rank's extended-slab A^T b (only the owned
    planes are used).  Per iteration: one halo exchange of p, K on the extended slab, and
    two FP64 all-reduces (<P, Q>, then <R, R>).  Returns (x_ext, iterations, rel. residual);
    `history` (optional) receives (alpha, beta, rho) of every iteration.
    """
    s = part.slab(rank)
    own = s.owned
    world = part.world
    x = be.zeros()
    r = be.zeros()
    r[own].copy_(rhs_ext[own])
    p = be.zeros()
    q = be.zeros()
    rho, bb = allreduce_sum([be.dot(r[own], r[own]), be.dot(rhs_ext[own], rhs_ext[own])], dist, world)
    bnorm = float(np.sqrt(bb))
    p[own].copy_(r[own])
    it = 0
    rel = float(np.sqrt(rho)) / bnorm if bnorm > 0 else 0.0
    while rel > rtol and it < max_iter:
        exchange_halo(part, rank, p, dist)
        be.apply_K(p, q)
        (pq,) = allreduce_sum([be.dot(p[own], q[own])], dist, world)
        alpha = rho / pq
        be.axpby(x[own], p[own], alpha, 1.0)
        be.axpby(r[own], q[own], -alpha, 1.0)
        (rho1,) = allreduce_sum([be.dot(r[own], r[own])], dist, world)
        beta = rho1 / rho
        be.axpby(p[own], r[own], 1.0, beta)  # p = r + beta p
        if history is not None:
            history.append((alpha, beta, rho1))
        rho = rho1
        it += 1
        rel = float(np.sqrt(rho)) / bnorm
    return x, it, rel
