"""Slab partition of the solve along mode 1: partition, halo exchange and the distributed CG
driver on CPU ranks (gloo, world size 2 and 3), against the single-rank run and the oracle.

The ranks apply K to their extended slabs with the oracle (FP64, the long way through sample
space, embedded in the global tensor); what is under test is the host logic of
paper_1001_5460_gb300.slab: which planes each rank owns and exchanges, and that the
all-reduced CG scalars and the assembled solution equal the single-rank run's.
"""
import os
import socket

import numpy as np
import pytest
import torch

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import slab, synth

SHAPE = (23, 9, 8, 4)


def _problem():
    inst = synth.instance_bspline(SHAPE, seed=61, lam=2e-2, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    return inst, mats, b


class OracleSlab:
    """CPU backend: K of the extended slab through the oracle on the global tensor."""

    def __init__(self, part, rank, mats, lam):
        self.s = part.slab(rank)
        self.mats, self.lam = mats, lam
        self.shape = (self.s.planes,) + SHAPE[1:]

    def zeros(self):
        return torch.zeros(self.shape, dtype=torch.float64)

    def apply_K(self, p_ext, q_ext):
        g = np.zeros(SHAPE)
        g[self.s.lo:self.s.hi] = p_ext.numpy()
        q_ext.copy_(torch.from_numpy(O.normal_apply(g, self.mats, self.lam)[self.s.lo:self.s.hi]))

    def dot(self, a, b):
        return float(torch.dot(a.reshape(-1), b.reshape(-1)))

    def axpby(self, y, x, a, b):
        y.mul_(b).add_(x, alpha=a)


@pytest.mark.parametrize("n1,world", [(23, 2), (23, 3), (9, 3), (40, 4)])
def test_partition_covers_mode_1_and_halos_match(n1, world):
    part = slab.SlabPartition(n1, world)
    owned = np.concatenate([np.arange(s.start, s.stop) for s in part.slabs])
    np.testing.assert_array_equal(owned, np.arange(n1))  # disjoint, in order, complete
    for r, s in enumerate(part.slabs):
        assert s.lo == max(0, s.start - slab.HALO) and s.hi == min(n1, s.stop + slab.HALO)
        assert s.stop - s.start >= slab.HALO
        # What r receives from a neighbour is exactly what that neighbour sends to r, in
        # global plane numbers, and together with r's owned planes it fills r's extended slab.
        got = set(range(s.start, s.stop))
        for peer, sl in part.recvs(r):
            t = part.slab(peer)
            sent = [sl2 for p2, sl2 in part.sends(peer) if p2 == r]
            assert len(sent) == 1
            g_recv = range(s.lo + sl.start, s.lo + sl.stop)
            g_sent = range(t.lo + sent[0].start, t.lo + sent[0].stop)
            assert list(g_recv) == list(g_sent)
            got |= set(g_recv)
        assert got == set(range(s.lo, s.hi))
    with pytest.raises(ValueError):
        slab.SlabPartition(5, 2)  # fewer than HALO planes per rank


def test_restricted_factor_gives_the_gram_rows_of_the_slab():
    """(A_1[:, lo:hi])^T A_1[:, lo:hi] = G_1[lo:hi, lo:hi] (plain matrix algebra), and the
    ELL-4 restriction keeps exactly the entries inside the slab's columns."""
    from paper_1001_5460_gb300 import tca  # noqa: F401  (restrict_columns builds tca.Factor)

    inst, mats, _ = _problem()
    a = mats[0]
    for lo, hi in ((0, 11), (5, 17), (12, 23)):
        f = slab.restrict_columns(inst.factors[0], lo, hi)
        dense = synth.ell4_to_dense(f.col0, f.values, hi - lo)
        np.testing.assert_array_equal(dense, a[:, lo:hi])
        np.testing.assert_allclose(dense.T @ dense, (a.T @ a)[lo:hi, lo:hi], rtol=1e-14, atol=1e-15)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, iters):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst, mats, b = _problem()
        part = slab.SlabPartition(SHAPE[0], world)
        s = part.slab(rank)
        be = OracleSlab(part, rank, mats, inst.lam)
        # Halo exchange: fill a vector's owned planes from the global one, exchange, compare.
        g = np.random.default_rng(5).standard_normal(SHAPE)
        v = torch.zeros(be.shape, dtype=torch.float64)
        v[s.owned] = torch.from_numpy(g[s.start:s.stop])
        slab.exchange_halo(part, rank, v)
        np.testing.assert_array_equal(v.numpy(), g[s.lo:s.hi])
        rhs = O.apply_T(b, mats)
        rhs_ext = torch.from_numpy(np.ascontiguousarray(rhs[s.lo:s.hi]))
        hist = []
        x, it, rel = slab.slab_cg(part, rank, be, rhs_ext, rtol=0.0, max_iter=iters, history=hist)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), x=x[s.owned].numpy(), start=s.start, stop=s.stop,
                 hist=np.array(hist), it=it)
    finally:
        dist.destroy_process_group()


def _run(world, tmp_path, iters):
    import torch.multiprocessing as mp

    if world == 1:
        inst, mats, b = _problem()
        part = slab.SlabPartition(SHAPE[0], 1)
        be = OracleSlab(part, 0, mats, inst.lam)
        hist = []
        x, it, rel = slab.slab_cg(part, 0, be, torch.from_numpy(O.apply_T(b, mats)), rtol=0.0, max_iter=iters,
                                  history=hist)
        return x.numpy(), np.array(hist)
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), iters), nprocs=world,
                       start_method="spawn", join=True)
    x = np.zeros(SHAPE)
    hists = []
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        x[int(d["start"]):int(d["stop"])] = d["x"]
        hists.append(d["hist"])
    for h in hists[1:]:
        np.testing.assert_array_equal(h, hists[0])  # every rank holds the same all-reduced scalars
    return x, hists[0]


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_cg_equals_single_rank_and_oracle(world, tmp_path):
    iters = 12
    x1, h1 = _run(1, tmp_path, iters)
    xw, hw = _run(world, tmp_path, iters)
    # The scalars are sums of the same FP64 terms grouped by rank: equal to rounding.
    np.testing.assert_allclose(hw, h1, rtol=1e-10)
    np.testing.assert_allclose(xw, x1, rtol=1e-10, atol=1e-12)
    # And both are the oracle's CG iterate (Fig. 2).
    inst, mats, b = _problem()
    ref = O.cg(lambda v: O.normal_apply(v, mats, inst.lam), O.apply_T(b, mats), rtol=0.0, max_iter=iters).x
    np.testing.assert_allclose(xw, ref, rtol=1e-9, atol=1e-11)
