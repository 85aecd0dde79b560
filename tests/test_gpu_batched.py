"""Batched solves in one graph launch and the fused-sweep autotuner, against the FP64 oracle.

The batch mixes 3D and 4D instances, dense and B-spline factors and per-instance
lambda (the uneven-instance generator at reduced sizes so that the oracle's
solves take seconds).  Every instance must reach the stated true relative
residual, measured by the oracle in FP64, and agree with the oracle's own CG
solution.
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import TOL_F32, empty_dev, lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _batch(count, base_seed, lo=8, hi=28):
    insts, bs = [], []
    for i in range(count):
        inst = synth.instance_batched(i, base_seed=base_seed, lo=lo, hi=hi)
        mats = [f.dense() for f in inst.factors]
        b = O.apply(inst.x_true.astype(np.float64), mats) + inst.noise
        insts.append(inst)
        bs.append(b.astype(np.float32))
    return insts, bs


@pytest.mark.parametrize("count,check_every", [(8, 16), (5, 2)])
def test_solve_batched_matches_oracle(count, check_every):
    tca = lib()
    need_cuda()
    insts, bs = _batch(count, 300 + count)
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bd = [to_dev(b, np.float32) for b in bs]
    xs = [empty_dev(inst.shape, np.float32) for inst in insts]
    st, infos = tca.solve_batched(plans, bd, xs, rtol=1e-6, max_iter=20000, check_every=check_every)
    assert st == tca.OK, infos
    for inst, b, x, info in zip(insts, bs, xs, infos):
        mats = [f.dense() for f in inst.factors]
        got = x.cpu().numpy()
        rel = O.rel_residual(got, b.astype(np.float64), mats, inst.lam)
        assert rel <= 1.5e-6, (inst.shape, rel, info)
        assert abs(info["rel_res_true"] - rel) < 1e-7, (rel, info)
        ref = O.solve(b.astype(np.float64), mats, inst.lam, rtol=1e-12).x
        assert rel_l2(got, ref) < 1e-3, inst.shape
    # A second call replays the cached graphs and gives the same iterates.
    first = [x.clone() for x in xs]
    st2, infos2 = tca.solve_batched(plans, bd, xs, rtol=1e-6, max_iter=20000, check_every=check_every)
    assert st2 == tca.OK
    for a, b_, i1, i2 in zip(first, xs, infos, infos2):
        assert i1["iters"] == i2["iters"]
        assert bool((a == b_).all())


def test_solve_batched_equals_single_solves():
    """One instance per branch runs the same kernels as tca_solve: identical iteration counts."""
    tca = lib()
    insts, bs = _batch(4, 410)
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bd = [to_dev(b, np.float32) for b in bs]
    xs = [empty_dev(inst.shape, np.float32) for inst in insts]
    st, infos = tca.solve_batched(plans, bd, xs, rtol=1e-6, max_iter=20000, check_every=8)
    assert st == tca.OK
    for plan, b, x, info in zip(plans, bd, xs, infos):
        y = empty_dev(x.shape, np.float32)
        st1, info1 = plan.solve(b, y, rtol=1e-6, max_iter=20000, check_every=8)
        assert st1 == tca.OK
        assert info1["iters"] == info["iters"]
        assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-6


def test_solve_batched_zero_rhs_and_max_iter():
    tca = lib()
    torch = need_cuda()
    insts, bs = _batch(3, 520)
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bd = [to_dev(b, np.float32) for b in bs]
    bd[1] = torch.zeros_like(bd[1])
    xs = [empty_dev(inst.shape, np.float32) for inst in insts]
    st, infos = tca.solve_batched(plans, bd, xs, rtol=1e-6, max_iter=3, check_every=2, raise_on_error=False)
    assert st == tca.ERR_NOT_CONVERGED
    assert infos[1]["iters"] == 0 and infos[1]["rel_res_true"] == 0.0
    assert bool((xs[1] == 0).all())
    for k in (0, 2):
        assert infos[k]["iters"] == 3


def test_solve_batched_argument_checks():
    tca = lib()
    insts, bs = _batch(2, 610)
    p32 = tca.plan_from_instance(insts[0], precision="f32")
    p64 = tca.plan_from_instance(insts[1], precision="f64")
    b0 = to_dev(bs[0], np.float32)
    x0 = empty_dev(insts[0].shape, np.float32)
    with pytest.raises(tca.TcaError):
        tca.solve_batched([p32, p32], [b0, b0], [x0, x0])  # a plan twice
    b1 = to_dev(bs[1], np.float64)
    x1 = empty_dev(insts[1].shape, np.float64)
    with pytest.raises(tca.TcaError):
        tca.solve_batched([p32, p64], [b0, b1], [x0, x1])  # FP64 plan
    with pytest.raises(tca.TcaError):
        tca.solve_batched([p32], [bs[0]], [x0])  # host right-hand side


@pytest.mark.parametrize("shape", [(40, 37, 29, 8), (33, 41, 70), (23, 50, 45, 4)])
def test_autotune_keeps_parity(shape):
    tca = lib()
    inst = synth.instance_bspline(shape, seed=720 + len(shape), dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision="f32")
    chunks = plan.autotune()
    assert 1 <= chunks <= shape[0]
    again = tca.plan_from_instance(inst, precision="f32")
    assert again.autotune() == chunks  # cached per shape
    rng = np.random.default_rng(7)
    x = rng.standard_normal(shape)
    y = empty_dev(shape, np.float32)
    plan.apply_normal(to_dev(x, np.float32), y)
    ref = O.normal_apply(x.astype(np.float32).astype(np.float64), mats, inst.lam)
    assert rel_l2(y.cpu().numpy(), ref) < TOL_F32


def test_autotune_batched_picks_a_share_and_keeps_the_results():
    """tca_autotune_batched times the batch at every SM share and records the fastest for this
    batch; the tuned solve still meets the tolerance by the oracle, and a later call with the same
    arguments replays the same graph (identical iterates)."""
    tca = lib()
    insts, bs = _batch(6, 520)
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bd = [to_dev(b, np.float32) for b in bs]
    xs = [empty_dev(inst.shape, np.float32) for inst in insts]
    share = tca.autotune_batched(plans, bd, xs, rtol=1e-6, max_iter=20000)
    assert share in (1, 2, 3, 4, 6, 8)
    st, infos = tca.solve_batched(plans, bd, xs, rtol=1e-6, max_iter=20000)
    assert st == tca.OK
    first = [x.clone() for x in xs]
    for inst, b, x in zip(insts, bs, xs):
        mats = [f.dense() for f in inst.factors]
        assert O.rel_residual(x.cpu().numpy(), b.astype(np.float64), mats, inst.lam) <= 1.5e-6
    st2, infos2 = tca.solve_batched(plans, bd, xs, rtol=1e-6, max_iter=20000)
    for a, b_, i1, i2 in zip(first, xs, infos, infos2):
        assert i1["iters"] == i2["iters"]
        assert bool((a == b_).all())
