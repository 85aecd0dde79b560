"""Parity of the point-Jacobi preconditioned CG (M = diag(K), the Fig. 1 solver family) with the
oracle, through the C ABI.

The GPU solve with precond="jacobi" is compared with ``oracle.pcg`` driven by
``oracle.jacobi_diagonal`` on the same seeded inputs: iterate by iterate for the
first steps (every position of the four-iteration update group), then solves to
the oracle's own verdict, batched and single.
"""
import math

import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import empty_dev, lib, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _dense(shape, seed, lam, spread=0.0):
    """Dense Gaussian factors; spread > 0 scales factor k's columns by 10^U(-spread, spread)."""
    rng = np.random.default_rng(seed)
    facs = []
    for n in shape:
        m = int(np.ceil(1.5 * n))
        a = synth.dense_gaussian_factor(m, n, rng) * 10.0 ** rng.uniform(-spread, spread, n)
        facs.append(synth.Factor("dense", m, n, a=a))
    x = rng.standard_normal(shape)
    noise = 0.01 * rng.standard_normal(tuple(f.m for f in facs))
    return synth.Instance(tuple(shape), facs, x, noise, lam, seed)


CASES = [
    ("bspline", (20, 18, 16, 8), "f32"),    # fused sweep from z, n4 = 8
    ("bspline", (33, 41, 30), "f32"),       # fused sweep, order 3
    ("bspline", (12, 13, 11, 16), "f32"),   # generic sweeps
    ("dense", (14, 12, 10, 4), "f32"),      # tensor-core Gram products
    ("dense", (12, 11, 10), "f64"),         # native FP64
    ("bspline", (17, 14, 19, 3), "f64"),
]


@pytest.mark.parametrize("kind,shape,prec", CASES)
def test_jacobi_pcg_iterates_match_oracle(kind, shape, prec):
    tca = lib()
    dt = np.float32 if prec == "f32" else np.float64
    # As for the other preconditioned iterates: FP32 1e-4, dense FP32 1e-3 (3xTF32
    # products), FP64 1e-10.
    tol = (1e-3 if kind == "dense" else 1e-4) if prec == "f32" else 1e-10
    inst = (synth.instance_bspline(shape, seed=750, dtype=np.float64) if kind == "bspline"
            else _dense(shape, 750, 1e-3, spread=0.5))
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(dt)
    plan = tca.plan_from_instance(inst, precision=prec)
    rhs = O.apply_T(b.astype(np.float64), mats)
    kop = lambda v: O.normal_apply(v, mats, inst.lam)
    dia = O.jacobi_diagonal(mats, inst.lam, inst.shape)
    for k in (1, 2, 3, 4, 5, 7):
        x = empty_dev(inst.shape, dt)
        st, info = plan.solve(to_dev(b, dt), x, rtol=1e-14, max_iter=k, raise_on_error=False, precond="jacobi")
        assert st == tca.ERR_NOT_CONVERGED and info["iters"] == k
        ref = O.pcg(kop, lambda r: r / dia, rhs, rtol=0.0, max_iter=k).x
        assert rel_l2(x.cpu().numpy(), ref) < tol, k


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_jacobi_solves_a_badly_scaled_problem_that_plain_cg_struggles_with(prec):
    """Columns scaled over two decades: Jacobi brings the solve to 1e-6 (oracle's verdict) in a
    fraction of the plain CG's iterations on the same plan."""
    tca = lib()
    dt = np.float64 if prec == "f64" else np.float32
    inst = _dense((14, 12, 11), 760, 1e-4, spread=1.0)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(dt)
    plan = tca.plan_from_instance(inst, precision=prec)
    x = empty_dev(inst.shape, dt)
    st, info = plan.solve(to_dev(b, dt), x, rtol=1e-6, max_iter=20000, precond="jacobi")
    assert st == tca.OK, info
    assert O.rel_residual(x.cpu().numpy().astype(np.float64), b.astype(np.float64), mats, inst.lam) <= 1.5e-6
    x0 = empty_dev(inst.shape, dt)
    st0, info0 = plan.solve(to_dev(b, dt), x0, rtol=1e-6, max_iter=20000, raise_on_error=False)
    assert info["iters"] * 2 < info0["iters"], (info["iters"], info0["iters"])


def test_jacobi_batched_matches_single_solves_and_switches_with_separable():
    """One graph launch of Jacobi-preconditioned instances gives the single solves; switching the
    same plans to the separable preconditioner and back rebuilds the cached graphs."""
    tca = lib()
    insts = [synth.instance_batched(i, lo=16, hi=28) for i in range(5)]
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bs, xs = [], []
    for inst in insts:
        mats = [f.dense() for f in inst.factors]
        bs.append(to_dev((O.apply(inst.x_true, mats) + inst.noise).astype(np.float32), np.float32))
        xs.append(empty_dev(inst.shape, np.float32))
    st, infos = tca.solve_batched(plans, bs, xs, rtol=1e-6, max_iter=20000, precond="jacobi")
    assert st == tca.OK
    first = [x.cpu().numpy().copy() for x in xs]
    for i, (inst, plan) in enumerate(zip(insts, plans)):
        mats = [f.dense() for f in inst.factors]
        assert O.rel_residual(first[i], bs[i].cpu().numpy().astype(np.float64), mats, inst.lam) <= 1.5e-6
        xr = empty_dev(inst.shape, np.float32)
        st1, info1 = plan.solve(bs[i], xr, rtol=1e-6, max_iter=20000, precond="jacobi")
        assert st1 == tca.OK
        assert abs(infos[i]["iters"] - info1["iters"]) <= 3
    st, _ = tca.solve_batched(plans, bs, xs, rtol=1e-6, max_iter=20000, precond="separable")
    assert st == tca.OK
    st, infos2 = tca.solve_batched(plans, bs, xs, rtol=1e-6, max_iter=20000, precond="jacobi")
    assert st == tca.OK
    for i in range(len(insts)):
        assert infos2[i]["iters"] == infos[i]["iters"]
        np.testing.assert_array_equal(xs[i].cpu().numpy(), first[i])
