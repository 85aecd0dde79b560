"""Parity of the preconditioned CG (separable tensor-inverse preconditioner) with the oracle.

The GPU solve with precond="separable" is compared with ``oracle.pcg`` driven by
``oracle.separable_inverse_factors`` (at the library's default shift, the plan's corner-model
shift, checked equal to ``oracle.corner_model_shift``) on the same seeded inputs: iterate by iterate for the first steps (every position of the
four-iteration solution-update group), then the converged solution against the
oracle's own verdict.  FP32 plans apply the preconditioner's dense factors on the
tensor cores in 3xTF32 at these sizes (about 2^-21 relative per product), FP64
plans natively.
"""
import ctypes

import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import empty_dev, lib, rel_l2, to_dev

pytestmark = pytest.mark.gpu



def _dense(shape, seed, lam):
    rng = np.random.default_rng(seed)
    facs = []
    for n in shape:
        m = int(np.ceil(1.5 * n))
        facs.append(synth.Factor("dense", m, n, a=synth.dense_gaussian_factor(m, n, rng)))
    x = rng.standard_normal(shape)
    noise = 0.01 * rng.standard_normal(tuple(f.m for f in facs))
    return synth.Instance(tuple(shape), facs, x, noise, lam, seed)


def _inst(kind, shape, seed, lam):
    if kind == "bspline":
        return synth.instance_bspline(shape, seed=seed, lam=lam, dtype=np.float64)
    return _dense(shape, seed, lam)


CASES = [
    ("bspline", (20, 18, 16, 8), "f32", 1e-3),    # fused sweep from z, n4 = 8
    ("bspline", (33, 41, 30), "f32", 1e-3),       # fused sweep, order 3
    ("bspline", (12, 13, 11, 16), "f32", 1e-3),   # generic sweeps
    ("dense", (14, 12, 10, 4), "f32", 1e-3),      # tensor-core Gram and preconditioner
    ("dense", (12, 11, 10), "f64", 1e-3),         # native FP64
    ("bspline", (17, 14, 19, 3), "f64", 1e-3),
]


@pytest.mark.parametrize("kind,shape,prec,lam", CASES)
def test_pcg_partial_iterates_match_oracle(kind, shape, prec, lam):
    tca = lib()
    dt = np.float32 if prec == "f32" else np.float64
    # FP32: 1e-4 as for the plain iterates.  Dense FP32 plans form their products
    # in 3xTF32 (about 2^-21 relative per product, not 2^-24), and z = M^-1 r
    # amplifies the roundings of r by the preconditioner factors' condition
    # numbers (6 to 75 per mode in this case): an oracle run with every vector
    # and mode product rounded to FP32 already differs by 3.5e-5 at k = 2, so
    # the dense case is held to 1e-3.
    tol = (1e-3 if kind == "dense" else 1e-4) if prec == "f32" else 1e-10
    inst = _inst(kind, shape, 700, lam)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(dt)
    plan = tca.plan_from_instance(inst, precision=prec)
    rhs = O.apply_T(b.astype(np.float64), mats)
    kop = lambda v: O.normal_apply(v, mats, inst.lam)
    shift = plan.precond_default_shift()
    assert shift == O.corner_model_shift(mats, inst.lam)
    inv = O.separable_inverse_factors(mats, inst.lam, shift)
    minv = lambda r: O.apply_separable(r, inv)
    for k in (1, 2, 3, 4, 5, 7):
        x = empty_dev(inst.shape, dt)
        st, info = plan.solve(to_dev(b, dt), x, rtol=1e-14, max_iter=k, raise_on_error=False,
                              precond="separable")
        assert st == tca.ERR_NOT_CONVERGED and info["iters"] == k
        ref = O.pcg(kop, minv, rhs, rtol=0.0, max_iter=k).x
        assert rel_l2(x.cpu().numpy(), ref) < tol, k


@pytest.mark.parametrize("kind,shape,prec,lam", [("bspline", (24, 20, 22, 8), "f32", 1e-3),
                                                 ("dense", (16, 14, 12, 4), "f32", 2e-4),
                                                 ("dense", (18, 15, 13), "f64", 5e-4),
                                                 ("bspline", (20, 18, 16, 4), "tf32_ir", 1e-3)])
def test_pcg_solve_meets_tolerance_in_fewer_iterations(kind, shape, prec, lam):
    """Solved to a true relative residual of 1e-6 (the oracle's verdict on the GPU's x), matching
    the oracle's solution, in fewer iterations than the plain CG of the same plan."""
    tca = lib()
    dt = np.float64 if prec == "f64" else np.float32
    inst = _inst(kind, shape, 710, lam)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(dt)
    plan = tca.plan_from_instance(inst, precision=prec)
    x = empty_dev(inst.shape, dt)
    st, info = plan.solve(to_dev(b, dt), x, rtol=1e-6, precond="separable")
    assert st == tca.OK, info
    got = x.cpu().numpy()
    assert info["rel_res_true"] <= 1e-6
    assert O.rel_residual(got, b.astype(np.float64), mats, inst.lam) <= 1.5e-6
    x0 = empty_dev(inst.shape, dt)
    st0, info0 = plan.solve(to_dev(b, dt), x0, rtol=1e-6)
    assert st0 == tca.OK
    assert info["iters"] < info0["iters"], (info["iters"], info0["iters"])
    # Both meet the same tolerance: their difference is what that tolerance allows.
    assert rel_l2(got, x0.cpu().numpy()) < 1e-3


def test_pcg_batched_matches_single_solves():
    tca = lib()
    insts = [synth.instance_batched(i, lo=16, hi=28) for i in range(6)]
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bs, xs, xr = [], [], []
    for inst in insts:
        mats = [f.dense() for f in inst.factors]
        b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
        bs.append(to_dev(b, np.float32))
        xs.append(empty_dev(inst.shape, np.float32))
        xr.append(empty_dev(inst.shape, np.float32))
    st, infos = tca.solve_batched(plans, bs, xs, rtol=1e-6, max_iter=5000, precond="separable")
    assert st == tca.OK
    for i, (inst, plan) in enumerate(zip(insts, plans)):
        st1, info1 = plan.solve(bs[i], xr[i], rtol=1e-6, max_iter=5000, precond="separable")
        assert st1 == tca.OK
        mats = [f.dense() for f in inst.factors]
        b64 = bs[i].cpu().numpy().astype(np.float64)
        assert infos[i]["rel_res_true"] <= 1e-6
        assert O.rel_residual(xs[i].cpu().numpy(), b64, mats, inst.lam) <= 1.5e-6
        assert abs(infos[i]["iters"] - info1["iters"]) <= 3, (i, infos[i]["iters"], info1["iters"])


def test_pcg_host_buffers_match_device():
    """A preconditioned solve from host buffers (b uploaded under A^T b) gives the device-buffer
    result bit for bit."""
    tca = lib()
    inst = synth.instance_bspline((24, 20, 22, 8), seed=730, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    xd = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), xd, rtol=1e-6, precond="separable")
    assert st == tca.OK
    xh = np.zeros(inst.shape, np.float32)
    st, info_h = plan.solve(np.ascontiguousarray(b), xh, rtol=1e-6, precond="separable")
    assert st == tca.OK and info_h["iters"] == info["iters"]
    np.testing.assert_array_equal(xh, xd.cpu().numpy())


def test_pcg_shift_change_rebuilds_factors_and_graph():
    """Switching the shift rebuilds the factors (and drops the cached iteration graph that held
    the old ones): shift 16, then 32, then 16 again gives the first result bit for bit."""
    tca = lib()
    inst = synth.instance_bspline((20, 18, 16, 8), seed=740, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = to_dev((O.apply(inst.x_true, mats) + inst.noise).astype(np.float32), np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    xs = [empty_dev(inst.shape, np.float32) for _ in range(3)]
    its = []
    for x, shift in zip(xs, (16.0, 32.0, 16.0)):
        st, info = plan.solve(b, x, rtol=1e-6, precond="separable", precond_shift=shift)
        assert st == tca.OK and info["rel_res_true"] <= 1e-6
        its.append(info["iters"])
    assert its[0] == its[2]
    np.testing.assert_array_equal(xs[0].cpu().numpy(), xs[2].cpu().numpy())


def test_pcg_argument_checks():
    tca = lib()
    inst = synth.instance_bspline((12, 10, 9, 4), seed=720, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = to_dev((O.apply(inst.x_true, mats) + inst.noise).astype(np.float32), np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(inst.shape, np.float32)
    with pytest.raises(ValueError):
        plan.solve(b, x, precond="multigrid")
    for code, shift in ((7, 0.0), (tca.PRECOND_SEPARABLE, -1.0)):
        opts = tca.tca_solve_opts(1e-6, 100, 0, 0.0, 0, 0, 0, code, shift)
        info = tca.tca_solve_info()
        st = tca._lib.tca_solve(plan.handle, b.data_ptr(), x.data_ptr(), ctypes.byref(opts), ctypes.byref(info),
                                None)
        assert st == tca.ERR_INVALID_ARG
    # A zero right-hand side needs no iteration with the preconditioner either.
    z = to_dev(np.zeros(inst.sample_shape, np.float32), np.float32)
    st, info = plan.solve(z, x, rtol=1e-6, precond="separable")
    assert st == tca.OK and info["iters"] == 0
    assert float(x.abs().max()) == 0.0


BANDED_CASES = [
    ("bspline", (20, 18, 16, 8), "f32"),    # the plain fused sweep applies M^-1 (n4 = 8, warp-specialised)
    ("bspline", (33, 41, 30), "f32"),       # fused sweep, order 3
    ("bspline", (23, 26, 21, 4), "f32"),    # fused sweep, n4 = 4
    ("bspline", (12, 13, 11, 16), "f32"),   # band mode products (no fused sweep)
    ("bspline", (17, 14, 19, 3), "f64"),    # FP64 band mode products
]


@pytest.mark.parametrize("kind,shape,prec", BANDED_CASES)
def test_banded_pcg_iterates_match_oracle(kind, shape, prec):
    """precond="separable_banded": the separable inverse factors cut to |i - j| <= 3, applied as one
    fused sweep (or band products); iterates k = 1..7 against the oracle's pcg with
    separable_inverse_factors(..., half_band=3) at the default shift."""
    tca = lib()
    dt = np.float32 if prec == "f32" else np.float64
    tol = 1e-4 if prec == "f32" else 1e-10
    inst = _inst(kind, shape, 770, 1e-3)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(dt)
    plan = tca.plan_from_instance(inst, precision=prec)
    rhs = O.apply_T(b.astype(np.float64), mats)
    kop = lambda v: O.normal_apply(v, mats, inst.lam)
    shift = plan.precond_default_shift()
    assert shift == O.corner_model_shift(mats, inst.lam)
    inv = O.separable_inverse_factors(mats, inst.lam, shift, half_band=3)
    minv = lambda r: O.apply_separable(r, inv)
    for k in (1, 2, 3, 4, 5, 7):
        x = empty_dev(inst.shape, dt)
        st, info = plan.solve(to_dev(b, dt), x, rtol=1e-14, max_iter=k, raise_on_error=False,
                              precond="separable_banded")
        assert st == tca.ERR_NOT_CONVERGED and info["iters"] == k
        ref = O.pcg(kop, minv, rhs, rtol=0.0, max_iter=k).x
        assert rel_l2(x.cpu().numpy(), ref) < tol, k


@pytest.mark.parametrize("shift", [16.0, 32.0])
def test_banded_pcg_solves_in_fewer_iterations(shift):
    tca = lib()
    inst = synth.instance_bspline((40, 36, 32, 8), seed=780, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, precond="separable_banded", precond_shift=shift)
    assert st == tca.OK, info
    assert O.rel_residual(x.cpu().numpy(), b.astype(np.float64), mats, inst.lam) <= 1.5e-6
    x0 = empty_dev(inst.shape, np.float32)
    st0, info0 = plan.solve(to_dev(b, np.float32), x0, rtol=1e-6)
    assert info["iters"] * 2 < info0["iters"], (info["iters"], info0["iters"])
    # Switching to the dense-factor form and back rebuilds graph and factors: same result.
    x1 = empty_dev(inst.shape, np.float32)
    plan.solve(to_dev(b, np.float32), x1, rtol=1e-6, precond="separable", precond_shift=shift)
    x2 = empty_dev(inst.shape, np.float32)
    st2, info2 = plan.solve(to_dev(b, np.float32), x2, rtol=1e-6, precond="separable_banded", precond_shift=shift)
    assert info2["iters"] == info["iters"]
    np.testing.assert_array_equal(x2.cpu().numpy(), x.cpu().numpy())


def test_banded_pcg_batched_matches_single_solves():
    tca = lib()
    insts = [synth.instance_batched(2 * i + 1, lo=16, hi=28) for i in range(4)]  # B-spline instances
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bs, xs = [], []
    for inst in insts:
        mats = [f.dense() for f in inst.factors]
        bs.append(to_dev((O.apply(inst.x_true, mats) + inst.noise).astype(np.float32), np.float32))
        xs.append(empty_dev(inst.shape, np.float32))
    st, infos = tca.solve_batched(plans, bs, xs, rtol=1e-6, max_iter=5000, precond="separable_banded")
    assert st == tca.OK
    for i, (inst, plan) in enumerate(zip(insts, plans)):
        mats = [f.dense() for f in inst.factors]
        assert O.rel_residual(xs[i].cpu().numpy(), bs[i].cpu().numpy().astype(np.float64), mats, inst.lam) <= 1.5e-6
        xr = empty_dev(inst.shape, np.float32)
        st1, info1 = plan.solve(bs[i], xr, rtol=1e-6, max_iter=5000, precond="separable_banded")
        assert st1 == tca.OK and abs(infos[i]["iters"] - info1["iters"]) <= 3


@pytest.mark.parametrize("lam", [1e-4, 1e-2])
@pytest.mark.parametrize("pc", ["separable", "separable_banded"])
def test_default_shift_follows_lambda(lam, pc):
    """With no shift given the preconditioner takes the plan's corner-model shift (equal to the
    oracle's model; 128 at lambda = 1e-4, 5.7 at 1e-2 on this instance, against 16 fixed): the solve
    meets 1e-6 in no more iterations than at s = 16."""
    tca = lib()
    inst = _inst("bspline", (24, 20, 22, 8), 720, lam)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    shift = plan.precond_default_shift()
    assert shift == O.corner_model_shift(mats, lam)
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, precond=pc)
    assert st == tca.OK and info["rel_res_true"] <= 1e-6
    st16, info16 = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, precond=pc, precond_shift=16.0)
    assert st16 == tca.OK
    assert info["iters"] <= info16["iters"], (shift, info["iters"], info16["iters"])
