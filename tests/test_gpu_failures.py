"""Failure paths made on the host, through the C ABI: a non-finite right-hand side or
initial guess, and a singular normal operator.

No GPU fault is involved: the inputs are ordinary buffers holding NaN or Inf, or
factors with fewer rows than columns.  After every failure the same plan solves a
regular problem, so the context and the plan's state are shown to be usable.
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import lib, need_cuda, to_dev

pytestmark = pytest.mark.gpu


def _bspline_case():
    inst = synth.instance_bspline((24, 20, 22, 8), seed=11, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    return inst, mats, b


def _assert_recovers(tca, plan, inst, mats, b, dtype):
    torch = need_cuda()
    x = torch.zeros(inst.shape, dtype=torch.float64 if dtype == np.float64 else torch.float32, device="cuda")
    st, info = plan.solve(to_dev(b, dtype), x, rtol=1e-6)
    assert st == tca.OK, info
    assert O.rel_residual(x.cpu().numpy().astype(np.float64), b, mats, inst.lam) <= 1.5e-6


@pytest.mark.parametrize("precision", ["f32", "f64", "tf32_ir", "bf16_ir"])
def test_nan_in_b_is_a_breakdown(precision):
    tca = lib()
    torch = need_cuda()
    inst, mats, b = _bspline_case()
    dtype = np.float64 if precision == "f64" else np.float32
    plan = tca.plan_from_instance(inst, precision=precision)
    bad = b.copy()
    bad[3, 5, 7, 1] = np.nan
    x = torch.zeros(inst.shape, dtype=torch.float64 if dtype == np.float64 else torch.float32, device="cuda")
    st, info = plan.solve(to_dev(bad, dtype), x, rtol=1e-6, raise_on_error=False)
    assert st == tca.ERR_BREAKDOWN, (st, info)
    _assert_recovers(tca, plan, inst, mats, b, dtype)


def test_nan_in_b_dense_generic_path():
    """Dense factors take the generic iteration (tensor-core mode products), not the fused sweep."""
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_dense_3d(seed=0)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    plan = tca.plan_from_instance(inst, precision="f32")
    bad = b.copy()
    bad[0, 0, 0] = np.inf
    x = torch.zeros(inst.shape, dtype=torch.float32, device="cuda")
    st, _ = plan.solve(to_dev(bad, np.float32), x, rtol=1e-6, raise_on_error=False)
    assert st == tca.ERR_BREAKDOWN
    _assert_recovers(tca, plan, inst, mats, b, np.float32)


def test_inf_in_initial_guess_is_a_breakdown():
    tca = lib()
    torch = need_cuda()
    inst, mats, b = _bspline_case()
    plan = tca.plan_from_instance(inst, precision="f32")
    x0 = np.zeros(inst.shape, np.float32)
    x0[1, 2, 3, 4] = np.inf
    x = to_dev(x0, np.float32)
    st, _ = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, x0_given=True, raise_on_error=False)
    assert st == tca.ERR_BREAKDOWN
    _assert_recovers(tca, plan, inst, mats, b, np.float32)


def test_nan_in_one_batched_instance_leaves_the_others_converged():
    tca = lib()
    torch = need_cuda()
    insts = [synth.instance_batched(i, lo=24, hi=32) for i in range(3)]
    plans, bs, xs, mats_all, b_all = [], [], [], [], []
    for i, inst in enumerate(insts):
        mats = [f.dense() for f in inst.factors]
        b = O.apply(inst.x_true.astype(np.float64), mats) + inst.noise
        mats_all.append(mats)
        b_all.append(b)
        bb = b.copy()
        if i == 1:
            bb.flat[17] = np.nan
        plans.append(tca.plan_from_instance(inst, precision="f32"))
        bs.append(to_dev(bb, np.float32))
        xs.append(torch.zeros(inst.shape, dtype=torch.float32, device="cuda"))
    st, infos = tca.solve_batched(plans, bs, xs, rtol=1e-6, raise_on_error=False)
    assert st == tca.ERR_BREAKDOWN
    for i in (0, 2):
        rel = O.rel_residual(xs[i].cpu().numpy().astype(np.float64), b_all[i], mats_all[i], insts[i].lam)
        assert rel <= 1.5e-6, (i, rel, infos[i])
    # The plans still solve on their own afterwards.
    _assert_recovers(tca, plans[1], insts[1], mats_all[1], b_all[1], np.float32)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_singular_normal_operator(precision):
    """lambda = 0 and factors with fewer rows than columns: K = kron(A_k^T A_k) is singular
    (rank 10^3 of 16^3).  A^T b lies in K's range, so the system is consistent: the FP64
    plan converges to a least-squares solution (checked by the oracle's own FP64
    residual).  In FP32 the roundings feed K's null space into the directions until
    <p, Kp> stops being positive; the header documents TCA_ERR_BREAKDOWN for that case
    (or NOT_CONVERGED / OK if the iteration outruns it), with x the last iterate and its
    true residual reported.  Either way x is finite and the plan solves again."""
    tca = lib()
    torch = need_cuda()
    rng = np.random.default_rng(5)
    n, m = 16, 10
    factors = [synth.Factor("dense", m, n, a=synth.dense_gaussian_factor(m, n, rng)) for _ in range(3)]
    inst = synth.Instance((n, n, n), factors, synth.gaussian_blobs((n, n, n), 5, 3.0, rng),
                          0.01 * rng.standard_normal((m, m, m)), 0.0, 5)
    mats = [f.dense() for f in inst.factors]
    assert np.linalg.matrix_rank(O.dense_normal_matrix(mats, 0.0, inst.shape)) == m ** 3
    b = O.apply(inst.x_true, mats) + inst.noise
    dtype = np.float64 if precision == "f64" else np.float32
    plan = tca.plan_from_instance(inst, precision=precision)
    x = torch.zeros(inst.shape, dtype=torch.float64 if dtype == np.float64 else torch.float32, device="cuda")
    st, info = plan.solve(to_dev(b, dtype), x, rtol=1e-6, max_iter=4000, raise_on_error=False)
    xs = x.cpu().numpy().astype(np.float64)
    assert np.isfinite(xs).all()
    rel = O.rel_residual(xs, b, mats, 0.0)
    if precision == "f64":
        assert st == tca.OK, (st, info)
        assert rel <= 1.5e-6
    else:
        assert st in (tca.OK, tca.ERR_BREAKDOWN, tca.ERR_NOT_CONVERGED), (st, info)
        if st == tca.OK:
            assert rel <= 1.5e-6
        else:
            # The reported residual is the iterate's own, not a placeholder.
            assert abs(info["rel_res_true"] - rel) <= 1e-3 * rel + 1e-9, (info, rel)
    # A regular problem on a fresh plan right after: the context is fine.
    inst2, mats2, b2 = _bspline_case()
    plan2 = tca.plan_from_instance(inst2, precision="f32")
    _assert_recovers(tca, plan2, inst2, mats2, b2, np.float32)
