"""The bfloat16 form (TCA_BF16_IR) against the CPU FP64 oracle, through the C ABI.

The normal operator of a TCA_BF16_IR plan runs the tensor-core sweep: p and q in
bfloat16, the G_3 kron G_4 and regulariser contractions of modes 3-4 on tcgen05
with FP32 accumulation, modes 1-2 in FP32 registers.  Tolerance: relative L2
error <= 3e-2 against the FP64 oracle (the BF16 bound of the design notes: unit
roundoff 2^-9 for the rounded input, the rounded coefficients and the rounded
output, times the growth over the chained products), and >= 1e-5, which an
FP32 sweep would not reach - the check that the bfloat16 path is what ran.
Solves: the outer refinement in double-float arithmetic must still bring the
true residual to rtol, checked by the oracle's own FP64 residual.
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import empty_dev, lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu

TOL_BF16 = 3e-2


def _round_bf16(a):
    """bfloat16 rounding (nearest, ties to even) of float32 values, as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# (shape, lambda): TMA and cp.async halo paths, n4 = 8 / 4 / 1 and order 3,
# ragged row tiles (n2 % 16), ragged inner tiles (n3 n4 % 128), several tiles.
SHAPES = [
    ((24, 22, 23, 8), 1e-3),   # TMA boxes (n2 >= 22, 23 chunks >= 22), 2 inner tiles (184 = 128 + 56)
    ((24, 22, 23, 8), 0.1),    # a large lambda: a dropped regulariser term would show
    ((13, 30, 40, 4), 1e-3),   # n4 = 4 (KC = 20), 2 row tiles (second ragged), TMA
    ((9, 20, 22, 8), 0.1),     # n2 < 22: cp.async halo pieces
    ((11, 26, 152), 1e-2),     # order 3 (n4 = 1, KC = 18), TMA
    ((10, 17, 24, 1), 1e-2),   # order 4 with n4 = 1, cp.async (3 chunks < KC)
    ((40, 40, 40, 8), 1e-3),   # 3 row tiles and 3 inner tiles, both ragged
]


@pytest.mark.parametrize("shape,lam", SHAPES)
def test_bf16_normal_operator(shape, lam):
    tca = lib()
    inst = synth.instance_bspline(shape, seed=300 + len(shape) + shape[0], lam=lam, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(inst.shape).astype(np.float32)
    y = empty_dev(inst.shape, np.float32)
    plan.apply_normal(to_dev(x, np.float32), y)
    got = y.cpu().numpy()
    ref = O.normal_apply(x.astype(np.float64), mats, inst.lam)
    err = rel_l2(got, ref)
    assert 1e-5 < err < TOL_BF16, err
    # The same operator on the bfloat16-rounded input: what is left is the
    # rounding of the coefficients and of q, so it is tighter still.
    err_r = rel_l2(got, O.normal_apply(_round_bf16(x), mats, inst.lam))
    assert err_r < TOL_BF16 / 3, err_r


@pytest.mark.parametrize("shape", [(24, 22, 23, 8), (9, 20, 22, 8), (11, 26, 152)])
def test_bf16_inner_iterates_follow_the_oracle(shape):
    """max_iter = k stops the refinement after k inner CG iterations from d = 0, so x is
    the k-th CG iterate of Fig. 2 (one start, no restart).  It must match the oracle's
    FP64 CG iterate x_k, k = 1..6: this checks the CG form of the sweep
    (p = r + beta p_old, <p, q>, alpha), the bfloat16 update and the grouped
    correction update at every group position.  Each step perturbs the iteration by
    about 3 bfloat16 roundings (p, q, r: 3 x 2^-9 relative) and the perturbations
    of the k steps add up, so iterate k is held to max(3e-2, k x 6e-3)."""
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_bspline(shape, seed=41, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    rhs = O.apply_T(b.astype(np.float64), mats)
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    for k in range(1, 7):
        x = torch.zeros(inst.shape, dtype=torch.float32, device="cuda")
        st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-9, inner_rtol=1e-9, max_iter=k,
                              raise_on_error=False)
        assert st == tca.ERR_NOT_CONVERGED and info["iters"] == k, (st, info)
        ref = O.cg(lambda v: O.normal_apply(v, mats, inst.lam), rhs, rtol=0.0, max_iter=k).x
        err = rel_l2(x.cpu().numpy(), ref)
        print(f"bf16 iterate {shape} k={k}: rel. error {err:.2e}")
        assert err < max(TOL_BF16, k * 6e-3), (k, err)


@pytest.mark.parametrize("shape", [(24, 22, 23, 8), (13, 30, 40, 4), (9, 20, 22, 8), (11, 26, 152)])
def test_bf16_ir_solve_reaches_the_fp64_tolerance(shape):
    tca = lib()
    inst = synth.instance_bspline(shape, seed=77 + shape[0], dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, inner_rtol=1e-2)
    assert st == tca.OK, info
    assert info["refinements"] >= 2  # a bfloat16 inner solve alone cannot reach 1e-6
    got = x.cpu().numpy()
    rel = O.rel_residual(got, b.astype(np.float64), mats, inst.lam)
    assert rel <= 1.5e-6, (rel, info)
    assert abs(info["rel_res_true"] - rel) < 1e-7
    ref = O.solve(b.astype(np.float64), mats, inst.lam, rtol=1e-12).x
    assert rel_l2(got, ref) < 1e-4


def test_bf16_error_on_the_40cube_instance_of_the_workload_generator():
    """The 40x40x40x8 instance of the 160x160x160x8 workload's generator (same seed,
    60^3 x 12 samples): the mixed-precision solve against the FP64 oracle's solution."""
    tca = lib()
    inst = synth.instance_bspline((40, 40, 40, 8), seed=2, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, inner_rtol=1e-2)
    assert st == tca.OK, info
    got = x.cpu().numpy()
    ref = O.solve(b.astype(np.float64), mats, inst.lam, rtol=1e-12).x
    err = rel_l2(got, ref)
    print(f"bf16_ir 40x40x40x8: rel. error vs FP64 oracle {err:.3e}, inner iters {info['iters']}, "
          f"refinements {info['refinements']}")
    assert err < 1e-4
    assert O.rel_residual(got, b.astype(np.float64), mats, inst.lam) <= 1.5e-6


@pytest.mark.slow
def test_bf16_ir_full_size_solve():
    """The 160x160x160x8 workload solved in the mixed-precision form, its true residual
    recomputed by the oracle in FP64."""
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_bspline((160, 160, 160, 8), seed=2, dtype=np.float32)
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    xt = torch.from_numpy(inst.x_true).cuda()
    bd = torch.empty(inst.sample_shape, dtype=torch.float32, device="cuda")
    plan.apply(xt, bd)
    bd += torch.from_numpy(inst.noise).cuda()
    x = torch.zeros(inst.shape, dtype=torch.float32, device="cuda")
    st, info = plan.solve(bd, x, rtol=1e-6, inner_rtol=1e-2)
    assert st == tca.OK, info
    rel = O.rel_residual(x.cpu().numpy(), bd.cpu().numpy().astype(np.float64), mats, inst.lam)
    assert rel <= 1.5e-6, (rel, info)


def test_bf16_plans_refuse_what_they_do_not_compute():
    """Dense factors, n4 > 8 and inner axes that are not a multiple of 8 have no bfloat16
    sweep: the plan says so instead of running another precision under this name."""
    tca = lib()
    rng = np.random.default_rng(0)
    dense = synth.Instance((8, 8, 8), [synth.Factor("dense", 12, 8, a=synth.dense_gaussian_factor(12, 8, rng))
                                       for _ in range(3)], None, None, 1e-3, 0)
    for inst in (dense, synth.instance_bspline((8, 8, 8, 16), seed=1, with_truth=False),
                 synth.instance_bspline((8, 8, 13), seed=1, with_truth=False)):
        with pytest.raises(tca.TcaError) as e:
            tca.plan_from_instance(inst, precision="bf16_ir")
        assert e.value.status == tca.ERR_UNSUPPORTED
    # The solver takes no preconditioner in this form.
    inst = synth.instance_bspline((9, 20, 22, 8), seed=5, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    x = empty_dev(inst.shape, np.float32)
    st, _ = plan.solve(to_dev(b, np.float32), x, precond="separable", raise_on_error=False)
    assert st == tca.ERR_UNSUPPORTED


def test_bf16_autotune_keeps_parity_and_solves():
    """tca_autotune times the CG form of the tensor-core sweep over chunk counts and both
    worker layouts and keeps the fastest; the tuned plan still matches the oracle and
    still solves to the FP64 tolerance."""
    tca = lib()
    inst = synth.instance_bspline((40, 40, 40, 8), seed=12, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    chunks = plan.autotune()
    assert chunks >= 1 and plan.autotuned_rows() in (4, 8)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(inst.shape).astype(np.float32)
    y = empty_dev(inst.shape, np.float32)
    plan.apply_normal(to_dev(x, np.float32), y)
    assert rel_l2(y.cpu().numpy(), O.normal_apply(x.astype(np.float64), mats, inst.lam)) < TOL_BF16
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    xs = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), xs, rtol=1e-6, inner_rtol=3e-2)
    assert st == tca.OK, info
    assert O.rel_residual(xs.cpu().numpy(), b.astype(np.float64), mats, inst.lam) <= 1.5e-6
