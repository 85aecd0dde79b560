"""Scattered (off-grid) samples on the GPU against the CPU FP64 oracle, through the C ABI.

The plan's system tensor has one row per sample, the Kronecker product of the sample's
per-mode cubic B-spline rows (tca_plan_scattered).  Gather, scatter-add and the normal
operator are compared with the oracle's windowed sums on 3D and 4D grids with samples
everywhere in the box (windows cut by every face); FP64 with atomic additions, so the
tolerance is FP64 rounding over a few hundred terms per unknown (1e-12 relative L2).  The
solve is compared with a direct solve of the explicit normal matrix.
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import TOL_F64, empty_dev, lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _plan(tca, inst, **kw):
    return tca.ScatteredPlan(inst.shape, inst.col0, inst.w, lam=inst.lam, **kw)


@pytest.mark.parametrize("shape,m", [((20, 18, 16, 4), 30000), ((24, 20, 22), 20000), ((9, 7, 8, 5), 4000),
                                     ((6, 5, 4), 50)])
def test_scattered_operators_match_oracle(shape, m):
    tca = lib()
    inst = synth.instance_scattered(shape, m, seed=m % 97, lam=3e-3)
    plan = _plan(tca, inst)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape)
    y = rng.standard_normal(m)
    ax = empty_dev((m,), np.float64)
    plan.apply(to_dev(x, np.float64), ax)
    assert rel_l2(ax.cpu().numpy(), O.scattered_apply(x, inst.col0, inst.w)) < TOL_F64
    aty = empty_dev(shape, np.float64)
    plan.apply_T(to_dev(y, np.float64), aty)
    assert rel_l2(aty.cpu().numpy(), O.scattered_apply_T(y, inst.col0, inst.w, shape)) < TOL_F64
    kx = empty_dev(shape, np.float64)
    plan.apply_normal(to_dev(x, np.float64), kx)
    assert rel_l2(kx.cpu().numpy(), O.scattered_normal_apply(x, inst.col0, inst.w, inst.lam)) < TOL_F64
    # Host buffers through the same calls.
    axh = np.zeros(m)
    plan.apply(np.ascontiguousarray(x), axh)
    np.testing.assert_allclose(axh, ax.cpu().numpy(), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("shape,m", [((10, 9, 8), 700), ((7, 6, 5, 4), 900)])
def test_scattered_solve_matches_direct_solve(shape, m):
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_scattered(shape, m, seed=5, lam=1e-2)
    a = O.scattered_rows_matrix(inst.col0, inst.w, shape)
    b = a @ inst.x_true.ravel() + inst.noise
    k = a.T @ a + O.dense_normal_matrix([np.zeros((1, n)) for n in shape], inst.lam, shape)
    ref = np.linalg.solve(k, a.T @ b)
    plan = _plan(tca, inst)
    x = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, info = plan.solve(to_dev(b, np.float64), x, rtol=1e-10, max_iter=20000)
    assert st == tca.OK, info
    got = x.cpu().numpy().ravel()
    assert rel_l2(got, ref) < 1e-8
    rel = np.linalg.norm(a.T @ b - k @ got) / np.linalg.norm(a.T @ b)
    assert rel <= 1.5e-10 and abs(info["rel_res_true"] - rel) <= 1e-3 * rel + 1e-14, (rel, info)


def test_scattered_plan_refusals():
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_scattered((8, 7, 6), 200, seed=1, lam=1e-2)
    for prec in ("f32", "bf16_ir", "tf32_ir"):
        with pytest.raises(tca.TcaError) as e:
            _plan(tca, inst, precision=prec)
        assert e.value.status == tca.ERR_UNSUPPORTED
    bad = synth.instance_scattered((8, 7, 6), 200, seed=1)
    bad.col0[1] = bad.col0[1][:150]
    bad.w[1] = bad.w[1][:150]
    with pytest.raises(tca.TcaError) as e:
        _plan(tca, bad)
    assert e.value.status == tca.ERR_SHAPE
    plan = _plan(tca, inst)
    b = to_dev(np.ones(200), np.float64)
    x = torch.zeros((8, 7, 6), dtype=torch.float64, device="cuda")
    for pc in ("separable", "jacobi"):
        st, _ = plan.solve(b, x, precond=pc, raise_on_error=False)
        assert st == tca.ERR_UNSUPPORTED
    with pytest.raises(tca.TcaError) as e:
        plan.apply_mode(0, tca.OP_GRAM, (8, 7, 6), x, torch.zeros_like(x))
    assert e.value.status == tca.ERR_UNSUPPORTED
