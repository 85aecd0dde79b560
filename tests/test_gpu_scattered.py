"""Scattered (off-grid) samples on the GPU against the CPU FP64 oracle, through the C ABI.

The plan's system tensor has one row per sample, the Kronecker product of the sample's
per-mode cubic B-spline rows (tca_plan_scattered).  Gather, scatter-add and the normal
operator are compared with the oracle's windowed sums on 3D and 4D grids with samples
everywhere in the box (windows cut by every face), in FP64 (atomic additions: the tolerance
is FP64 rounding over a few hundred terms per unknown, 1e-12 relative L2) and in FP32 (the
FP32 tolerance of the other operator tests).  The grids span several shared-memory tiles
with ragged edge tiles, grids whose small modes do not fit one tile uncut, and rows with
arbitrary weights whose windows lie partly or wholly outside the grid.  Solves are compared
with a direct solve of the explicit normal matrix.
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import TOL_F32, TOL_F64, empty_dev, lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _plan(tca, inst, **kw):
    return tca.ScatteredPlan(inst.shape, inst.col0, inst.w, lam=inst.lam, **kw)


PRECS = [("f64", np.float64, TOL_F64), ("f32", np.float32, TOL_F32)]


def _check_operators(tca, plan, col0, w, shape, lam, dt, tol, seed=4):
    m = col0[0].shape[0]
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape).astype(dt)
    y = rng.standard_normal(m).astype(dt)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    ax = empty_dev((m,), dt)
    plan.apply(to_dev(x, dt), ax)
    assert rel_l2(ax.cpu().numpy(), O.scattered_apply(xd, col0, w)) < tol
    aty = empty_dev(shape, dt)
    plan.apply_T(to_dev(y, dt), aty)
    assert rel_l2(aty.cpu().numpy(), O.scattered_apply_T(yd, col0, w, shape)) < tol
    kx = empty_dev(shape, dt)
    plan.apply_normal(to_dev(x, dt), kx)
    assert rel_l2(kx.cpu().numpy(), O.scattered_normal_apply(xd, col0, w, lam)) < tol
    return x, ax


@pytest.mark.parametrize("prec,dt,tol", PRECS)
@pytest.mark.parametrize("shape,m", [((20, 18, 16, 4), 30000), ((24, 20, 22), 20000), ((9, 7, 8, 5), 4000),
                                     ((6, 5, 4), 50), ((40, 37, 35, 5), 60000), ((50, 45, 61), 40000),
                                     ((16, 16, 16, 16), 20000)])
def test_scattered_operators_match_oracle(shape, m, prec, dt, tol):
    tca = lib()
    inst = synth.instance_scattered(shape, m, seed=m % 97, lam=3e-3)
    plan = _plan(tca, inst, precision=prec)
    x, ax = _check_operators(tca, plan, inst.col0, inst.w, shape, inst.lam, dt, tol)
    # Host buffers through the same calls.
    axh = np.zeros(m, dtype=dt)
    plan.apply(np.ascontiguousarray(x), axh)
    r = 1e-13 if dt == np.float64 else 1e-5
    np.testing.assert_allclose(axh, ax.cpu().numpy(), rtol=r, atol=r)


@pytest.mark.parametrize("prec,dt,tol", PRECS)
@pytest.mark.parametrize("shape", [(23, 19, 30, 6), (41, 9, 27)])
def test_scattered_rows_with_windows_outside_the_grid(shape, prec, dt, tol):
    """General ELL-4 rows: random weights, first columns from far below 0 to past the last
    column and at the ends of the int32 range (windows partly or wholly outside the grid,
    whose taps are dropped)."""
    tca = lib()
    rng = np.random.default_rng(sum(shape))
    m = 5000
    col0 = [rng.integers(-6, n + 3, size=m).astype(np.int32) for n in shape]
    for c in col0:  # and first columns at the ends of the int32 range
        c[:4] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, -(10 ** 9), 10 ** 9]
    w = [rng.standard_normal((m, 4)) for _ in shape]
    plan = tca.ScatteredPlan(shape, col0, w, lam=2e-3, precision=prec)
    _, ax = _check_operators(tca, plan, col0, w, shape, 2e-3, dt, tol, seed=9)
    # A sample whose window misses the grid in some mode has A x = 0 exactly.
    outside = np.zeros(m, dtype=bool)
    for c, n in zip(col0, shape):
        c = c.astype(np.int64)
        outside |= (c + 3 < 0) | (c >= n)
    assert outside.any() and np.all(ax.cpu().numpy()[outside] == 0.0)


def _direct(inst, shape):
    a = O.scattered_rows_matrix(inst.col0, inst.w, shape)
    b = a @ inst.x_true.ravel() + inst.noise
    k = a.T @ a + O.dense_normal_matrix([np.zeros((1, n)) for n in shape], inst.lam, shape)
    return a, b, k, np.linalg.solve(k, a.T @ b)


@pytest.mark.parametrize("shape,m", [((10, 9, 8), 700), ((7, 6, 5, 4), 900)])
def test_scattered_solve_matches_direct_solve(shape, m):
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_scattered(shape, m, seed=5, lam=1e-2)
    a, b, k, ref = _direct(inst, shape)
    plan = _plan(tca, inst)
    x = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, info = plan.solve(to_dev(b, np.float64), x, rtol=1e-10, max_iter=20000)
    assert st == tca.OK, info
    got = x.cpu().numpy().ravel()
    assert rel_l2(got, ref) < 1e-8
    rel = np.linalg.norm(a.T @ b - k @ got) / np.linalg.norm(a.T @ b)
    assert rel <= 1.5e-10 and abs(info["rel_res_true"] - rel) <= 1e-3 * rel + 1e-14, (rel, info)


@pytest.mark.parametrize("shape,m", [((10, 9, 8), 700), ((7, 6, 5, 4), 900), ((30, 26, 28, 4), 25000)])
def test_scattered_fp32_solve_meets_the_fp64_true_residual(shape, m):
    """FP32 plan: FP32 iterations, A^T b and the true residual by the FP64 operator, so the
    reported residual is the FP64 one of the returned iterate and meets rtol = 1e-6."""
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_scattered(shape, m, seed=6, lam=1e-2)
    if m <= 1000:
        a, b, k, ref = _direct(inst, shape)
    else:
        b = O.scattered_apply(inst.x_true, inst.col0, inst.w) + inst.noise
    b32 = b.astype(np.float32)
    plan = _plan(tca, inst, precision="f32")
    x = torch.zeros(shape, dtype=torch.float32, device="cuda")
    st, info = plan.solve(to_dev(b32, np.float32), x, rtol=1e-6, max_iter=20000)
    assert st == tca.OK, info
    got = x.cpu().numpy().astype(np.float64)
    rhs = O.scattered_apply_T(b32.astype(np.float64), inst.col0, inst.w, shape)
    kx = O.scattered_normal_apply(got, inst.col0, inst.w, inst.lam)
    rel = np.linalg.norm(rhs - kx) / np.linalg.norm(rhs)
    assert rel <= 1e-6 and abs(info["rel_res_true"] - rel) <= 1e-3 * rel + 1e-12, (rel, info)
    if m <= 1000:
        # cond(K) is below 150 on these two instances (eigenvalues by numpy): error <= cond x rtol
        assert rel_l2(got.ravel(), ref) < 2e-4
    # b from host memory through the same call: the same iterations, the same residual bound.
    xh = np.zeros(shape, dtype=np.float32)
    st2, info2 = plan.solve(b32, xh, rtol=1e-6, max_iter=20000)
    assert st2 == tca.OK and info2["rel_res_true"] <= 1e-6
    assert rel_l2(xh, got) < 1e-5


def test_scattered_plan_refusals():
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_scattered((8, 7, 6), 200, seed=1, lam=1e-2)
    for prec in ("bf16_ir", "tf32_ir"):
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
    # FP32 scattered plans: no preconditioner, no batched solve.
    p32 = _plan(tca, inst, precision="f32")
    b32 = to_dev(np.ones(200), np.float32)
    x32 = torch.zeros((8, 7, 6), dtype=torch.float32, device="cuda")
    st, _ = p32.solve(b32, x32, precond="jacobi", raise_on_error=False)
    assert st == tca.ERR_UNSUPPORTED
    st, _ = tca.solve_batched([p32], [b32], [x32], raise_on_error=False)
    assert st == tca.ERR_UNSUPPORTED
