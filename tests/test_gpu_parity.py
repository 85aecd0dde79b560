"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Sizes span several tiles of every kernel and leave ragged tails; each case uses
the same seeded inputs on both sides.  Tolerances: relative L2 error <= 1e-12
for FP64 plans and <= 2e-5 for FP32 plans (derivation in the design notes).
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import TOL_F32, TOL_F64, empty_dev, lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _bspline(shape, seed, lam=1e-3):
    return synth.instance_bspline(shape, seed=seed, lam=lam, with_truth=False)


def _dense(shape, seed, lam=1e-2):
    rng = np.random.default_rng(seed)
    facs = []
    for n in shape:
        m = int(np.ceil(1.5 * n))
        facs.append(synth.Factor("dense", m, n, a=synth.dense_gaussian_factor(m, n, rng)))
    return synth.Instance(tuple(shape), facs, None, None, lam, seed)


CASES = [
    ("bspline", (40, 37, 29, 8), "f32"),     # fused sweep, n4 = 8, ragged tiles
    ("bspline", (23, 50, 45, 4), "f32"),     # fused sweep, n4 = 4
    ("bspline", (33, 41, 70), "f32"),        # order 3: fused sweep with n4 = 1
    ("bspline", (12, 13, 11, 16), "f32"),    # n4 = 16: generic sweeps
    ("bspline", (9, 10, 7, 5), "f32"),       # n4 = 5: generic sweeps
    ("bspline", (17, 14, 19, 3), "f64"),
    ("dense", (13, 11, 9, 4), "f32"),
    ("dense", (16, 16, 16), "f64"),
    ("dense", (20, 7, 33), "f32"),
]


def _inst(kind, shape, seed):
    return _bspline(shape, seed) if kind == "bspline" else _dense(shape, seed)


@pytest.mark.parametrize("kind,shape,prec", CASES)
def test_apply_and_apply_T(kind, shape, prec):
    tca = lib()
    inst = _inst(kind, shape, 100 + len(shape))
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision=prec)
    dt = plan.dtype
    rng = np.random.default_rng(7)
    x = rng.standard_normal(inst.shape).astype(dt)
    y = rng.standard_normal(inst.sample_shape).astype(dt)
    ax = empty_dev(inst.sample_shape, dt)
    aty = empty_dev(inst.shape, dt)
    plan.apply(to_dev(x, dt), ax)
    plan.apply_T(to_dev(y, dt), aty)
    tol = TOL_F64 if prec == "f64" else TOL_F32
    assert rel_l2(ax.cpu().numpy(), O.apply(x, mats)) < tol
    assert rel_l2(aty.cpu().numpy(), O.apply_T(y, mats)) < tol


@pytest.mark.parametrize("kind,shape,prec", CASES)
def test_normal_operator(kind, shape, prec):
    tca = lib()
    inst = _inst(kind, shape, 200 + len(shape))
    inst.lam = 0.05
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision=prec)
    dt = plan.dtype
    rng = np.random.default_rng(8)
    x = rng.standard_normal(inst.shape).astype(dt)
    kx = empty_dev(inst.shape, dt)
    plan.apply_normal(to_dev(x, dt), kx)
    ref = O.normal_apply(x, mats, inst.lam)
    tol = TOL_F64 if prec == "f64" else TOL_F32
    got = kx.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) < tol


@pytest.mark.parametrize("shape", [(1, 30, 25, 8), (7, 22, 22, 8), (300, 22, 23, 8), (9, 21, 40, 8)])
def test_fused_sweep_edge_shapes(shape):
    """The warp-specialised sweep at its edges: one plane along mode 1, n2 = n3 = 22 (the
    smallest extent copied by TMA boxes), a long mode 1 (many chunks), and n2 = 21 (the
    cp.async halo path); plain operator and, through 5 CG iterations, the CG-mode sweep."""
    tca = lib()
    inst = synth.instance_bspline(shape, seed=680, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision="f32")
    rng = np.random.default_rng(681)
    x = rng.standard_normal(inst.shape).astype(np.float32)
    kx = empty_dev(inst.shape, np.float32)
    plan.apply_normal(to_dev(x, np.float32), kx)
    ref = O.normal_apply(x.astype(np.float64), mats, inst.lam)
    assert rel_l2(kx.cpu().numpy(), ref) < TOL_F32
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    xs = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), xs, rtol=1e-14, max_iter=5, raise_on_error=False)
    assert info["iters"] == 5
    ref5 = O.solve(b.astype(np.float64), mats, inst.lam, rtol=0.0, max_iter=5).x
    assert rel_l2(xs.cpu().numpy(), ref5) < 1e-4


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_single_mode_products(mode, op):
    tca = lib()
    inst = _bspline((21, 18, 35, 8), 300)
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision="f32")
    dims = list(inst.shape)
    if op == tca.OP_FACTOR_T:
        dims[mode] = inst.factors[mode].m
    a = mats[mode]
    mat = a if op == tca.OP_FACTOR else a.T if op == tca.OP_FACTOR_T else a.T @ a
    out_dims = list(dims)
    out_dims[mode] = mat.shape[0]
    rng = np.random.default_rng(9)
    x = rng.standard_normal(dims).astype(np.float32)
    y = empty_dev(out_dims, np.float32)
    plan.apply_mode(mode, op, dims, to_dev(x, np.float32), y)
    assert rel_l2(y.cpu().numpy(), O.mode_product(x, mat, mode)) < TOL_F32


def test_ragged_and_degenerate_shapes():
    """Modes of size 1 and 2 (no regulariser), single-sample factors, prime sizes."""
    tca = lib()
    rng = np.random.default_rng(10)
    for shape in [(1, 5, 7), (2, 3, 1, 4), (7, 1, 13, 8), (3, 17, 2)]:
        facs = []
        for n in shape:
            m = max(1, int(round(1.5 * n)))
            col0, w, _ = synth.bspline_factor_ell4(n, m, rng)
            facs.append(synth.Factor("ell4", m, n, col0=col0, w=w))
        inst = synth.Instance(shape, facs, None, None, 0.1, 0)
        mats = [f.dense() for f in facs]
        for prec in ("f32", "f64"):
            plan = tca.plan_from_instance(inst, precision=prec)
            dt = plan.dtype
            x = rng.standard_normal(shape).astype(dt)
            kx = empty_dev(shape, dt)
            plan.apply_normal(to_dev(x, dt), kx)
            tol = TOL_F64 if prec == "f64" else TOL_F32
            assert rel_l2(kx.cpu().numpy(), O.normal_apply(x, mats, 0.1)) < tol, (shape, prec)


def test_solve_dense_3d_fp64_matches_cholesky():
    """Dense 16^3 problem, FP64, CG to 1e-10 vs the Cholesky solve of the reshaped system."""
    tca = lib()
    inst = synth.instance_dense_3d(seed=0)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    plan = tca.plan_from_instance(inst, precision="f64")
    x = empty_dev(inst.shape, np.float64)
    st, info = plan.solve(to_dev(b, np.float64), x, rtol=1e-10)
    assert st == tca.OK
    x_direct = O.direct_solve(b, mats, inst.lam, inst.shape)
    assert rel_l2(x.cpu().numpy(), x_direct) < 1e-8
    assert info["rel_res_true"] <= 1e-10
    assert O.rel_residual(x.cpu().numpy(), b, mats, inst.lam) <= 1e-10


@pytest.mark.parametrize("shape", [(32, 28, 24, 8), (30, 26, 40), (16, 18, 14, 16), (20, 22, 18, 4)])
def test_solve_bspline_fp32(shape):
    """FP32 CG to a true relative residual of 1e-6; solution matches the FP64 oracle's."""
    tca = lib()
    inst = synth.instance_bspline(shape, seed=400 + len(shape), dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6)
    assert st == tca.OK, info
    got = x.cpu().numpy()
    # The oracle's own verdict on the GPU solution (FP64, long way).
    assert O.rel_residual(got, b.astype(np.float64), mats, inst.lam) <= 1.5e-6
    ref = O.solve(b.astype(np.float64), mats, inst.lam, rtol=1e-12).x
    assert rel_l2(got, ref) < 5e-5
    assert info["rel_res_true"] <= 1e-6
    assert abs(info["rel_res_true"] - O.rel_residual(got, b.astype(np.float64), mats, inst.lam)) < 1e-7


@pytest.mark.parametrize("prec", ["f32", "f64", "tf32_ir"])
def test_solve_host_buffers_match_device(prec):
    """Host (pageable and pinned) buffers give the device-buffer result bit for bit; the
    plain plans copy x back under their final true-residual check, the _IR plan after."""
    tca = lib()
    torch = need_cuda()
    dt = np.float64 if prec == "f64" else np.float32
    tdt = torch.float64 if prec == "f64" else torch.float32
    inst = synth.instance_bspline((24, 20, 22, 8), seed=500, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(dt)
    plan = tca.plan_from_instance(inst, precision=prec)
    xd = empty_dev(inst.shape, dt)
    plan.solve(to_dev(b, dt), xd, rtol=1e-6)
    xh = np.zeros(inst.shape, dt)
    st, info = plan.solve(np.ascontiguousarray(b), xh, rtol=1e-6)
    assert st == tca.OK
    np.testing.assert_array_equal(xh, xd.cpu().numpy())
    pinned = torch.from_numpy(b).pin_memory()
    xp = torch.zeros(inst.shape, dtype=tdt).pin_memory()
    plan.solve(pinned, xp, rtol=1e-6)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(xp.numpy(), xd.cpu().numpy())


def test_solve_with_initial_guess_and_max_iter():
    tca = lib()
    inst = synth.instance_bspline((20, 18, 16, 4), seed=600, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6)
    full_iters = info["iters"]
    # Warm start from the solution: converges at once.
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-5, x0_given=True)
    assert st == tca.OK and info["iters"] <= 2
    # max_iter cap reports NOT_CONVERGED with x still filled.
    x2 = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x2, rtol=1e-9, max_iter=5, raise_on_error=False)
    assert st == tca.ERR_NOT_CONVERGED and info["iters"] == 5
    assert np.all(np.isfinite(x2.cpu().numpy()))
    assert full_iters > 5


@pytest.mark.parametrize("shape,prec,tol", [((20, 18, 16, 8), "f32", 1e-4),   # fused sweep
                                             ((19, 12, 15, 4), "f32", 1e-4),   # fused sweep, n4 = 4
                                             ((17, 14, 19, 3), "f64", 1e-10)])  # generic FP64 path
def test_partial_iterates_match_oracle(shape, prec, tol):
    """x after k CG iterations (max_iter = k) equals the oracle's k-th iterate.

    The solution update is applied once per group of four iterations; k = 1 .. 9
    stops at every position of a group, so a term left out, applied twice or
    taken with the wrong direction shows as an O(1) error here."""
    tca = lib()
    dt = np.float32 if prec == "f32" else np.float64
    inst = synth.instance_bspline(shape, seed=650, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(dt)
    plan = tca.plan_from_instance(inst, precision=prec)
    for k in range(1, 10):
        x = empty_dev(inst.shape, dt)
        st, info = plan.solve(to_dev(b, dt), x, rtol=1e-14, max_iter=k, raise_on_error=False)
        assert st == tca.ERR_NOT_CONVERGED and info["iters"] == k
        ref = O.solve(b.astype(np.float64), mats, inst.lam, rtol=0.0, max_iter=k).x
        assert rel_l2(x.cpu().numpy(), ref) < tol, k


@pytest.mark.parametrize("kind,shape", [("bspline", (20, 18, 16, 8)), ("bspline", (19, 12, 15, 4)),
                                        ("bspline", (33, 41, 70)), ("bspline", (12, 13, 11, 16)),
                                        ("bspline", (9, 10, 7, 5)), ("dense", (13, 11, 9, 4))])
def test_true_residual_is_fp64_accurate(kind, shape):
    """The reported true residual of an FP32 solve (A^T b and K x in double-float)
    equals the oracle's FP64 residual of the same x to ~1e-9 relative.

    Stopped after 3 iterations the residual is ~1e-2 of ||A^T b||; an FP32
    evaluation would be off by ~1e-5 relative there, so this pins the
    double-float products (every layout of the mode kernels and both
    residual kernels) rather than the iteration."""
    tca = lib()
    inst = _inst(kind, shape, 660)
    mats = [f.dense() for f in inst.factors]
    rng = np.random.default_rng(661)
    b = rng.standard_normal(inst.sample_shape).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-14, max_iter=3, raise_on_error=False)
    assert st == tca.ERR_NOT_CONVERGED
    ref = O.rel_residual(x.cpu().numpy().astype(np.float64), b.astype(np.float64), mats, inst.lam)
    assert abs(info["rel_res_true"] - ref) <= 1e-9 * ref + 1e-15, (info["rel_res_true"], ref)


def test_zero_rhs():
    tca = lib()
    inst = synth.instance_bspline((10, 9, 8, 4), seed=700, with_truth=False)
    plan = tca.plan_from_instance(inst, precision="f32")
    b = np.zeros(inst.sample_shape, np.float32)
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x)
    assert st == tca.OK and info["iters"] == 0
    assert np.all(x.cpu().numpy() == 0)


@pytest.mark.slow
def test_full_size_normal_operator_sampled():
    """160x160x160x8 with 240^3x12 B-spline factors (the timed workload): K x on sampled points."""
    tca = lib()
    inst = synth.instance_bspline((160, 160, 160, 8), seed=2, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    plan = tca.plan_from_instance(inst, precision="f32")
    rng = np.random.default_rng(11)
    x = rng.standard_normal(inst.shape, dtype=np.float32)
    kx = empty_dev(inst.shape, np.float32)
    plan.apply_normal(to_dev(x, np.float32), kx)
    got = kx.cpu().numpy()
    pts = [tuple(int(rng.integers(0, n)) for n in inst.shape) for _ in range(40)]
    pts += [(0, 0, 0, 0), (159, 159, 159, 7), (0, 159, 3, 7), (80, 0, 159, 0)]
    for pt in pts:
        ref = O.normal_apply_at(x, mats, inst.lam, pt)
        assert abs(got[pt] - ref) <= 1e-5 * (abs(ref) + 1.0), (pt, got[pt], ref)


@pytest.mark.slow
def test_full_size_solve_true_residual_by_oracle():
    """The timed workload end to end (160x160x160x8 unknowns, 240^3 x 12 B-spline samples,
    lambda 1e-3, rtol 1e-6; the TMA CG sweep, the grouped update and the device-side pass
    loop that bench.py times): the oracle's own FP64 true residual of the GPU solution
    meets the tolerance, and the double-float value the solve reports agrees with it to
    ~1e-6 relative (an FP32 evaluation would be off by ~1e-1 at this residual level)."""
    tca = lib()
    inst = synth.instance_bspline((160, 160, 160, 8), seed=2, lam=1e-3, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6)
    assert st == tca.OK, info
    ref = O.rel_residual(x.cpu().numpy().astype(np.float64), b.astype(np.float64), mats, inst.lam)
    assert ref <= 1.5e-6
    assert abs(info["rel_res_true"] - ref) <= 1e-6 * ref, (info["rel_res_true"], ref)


@pytest.mark.parametrize("shape", [(40, 30, 50, 8), (17, 96, 33), (64, 5, 9, 4)])
def test_dense_products_on_tensor_cores(shape):
    """Dense mode products run on tcgen05: a TF32 plan shows TF32 rounding (1e-5 .. 5e-3 relative),
    the FP32 plan's 3xTF32 split stays at FP32 level; several 128-row tiles, padded K and N."""
    tca = lib()
    inst = _dense(shape, 800 + len(shape))
    mats = [f.dense() for f in inst.factors]
    rng = np.random.default_rng(12)
    x = rng.standard_normal(inst.shape).astype(np.float32)
    ref = O.apply(x, mats)
    errs = {}
    for prec in ("f32", "tf32_ir"):
        plan = tca.plan_from_instance(inst, precision=prec)
        ax = empty_dev(inst.sample_shape, np.float32)
        plan.apply(to_dev(x, np.float32), ax)
        errs[prec] = rel_l2(ax.cpu().numpy(), ref)
    assert errs["f32"] < TOL_F32, errs
    assert 1e-5 < errs["tf32_ir"] < 5e-3, errs


@pytest.mark.parametrize("kind,shape,prec", [("dense", (20, 18, 16, 4), "tf32_ir"),
                                             ("dense", (24, 30, 20), "tf32_ir"),
                                             ("bspline", (24, 20, 22, 8), "bf16_ir"),
                                             ("bspline", (20, 22, 18, 4), "tf32_ir")])
def test_solve_mixed_precision_refinement(kind, shape, prec):
    """Reduced-precision inner CG + FP64-accurate refinement reaches the FP64 oracle's solution."""
    tca = lib()
    if kind == "dense":
        inst = _dense(shape, 900 + len(shape), lam=1e-2)
        rng = np.random.default_rng(5)
        inst.x_true = synth.smooth_random_field(shape, 3.0, rng, dtype=np.float64)
        inst.noise = 0.01 * rng.standard_normal(inst.sample_shape)
    else:
        inst = synth.instance_bspline(shape, seed=910 + len(shape), dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision=prec)
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, inner_rtol=1e-2)
    assert st == tca.OK, info
    assert info["refinements"] >= 1
    got = x.cpu().numpy()
    rel = O.rel_residual(got, b.astype(np.float64), mats, inst.lam)
    assert rel <= 1.5e-6, (rel, info)
    assert abs(info["rel_res_true"] - rel) < 1e-7
    ref = O.solve(b.astype(np.float64), mats, inst.lam, rtol=1e-12).x
    assert rel_l2(got, ref) < 1e-4


def test_bounded_wait_gives_up_and_context_survives():
    """A device wait that cannot succeed gives up after its poll limit, the
    status reaches the host as ERR_TIMEOUT, the flag clears, and the context
    keeps working (a solve right after is correct and reports OK)."""
    tca = lib()
    assert tca.check_timeout() == tca.OK
    for polls in (0, 1, 1000):
        assert tca.wait_selftest(polls) == tca.ERR_TIMEOUT
        assert tca.check_timeout() == tca.OK  # cleared by the report
    assert tca.wait_selftest(-1) == tca.ERR_INVALID_ARG
    inst = synth.instance_bspline((24, 22, 23, 8), seed=670, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(inst.shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6)
    assert st == tca.OK
    assert O.rel_residual(x.cpu().numpy(), b.astype(np.float64), mats, inst.lam) <= 1.5e-6
