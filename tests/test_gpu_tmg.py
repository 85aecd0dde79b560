"""Parity of the tensor multigrid preconditioner (two-grid V-cycle, Sec. 4.2, Fig. 3) with the oracle.

One cycle z = V r through ``tca_tmg_apply`` is compared element by element with
``oracle.tmg_vcycle`` on the same r, with the same smoothing steps, coarsened modes and
Chebyshev interval (lambda_max of D^-1 K from power steps of the oracle's own operator,
passed to both sides); then the preconditioned CG iterate by iterate against ``oracle.pcg``
driven by that cycle, and a solve with every default (the library's own lambda_max estimate,
coarse tolerance 0.3) against the oracle's verdict on its residual.

Tolerances.  FP64 plans: both sides solve the coarse system to 1e-13, so their cycles differ
by at most that residual times cond(K_c) (555 for the (9, 8, 7, 4) case): 1e-8.  FP32 plans:
every product and vector update rounds to 2^-24, and the coarse solve amplifies a relative
perturbation of its right-hand side by up to cond(K_c) (778 for the (12, 10, 9, 8) case),
so 800 x 6e-8 = 5e-5 at worst for one cycle; 5e-4 allows a tenfold margin.
"""
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


def _inst(kind, shape, seed, lam, dtype=np.float64):
    if kind == "bspline":
        return synth.instance_bspline(shape, seed=seed, lam=lam, dtype=dtype)
    return _dense(shape, seed, lam)


def _oracle_parts(inst, mask):
    mats = [f.dense() for f in inst.factors]
    shape = inst.shape
    kop = lambda v: O.normal_apply(v, mats, inst.lam)
    dia = O.jacobi_diagonal(mats, inst.lam, shape)
    prol = [O.tmg_prolongation(n) if (mask >> k) & 1 else np.eye(n) for k, n in enumerate(shape)]
    # lambda_max of D^-1 K by power steps on the oracle's operator (the value both sides take).
    v = np.random.default_rng(3).standard_normal(shape)
    lmax = 0.0
    for _ in range(60):
        v = kop(v) / dia
        lmax = float(np.linalg.norm(v))
        v /= lmax
    return mats, kop, dia, prol, lmax


def _oracle_cycle(kop, dia, prol, nu, lmax):
    return lambda r: O.tmg_vcycle(r, kop, dia, prol, nu=max(nu, 0), lam_lo=lmax / 30, lam_hi=1.05 * lmax,
                                  coarse_rtol=1e-13)


CYCLE_CASES = [
    # kind, shape, precision, coarsened modes, smoothing steps (-1: none)
    ("bspline", (9, 8, 7, 4), "f64", 0b0111, -1),   # bare coarse correction: P (P^T K P)^-1 P^T r
    ("bspline", (9, 8, 7, 4), "f64", 0b0111, 1),    # odd and even lengths: coarse 5, 4, 4
    ("bspline", (9, 8, 7, 4), "f64", 0b0111, 2),
    ("bspline", (11, 10, 9, 8), "f64", 0b0101, 3),  # modes 2 and 4 kept
    ("dense", (10, 9, 7), "f64", 0b111, 2),         # dense factors, order 3 (generic operator)
    ("bspline", (12, 10, 9, 8), "f32", 0b0111, 2),  # FP32 fused sweep (n4 = 8)
    ("bspline", (14, 13, 12, 4), "f32", 0b1111, 2),  # every mode coarsened, n4 = 4 sweep
]


@pytest.mark.parametrize("kind,shape,prec,mask,nu", CYCLE_CASES)
def test_tmg_cycle_matches_oracle(kind, shape, prec, mask, nu):
    tca = lib()
    dt = np.float64 if prec == "f64" else np.float32
    inst = _inst(kind, shape, 900, 1e-3)
    mats, kop, dia, prol, lmax = _oracle_parts(inst, mask)
    plan = tca.plan_from_instance(inst, precision=prec)
    r = np.random.default_rng(11).standard_normal(shape)
    z = empty_dev(shape, dt)
    plan.tmg_apply(to_dev(r, dt), z, nu=nu, coarse_rtol=1e-13 if prec == "f64" else 1e-9, lambda_max=lmax,
                   coarsen_mask=mask)
    ref = _oracle_cycle(kop, dia, prol, nu, lmax)(r.astype(dt).astype(np.float64))
    tol = 1e-8 if prec == "f64" else 5e-4
    assert rel_l2(z.cpu().numpy(), ref) < tol
    info = plan.tmg_info()
    assert info["lambda_max"] == lmax and info["coarse_iters"] > 0


@pytest.mark.parametrize("kind,shape,mask", [("bspline", (9, 8, 7, 4), 0b0111), ("dense", (10, 9, 7), 0b111)])
def test_tmg_pcg_partial_iterates_match_oracle(kind, shape, mask):
    """FP64 plans: the GPU's preconditioned CG after k iterations equals the oracle's pcg with the
    oracle's cycle as M^-1 (k = 1 .. 5, every position of the grouped solution update)."""
    tca = lib()
    inst = _inst(kind, shape, 910, 1e-3)
    mats, kop, dia, prol, lmax = _oracle_parts(inst, mask)
    b = O.apply(inst.x_true, mats) + inst.noise
    rhs = O.apply_T(b, mats)
    cyc = _oracle_cycle(kop, dia, prol, 2, lmax)
    plan = tca.plan_from_instance(inst, precision="f64")
    for k in (1, 2, 3, 4, 5):
        x = empty_dev(inst.shape, np.float64)
        st, info = plan.solve(to_dev(b, np.float64), x, rtol=1e-14, max_iter=k, raise_on_error=False,
                              precond="tmg", tmg_nu=2, tmg_coarse_rtol=1e-13, tmg_lambda_max=lmax,
                              tmg_coarsen_mask=mask)
        assert st == tca.ERR_NOT_CONVERGED and info["iters"] == k
        ref = O.pcg(kop, cyc, rhs, rtol=0.0, max_iter=k).x
        assert rel_l2(x.cpu().numpy(), ref) < 1e-8, k


def test_tmg_solve_meets_tolerance_in_fewer_iterations():
    """FP32 plan, every default (modes of at least 16 points coarsened, three smoothing steps, the
    library's own lambda_max estimate, coarse tolerance 0.3): the solve meets a true relative
    residual of 1e-6 by the oracle's verdict in under half the plain CG's iterations (the TMA halo
    path of the fused sweep: n2, n3 >= 22), and the estimate lies within 5 % of the oracle's."""
    tca = lib()
    shape = (24, 24, 24, 8)
    inst = _inst("bspline", shape, 920, 1e-3, dtype=np.float32)
    mats, kop, dia, prol, lmax = _oracle_parts(inst, 0b0111)
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = empty_dev(shape, np.float32)
    st, info = plan.solve(to_dev(b, np.float32), x, rtol=1e-6, precond="tmg")
    assert st == tca.OK, info
    assert info["rel_res_true"] <= 1e-6
    assert O.rel_residual(x.cpu().numpy(), b.astype(np.float64), mats, inst.lam) <= 1.5e-6
    est = plan.tmg_info()
    assert abs(est["lambda_max"] - lmax) <= 0.05 * lmax, (est, lmax)
    assert est["coarse_iters"] > 0
    x0 = empty_dev(shape, np.float32)
    st0, info0 = plan.solve(to_dev(b, np.float32), x0, rtol=1e-6)
    assert st0 == tca.OK
    assert 2 * info["iters"] <= info0["iters"], (info["iters"], info0["iters"])


def test_tmg_refusals():
    tca = lib()
    inst = _inst("bspline", (9, 8, 7, 4), 930, 1e-3)
    plan = tca.plan_from_instance(inst, precision="f64")
    r = to_dev(np.ones(inst.shape), np.float64)
    z = empty_dev(inst.shape, np.float64)
    for kw, want in (({"coarsen_mask": 0b10000}, tca.ERR_INVALID_ARG),   # a mode the plan lacks
                     ({"coarsen_mask": 0}, tca.ERR_UNSUPPORTED),         # no mode of 16 points
                     ({"coarsen_mask": 0b0111, "coarse_rtol": -1.0}, tca.ERR_INVALID_ARG),
                     ({"coarsen_mask": 0b0111, "lambda_max": -2.0}, tca.ERR_INVALID_ARG),
                     ({"coarsen_mask": 0b0111, "nu": 65}, tca.ERR_INVALID_ARG)):
        with pytest.raises(tca.TcaError) as e:
            plan.tmg_apply(r, z, **kw)
        assert e.value.status == want, kw
    # Not in a batched graph; not on bfloat16 plans.
    b = to_dev(O.apply(inst.x_true, [f.dense() for f in inst.factors]) + inst.noise, np.float32)
    fplan = tca.plan_from_instance(inst, precision="f32")
    xs = [empty_dev(inst.shape, np.float32)]
    st, _ = tca.solve_batched([fplan], [b], xs, precond="tmg", raise_on_error=False)
    assert st == tca.ERR_UNSUPPORTED
    binst = _inst("bspline", (16, 16, 16, 8), 931, 1e-3, dtype=np.float32)
    bplan = tca.plan_from_instance(binst, precision="bf16_ir")
    bb = to_dev(np.zeros(binst.sample_shape), np.float32)
    st, _ = bplan.solve(bb, empty_dev(binst.shape, np.float32), precond="tmg", raise_on_error=False)
    assert st == tca.ERR_UNSUPPORTED
