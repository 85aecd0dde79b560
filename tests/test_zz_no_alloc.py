"""tca_rel_residual_noalloc against the solver's own true residual (GPU, through the C ABI).

The no-alloc entry point is for callers that must not allocate device memory
when they check a solution; it keeps its reduction scratch in a fixed device
array inside the library.  Here it must reproduce the FP64 true relative
residual that tca_solve reports for the same plan, on two calls in a row (the
second call reuses the scratch the first one left behind).  This file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import TOL_F64, lib, need_cuda, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_solver_residual_twice():
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_dense_3d(seed=0)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    plan = tca.plan_from_instance(inst, precision="f64")
    bd = to_dev(b, np.float64)
    x = torch.zeros(inst.shape, dtype=torch.float64, device="cuda")
    # A loose tolerance leaves a residual well above rounding, so the check is sharp.
    st, info = plan.solve(bd, x, rtol=1e-4)
    assert st == tca.OK
    ref = info["rel_res_true"]
    assert 1e-9 < ref <= 1e-4

    # Same FP64 quantities through the existing entry points.
    rhs = torch.empty(inst.shape, dtype=torch.float64, device="cuda")
    kx = torch.empty(inst.shape, dtype=torch.float64, device="cuda")
    plan.apply_T(bd, rhs)
    plan.apply_normal(x, kx)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        tca.rel_residual_noalloc(rhs, kx, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= TOL_F64 * ref, (got, ref)
    # Independent check of the value by the FP64 oracle.
    assert abs(got - O.rel_residual(x.cpu().numpy(), b, mats, inst.lam)) <= 1e-9 * ref


def test_noalloc_rejects_oversized_and_bad_arguments():
    tca = lib()
    torch = need_cuda()
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = tca._lib.tca_rel_residual_noalloc
    assert f(a.data_ptr(), a.data_ptr(), (1 << 27) + 1, out.data_ptr(), None) == tca.ERR_UNSUPPORTED
    assert b"scratch limit" in tca._lib.tca_last_error_string()
    assert f(a.data_ptr(), a.data_ptr(), -1, out.data_ptr(), None) == tca.ERR_INVALID_ARG
    assert f(None, a.data_ptr(), 4, out.data_ptr(), None) == tca.ERR_INVALID_ARG
    assert f(a.data_ptr(), a.data_ptr(), 4, None, None) == tca.ERR_INVALID_ARG
    # n = 0: defined as 0.
    out.fill_(7.0)
    assert f(a.data_ptr(), a.data_ptr(), 0, out.data_ptr(), None) == tca.OK
    torch.cuda.synchronize()
    assert out.item() == 0.0


@pytest.mark.parametrize("n", [3 * 8192 + 17, 160 * 160 * 160 * 8])
def test_noalloc_residual_across_many_blocks_twice(n):
    """Lengths that span many reduction blocks and end in a ragged block: the per-block
    partials in the library's fixed array, the last-block reduction and the counter reset
    all run.  Each length is checked on two calls in a row with different data, then
    once more after a shorter call has left other partials behind, against NumPy's FP64
    norms of the same vectors."""
    tca = lib()
    torch = need_cuda()
    rng = np.random.default_rng(n)
    rhs = rng.standard_normal(n)
    kx1 = rhs + 1e-3 * rng.standard_normal(n)
    kx2 = rhs * (1.0 + 1e-2 * rng.standard_normal(n))
    want = [np.linalg.norm(rhs - k) / np.linalg.norm(rhs) for k in (kx1, kx2)]
    rd = to_dev(rhs, np.float64)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for k, w in zip((kx1, kx2), want):
        tca.rel_residual_noalloc(rd, to_dev(k, np.float64), out)
        torch.cuda.synchronize()
        assert abs(out.item() - w) <= 1e-12 * w, (n, out.item(), w)
    # A short call (one block) in between leaves stale partials in the array.
    short = to_dev(np.ones(100), np.float64)
    tca.rel_residual_noalloc(short, short, out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
    tca.rel_residual_noalloc(rd, to_dev(kx1, np.float64), out)
    torch.cuda.synchronize()
    assert abs(out.item() - want[0]) <= 1e-12 * want[0]


def test_noalloc_binding_rejects_device_buffers_of_the_wrong_kind():
    tca = lib()
    torch = need_cuda()
    a = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="float64"):
        tca.rel_residual_noalloc(a.float(), a, out)
    with pytest.raises(ValueError, match="kx holds"):
        tca.rel_residual_noalloc(a, a[:32], out)
    with pytest.raises(ValueError, match="device memory"):
        tca.rel_residual_noalloc(a, a, out.cpu())
