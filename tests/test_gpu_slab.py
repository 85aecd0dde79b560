"""The slab partition's per-rank pieces on the GPU, through the C ABI: each rank's slab plan
(factor 1 restricted to the extended slab's columns) applies K and A^T exactly like the global
operator on its owned planes, and the CG driver on the library's vector kernels solves the
one-rank case like tca_solve.  The multi-rank exchange itself is tested on CPU ranks
(tests/test_slab.py); this machine's runs have one GPU."""
import numpy as np
import pytest

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import slab, synth
from tests.gpu_common import TOL_F32, lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,world", [((24, 20, 22, 8), 3), ((30, 25, 27), 2), ((18, 12, 10, 4), 2)])
def test_slab_plans_reproduce_the_global_operator_on_owned_planes(shape, world):
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_bspline(shape, seed=88, lam=5e-3, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    part = slab.SlabPartition(shape[0], world)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape).astype(np.float32)
    b = rng.standard_normal(inst.sample_shape).astype(np.float32)
    kx = O.normal_apply(x.astype(np.float64), mats, inst.lam)
    atb = O.apply_T(b.astype(np.float64), mats)
    bd = to_dev(b, np.float32)
    for r in range(world):
        s = part.slab(r)
        g = slab.GpuSlab(part, r, inst.factors, shape, inst.lam)
        xe = to_dev(np.ascontiguousarray(x[s.lo:s.hi]), np.float32)
        q = g.zeros()
        g.apply_K(xe, q)
        assert rel_l2(q[s.owned].cpu().numpy(), kx[s.start:s.stop]) < TOL_F32, r
        rhs = g.rhs(bd)
        assert rel_l2(rhs[s.owned].cpu().numpy(), atb[s.start:s.stop]) < TOL_F32, r


def test_vector_kernels():
    tca = lib()
    torch = need_cuda()
    rng = np.random.default_rng(9)
    n = 3 * 8192 + 17
    a = rng.standard_normal(n).astype(np.float32)
    c = rng.standard_normal(n).astype(np.float32)
    ad, cd = to_dev(a, np.float32), to_dev(c, np.float32)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    tca.vec_dot(ad, cd, out)
    ref = float(np.dot(a.astype(np.float64), c.astype(np.float64)))
    assert abs(out.item() - ref) <= 1e-12 * np.sqrt(n) * np.linalg.norm(a) * np.linalg.norm(c)
    tca.vec_axpby(cd, ad, 0.5, -2.0)
    np.testing.assert_allclose(cd.cpu().numpy(), 0.5 * a - 2.0 * c, rtol=1e-6, atol=1e-6)


def test_one_rank_slab_cg_solves_like_tca_solve():
    tca = lib()
    torch = need_cuda()
    inst = synth.instance_bspline((24, 20, 22, 8), seed=89, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    bd = to_dev(b, np.float32)
    part = slab.SlabPartition(24, 1)
    g = slab.GpuSlab(part, 0, inst.factors, inst.shape, inst.lam)
    x, it, rel = slab.slab_cg(part, 0, g, g.rhs(bd), rtol=1e-6)
    assert rel <= 1e-6
    true_rel = O.rel_residual(x.cpu().numpy(), b.astype(np.float64), mats, inst.lam)
    assert true_rel <= 3e-6, true_rel
    plan = tca.plan_from_instance(inst, precision="f32")
    x2 = torch.zeros(inst.shape, dtype=torch.float32, device="cuda")
    st, info = plan.solve(bd, x2, rtol=1e-6)
    assert abs(info["iters"] - it) <= 2, (info["iters"], it)
    assert rel_l2(x.cpu().numpy(), x2.cpu().numpy()) < 1e-4
