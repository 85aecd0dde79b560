"""Parity of the DFT over several modes (Table 1, complex data as two real tensors) with the oracle.

``tca_apply_dft`` against ``oracle.dft`` (the separable definition with explicit DFT matrices,
pinned to numpy's FFT): orders 1 to 4, one to four transformed modes, real and complex inputs,
forward and inverse, FP32 and FP64; and the inverse undoing the forward on the GPU.
Tolerances: FP64 1e-12; FP32 2e-5 (the dense products run in 3xTF32, about 2^-21 relative per
product, over at most four modes of at most 20 terms).
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from tests.gpu_common import TOL_F32, lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    ((12, 10, 8), (0, 1, 2)),
    ((9, 7, 5, 6), (1, 3)),
    ((6, 5, 8, 3), (0, 1, 2, 3)),
    ((16, 12), (0,)),
    ((20,), (0,)),
    ((4, 20, 3, 9), (2,)),
]


@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("complex_in", [False, True])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("shape,modes", CASES)
def test_dft_matches_oracle(shape, modes, prec, complex_in, inverse):
    tca = lib()
    torch = need_cuda()
    dt = np.float64 if prec == "f64" else np.float32
    tdt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(80)
    re = rng.standard_normal(shape).astype(dt)
    im = rng.standard_normal(shape).astype(dt) if complex_in else None
    ore = torch.empty(shape, dtype=tdt, device="cuda")
    oim = torch.empty(shape, dtype=tdt, device="cuda")
    tca.apply_dft(to_dev(re, dt), None if im is None else to_dev(im, dt), ore, oim, modes, inverse=inverse)
    rr, ri = O.dft(re.astype(np.float64), None if im is None else im.astype(np.float64), modes, inverse=inverse)
    got = np.concatenate([ore.cpu().numpy().ravel(), oim.cpu().numpy().ravel()])
    tol = 1e-12 if prec == "f64" else TOL_F32
    assert rel_l2(got, np.concatenate([rr.ravel(), ri.ravel()])) < tol


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_dft_inverse_undoes_forward(prec):
    tca = lib()
    torch = need_cuda()
    dt = np.float64 if prec == "f64" else np.float32
    tdt = torch.float64 if prec == "f64" else torch.float32
    shape = (10, 12, 6, 4)
    rng = np.random.default_rng(81)
    re, im = to_dev(rng.standard_normal(shape), dt), to_dev(rng.standard_normal(shape), dt)
    fr, fi = (torch.empty(shape, dtype=tdt, device="cuda") for _ in range(2))
    br, bi = (torch.empty(shape, dtype=tdt, device="cuda") for _ in range(2))
    tca.apply_dft(re, im, fr, fi, (0, 1, 3))
    tca.apply_dft(fr, fi, br, bi, (0, 1, 3), inverse=True)
    tol = 1e-12 if prec == "f64" else TOL_F32
    assert rel_l2(br.cpu().numpy(), re.cpu().numpy()) < tol
    assert rel_l2(bi.cpu().numpy(), im.cpu().numpy()) < tol


def test_dft_refusals():
    tca = lib()
    torch = need_cuda()
    x = torch.zeros((4, 300), dtype=torch.float32, device="cuda")
    y, z = torch.empty_like(x), torch.empty_like(x)
    with pytest.raises(tca.TcaError) as e:
        tca.apply_dft(x, None, y, z, (1,))  # a transformed mode longer than 256
    assert e.value.status == tca.ERR_UNSUPPORTED
    with pytest.raises(tca.TcaError) as e:
        tca.apply_dft(x, None, y, y, (0,))  # the outputs alias
    assert e.value.status == tca.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        tca.apply_dft(x, None, y, torch.empty((300, 4), dtype=torch.float32, device="cuda"), (0,))
