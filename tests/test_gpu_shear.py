"""Parity of the one-dimensional shear transform (Table 1 rotation) with the oracle.

``tca_apply_shear`` against ``oracle.shear`` element by element: modes a and b in every
relative position (a before or after b, either of them the fastest mode), fractional slopes of
both signs, shifts that move whole lines off the grid, lines of one point, 2D to 4D, both
kernels, FP32 and FP64; then three shears rotating planes of a 4D volume against the oracle's
three shears.  Tolerances: FP64 1e-13; FP32 2e-6 (at most four FP32 products per output with
weights rounded to FP32: 4 x 2 x 2^-24 relative to the largest input, with margin).
"""
import numpy as np
import pytest

from oracle import tca_oracle as O
from tests.gpu_common import lib, need_cuda, rel_l2, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    # shape, mode_a, mode_b, slope, center
    ((17, 13), 0, 1, 0.37, 6.0),
    ((17, 13), 1, 0, -0.81, 8.5),
    ((9, 11, 6), 2, 0, 0.25, 4.0),       # a is the fastest mode
    ((9, 11, 6), 0, 2, -1.6, 2.5),       # b is the fastest mode
    ((7, 8, 5, 6), 1, 3, 0.5, 0.0),
    ((7, 8, 5, 6), 3, 1, 2.75, 3.0),     # shifts past the line's end for most i_b
    ((5, 1, 9), 1, 2, 0.3, 4.0),         # lines of one point
    ((12, 10, 8, 4), 2, 1, -0.125, 4.5),  # 16-byte vectors along the fastest mode
    ((6, 9, 12), 0, 1, 0.6, 3.0),
    ((10, 7, 5, 8), 1, 0, -0.45, 2.0),
]


@pytest.mark.parametrize("kind", ["linear", "cubic"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("shape,mode_a,mode_b,slope,center", CASES)
def test_shear_matches_oracle(shape, mode_a, mode_b, slope, center, prec, kind):
    tca = lib()
    torch = need_cuda()
    dt = np.float64 if prec == "f64" else np.float32
    x = np.random.default_rng(60).standard_normal(shape).astype(dt)
    y = torch.full(shape, float("nan"), dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")
    tca.apply_shear(to_dev(x, dt), y, mode_a, mode_b, slope, center, kind=kind)
    ref = O.shear(x.astype(np.float64), mode_a, mode_b, slope, center, kind=tca.SHEAR_KINDS[kind])
    got = y.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    tol = 1e-13 if prec == "f64" else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * max(np.max(np.abs(x)), 1.0) * 4


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_three_shears_rotate_planes_like_the_oracle(prec):
    """Rotation of the (mode 1, mode 2) planes of a 4D volume by 30 degrees with three shears
    (slopes tan 15, -sin 30, tan 15 about the planes' centre) against the oracle's three shears."""
    tca = lib()
    torch = need_cuda()
    dt = np.float64 if prec == "f64" else np.float32
    shape, t = (3, 41, 37, 4), np.deg2rad(30.0)
    c = (shape[1] - 1) / 2.0, (shape[2] - 1) / 2.0
    x = np.random.default_rng(61).standard_normal(shape).astype(dt)
    tdt = torch.float64 if prec == "f64" else torch.float32
    a, b = to_dev(x, dt), torch.empty(shape, dtype=tdt, device="cuda")
    tca.apply_shear(a, b, 1, 2, np.tan(t / 2), c[1], kind="cubic")
    tca.apply_shear(b, a, 2, 1, -np.sin(t), c[0], kind="cubic")
    tca.apply_shear(a, b, 1, 2, np.tan(t / 2), c[1], kind="cubic")
    ref = O.shear(x.astype(np.float64), 1, 2, np.tan(t / 2), c[1], kind=3)
    ref = O.shear(ref, 2, 1, -np.sin(t), c[0], kind=3)
    ref = O.shear(ref, 1, 2, np.tan(t / 2), c[1], kind=3)
    assert rel_l2(b.cpu().numpy(), ref) < (1e-13 if prec == "f64" else 1e-6)


def test_shear_refuses_bad_buffers():
    tca = lib()
    torch = need_cuda()
    x = torch.zeros((4, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        tca.apply_shear(x, torch.zeros((5, 4), dtype=torch.float32, device="cuda"), 0, 1, 0.5, 2.0)
    with pytest.raises(tca.TcaError) as e:
        tca.apply_shear(x, x, 0, 1, 0.5, 2.0)
    assert e.value.status == tca.ERR_INVALID_ARG
    with pytest.raises(tca.TcaError) as e:
        tca.apply_shear(x, torch.zeros((4, 5), dtype=torch.float32), 0, 1, 0.5, 2.0)  # host output
    assert e.value.status == tca.ERR_INVALID_ARG
