"""Other separable factor types of Table 1 on the GPU, through the C ABI: the orthonormal
DCT-II (a dense factor, tensor-core mode products), an FIR filter (a banded Toeplitz factor in
ELL-4 form), up- and downsampling (rectangular ELL-4 factors), and the DFT along one mode as its
real and imaginary parts (two real dense factors).

Each is compared with a library routine that needs no oracle - scipy.fft.dct / numpy.fft.fft,
scipy.ndimage.correlate1d, numpy interpolation - and with the oracle's mode product.  The paper's
rotation by 1D shears shifts each line by an amount that depends on another mode (a factor that
varies along the tensor), which a separable transformation with one factor per mode cannot
express; it is not built.
"""
import numpy as np
import pytest
from scipy import fft as sfft
from scipy import ndimage

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth
from tests.gpu_common import TOL_F32, empty_dev, lib, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _dct(n):
    k = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    c = np.cos(np.pi * k * (2 * i + 1) / (2 * n)) * np.sqrt(2.0 / n)
    c[0, :] = np.sqrt(1.0 / n)
    return c


def _identity(tca, n):
    """Identity as an ELL-4 factor (one tap per row)."""
    w = np.zeros((n, 4))
    w[:, 0] = 1.0
    return tca.Factor(tca.FACTOR_ELL4, n, n, w, np.arange(n, dtype=np.int32))


def _dense_identity(tca, n):
    return tca.Factor(tca.FACTOR_DENSE, n, n, np.eye(n))


@pytest.mark.parametrize("shape,axis", [((24, 20, 22, 8), 1), ((33, 18, 40), 2), ((16, 12, 10, 8), 0)])
def test_dct_factor_on_tensor_cores_equals_scipy_dct(shape, axis):
    tca = lib()
    n = shape[axis]
    facs = [tca.Factor(tca.FACTOR_DENSE, n, n, _dct(n)) if k == axis else _dense_identity(tca, shape[k])
            for k in range(len(shape))]
    plan = tca.Plan(shape, facs, lam=0.0, precision="f32")
    rng = np.random.default_rng(21)
    x = rng.standard_normal(shape).astype(np.float32)
    y = empty_dev(shape, np.float32)
    plan.apply(to_dev(x, np.float32), y)
    ref = sfft.dct(x.astype(np.float64), type=2, norm="ortho", axis=axis)
    assert rel_l2(y.cpu().numpy(), ref) < TOL_F32
    # The transpose of the orthonormal DCT is its inverse.
    z = empty_dev(shape, np.float32)
    plan.apply_T(y, z)
    assert rel_l2(z.cpu().numpy(), x) < TOL_F32


@pytest.mark.parametrize("shape,axis", [((30, 20, 22, 8), 2), ((25, 31, 19), 0), ((17, 40, 12, 4), 3)])
def test_fir_factor_equals_correlate1d(shape, axis):
    """A 4-tap FIR filter along one mode: ELL-4 rows i -> columns i-1 .. i+2, zero boundary."""
    tca = lib()
    rng = np.random.default_rng(22 + axis)
    h = rng.standard_normal(4)
    n = shape[axis]
    fir = tca.Factor(tca.FACTOR_ELL4, n, n, np.tile(h, (n, 1)), (np.arange(n) - 1).astype(np.int32))
    facs = [fir if k == axis else _identity(tca, shape[k]) for k in range(len(shape))]
    plan = tca.Plan(shape, facs, lam=0.0, precision="f32")
    x = rng.standard_normal(shape).astype(np.float32)
    y = empty_dev(shape, np.float32)
    plan.apply(to_dev(x, np.float32), y)
    # correlate1d with weights w puts w[j] at offset j - len(w)//2 = j - 2; our taps sit at -1..2.
    ref = ndimage.correlate1d(x.astype(np.float64), np.concatenate([[0.0], h]), axis=axis, mode="constant")
    assert rel_l2(y.cpu().numpy(), ref) < TOL_F32
    mats = [_as_dense(tca, f) for f in facs]
    assert rel_l2(y.cpu().numpy(), O.apply(x.astype(np.float64), mats)) < TOL_F32


def _as_dense(tca, f):
    if f.kind == tca.FACTOR_DENSE:
        return f.values.reshape(f.m, f.n)
    return synth.ell4_to_dense(f.col0, f.values.reshape(f.m, 4), f.n)


def test_up_and_downsampling_factors():
    """Table 1's up- and downsampling as rectangular banded factors: linear interpolation to twice
    the points (2 taps per row) and averaging of pairs (2 taps per row), on two modes at once;
    checked against numpy's interpolation and reshape-mean."""
    tca = lib()
    shape = (20, 24, 18, 4)
    n1, n2 = shape[0], shape[1]
    # upsampling mode 1: output point t = i / 2 (i = 0 .. 2 n1 - 2), linear between neighbours
    m1 = 2 * n1 - 1
    col0 = (np.arange(m1) // 2).astype(np.int32)
    w = np.zeros((m1, 4))
    w[0::2, 0] = 1.0
    w[1::2, 0] = 0.5
    w[1::2, 1] = 0.5
    up = tca.Factor(tca.FACTOR_ELL4, m1, n1, w, col0)
    # downsampling mode 2: mean of pairs
    m2 = n2 // 2
    down = tca.Factor(tca.FACTOR_ELL4, m2, n2, np.tile([0.5, 0.5, 0.0, 0.0], (m2, 1)),
                      (2 * np.arange(m2)).astype(np.int32))
    facs = [up, down, _identity(tca, shape[2]), _identity(tca, shape[3])]
    plan = tca.Plan(shape, facs, lam=0.0, precision="f32")
    rng = np.random.default_rng(23)
    x = rng.standard_normal(shape).astype(np.float32)
    y = empty_dev((m1, m2) + shape[2:], np.float32)
    plan.apply(to_dev(x, np.float32), y)
    xd = x.astype(np.float64)
    ref = xd.reshape(n1, m2, 2, *shape[2:]).mean(axis=2)
    t = np.arange(m1) / 2.0
    ref = np.apply_along_axis(lambda v: np.interp(t, np.arange(n1), v), 0, ref)
    assert rel_l2(y.cpu().numpy(), ref) < TOL_F32


@pytest.mark.parametrize("axis", [1, 2])
def test_dft_along_one_mode_as_two_real_factors(axis):
    """The DFT of a real tensor along one mode: real part = C x, imaginary part = -S x with the
    cosine and sine matrices as dense factors - two real separable transformations."""
    tca = lib()
    shape = (12, 20, 16, 8)
    n = shape[axis]
    k = np.arange(n)[:, None] * np.arange(n)[None, :]
    cmat, smat = np.cos(2 * np.pi * k / n), np.sin(2 * np.pi * k / n)
    rng = np.random.default_rng(24)
    x = rng.standard_normal(shape).astype(np.float32)
    parts = []
    for mat in (cmat, -smat):
        facs = [tca.Factor(tca.FACTOR_DENSE, n, n, mat) if a == axis else _dense_identity(tca, shape[a])
                for a in range(4)]
        plan = tca.Plan(shape, facs, lam=0.0, precision="f32")
        y = empty_dev(shape, np.float32)
        plan.apply(to_dev(x, np.float32), y)
        parts.append(y.cpu().numpy())
    ref = np.fft.fft(x.astype(np.float64), axis=axis)
    assert rel_l2(parts[0], ref.real) < TOL_F32
    assert rel_l2(parts[1], ref.imag) < TOL_F32


@pytest.mark.parametrize("prec,dt,tol", [("f32", np.float32, TOL_F32), ("f64", np.float64, 1e-12)])
def test_ell4_rows_starting_far_outside_the_grid(prec, dt, tol):
    """An ELL-4 factor whose first and last rows start at the ends of the int32 range (no column
    of theirs is in the grid) and whose other rows start anywhere from below 0 to past the last
    column: the operator equals the dense matrix with those weights dropped."""
    tca = lib()
    shape = (20, 17, 12, 4)
    rng = np.random.default_rng(31)
    n = shape[0]
    m = 30
    mid = np.sort(rng.integers(-6, n + 3, size=m - 6))
    col0 = np.concatenate([[np.iinfo(np.int32).min] * 3, mid, [np.iinfo(np.int32).max] * 3]).astype(np.int32)
    w = rng.standard_normal((m, 4))
    facs = [tca.Factor(tca.FACTOR_ELL4, m, n, w, col0)] + [_identity(tca, k) for k in shape[1:]]
    lam = 3e-3
    plan = tca.Plan(shape, facs, lam=lam, precision=prec)
    mats = [synth.ell4_to_dense(col0, w, n)] + [np.eye(k) for k in shape[1:]]
    x = rng.standard_normal(shape).astype(dt)
    y = rng.standard_normal((m,) + shape[1:]).astype(dt)
    ax = empty_dev((m,) + shape[1:], dt)
    plan.apply(to_dev(x, dt), ax)
    assert rel_l2(ax.cpu().numpy(), O.apply(x.astype(np.float64), mats)) < tol
    aty = empty_dev(shape, dt)
    plan.apply_T(to_dev(y, dt), aty)
    assert rel_l2(aty.cpu().numpy(), O.apply_T(y.astype(np.float64), mats)) < tol
    kx = empty_dev(shape, dt)
    plan.apply_normal(to_dev(x, dt), kx)
    assert rel_l2(kx.cpu().numpy(), O.normal_apply(x.astype(np.float64), mats, lam)) < tol
