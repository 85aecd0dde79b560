"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Each test ties an oracle function to something other than itself: a library
routine (np.kron, scipy.fft.dct, scipy.ndimage.correlate1d, Cholesky, eigh,
lstsq, scipy's B-spline basis), an exact closed form, an invariant, or a brute
force written directly from the definition on a tiny input.
"""
import functools
import itertools
import math
import os

import numpy as np
import pytest
from scipy import fft as sfft
from scipy import interpolate, linalg, ndimage

from oracle import tca_oracle as O
from paper_1001_5460_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_mats(rng, shape, sample_shape):
    return [rng.standard_normal((m, n)) for m, n in zip(sample_shape, shape)]


# --- mode product / separable transformation (Sec. 2.1, Eq. separable_transf) ---

def test_apply_equals_kronecker_matvec():
    """X x_1 A1 ... x_4 A4 equals (A1 kron A2 kron A3 kron A4) vec(X) for C-order vec (Sec. 3)."""
    rng = np.random.default_rng(1)
    shape, sshape = (3, 4, 5, 2), (4, 2, 6, 3)
    x = rng.standard_normal(shape)
    mats = _rand_mats(rng, shape, sshape)
    big = mats[0]
    for a in mats[1:]:
        big = np.kron(big, a)  # library Kronecker product
    ref = (big @ x.ravel()).reshape(sshape)
    np.testing.assert_allclose(O.apply(x, mats), ref, rtol=1e-12, atol=1e-12)


def test_apply_equals_bruteforce_sum():
    """Direct elementwise sum of Eq. separable_transf on a tiny 3D tensor (no chaining)."""
    rng = np.random.default_rng(2)
    shape, sshape = (2, 3, 2), (3, 2, 4)
    x = rng.standard_normal(shape)
    a, b, c = _rand_mats(rng, shape, sshape)
    ref = np.zeros(sshape)
    for x1, y1, z1 in itertools.product(*map(range, sshape)):
        s = 0.0
        for xi, yi, zi in itertools.product(*map(range, shape)):
            s += a[x1, xi] * b[y1, yi] * c[z1, zi] * x[xi, yi, zi]
        ref[x1, y1, z1] = s
    np.testing.assert_allclose(O.apply(x, [a, b, c]), ref, rtol=1e-12, atol=1e-13)


def test_commutativity_all_orders():
    """Every order of the one-dimensional transformations gives one result (Sec. 2.1)."""
    rng = np.random.default_rng(3)
    shape, sshape = (3, 4, 2, 5), (5, 3, 4, 2)
    x = rng.standard_normal(shape)
    mats = _rand_mats(rng, shape, sshape)
    ref = O.apply(x, mats)
    for order in O.all_mode_orders(4):
        np.testing.assert_allclose(O.apply(x, mats, order=order), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2, 3])
def test_dct_factor_equals_library_dct(axis):
    """A factor holding the orthonormal DCT-II matrix equals scipy's DCT along that axis (Table 1)."""
    rng = np.random.default_rng(4 + axis)
    shape = (5, 6, 7, 4)
    x = rng.standard_normal(shape)
    n = shape[axis]
    k = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    c = np.cos(np.pi * k * (2 * i + 1) / (2 * n)) * np.sqrt(2.0 / n)
    c[0, :] = np.sqrt(1.0 / n)
    ref = sfft.dct(x, type=2, norm="ortho", axis=axis)
    np.testing.assert_allclose(O.mode_product(x, c, axis), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_fir_factor_equals_correlate1d(axis):
    """A banded Toeplitz factor equals 1D correlation with zero boundary (Table 1, convolution)."""
    rng = np.random.default_rng(10 + axis)
    shape = (9, 8, 11)
    x = rng.standard_normal(shape)
    w = rng.standard_normal(5)
    n = shape[axis]
    a = np.zeros((n, n))
    for row in range(n):
        for d in range(-2, 3):
            if 0 <= row + d < n:
                a[row, row + d] = w[d + 2]
    ref = ndimage.correlate1d(x, w, axis=axis, mode="constant", cval=0.0)
    np.testing.assert_allclose(O.mode_product(x, a, axis), ref, rtol=1e-12, atol=1e-12)


def test_adjointness():
    """<A x, y> = <x, A^T y> (App. "Tensor transposition")."""
    rng = np.random.default_rng(5)
    shape, sshape = (4, 3, 5, 2), (6, 5, 7, 3)
    mats = _rand_mats(rng, shape, sshape)
    x = rng.standard_normal(shape)
    y = rng.standard_normal(sshape)
    lhs = O.inner(O.apply(x, mats), y)
    rhs = O.inner(x, O.apply_T(y, mats))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_inner_product_definition():
    """<A, B> is the full contraction of matching indices (Eq. A13) = vdot of the flattened arrays."""
    rng = np.random.default_rng(6)
    a = rng.standard_normal((3, 4, 5))
    b = rng.standard_normal((3, 4, 5))
    assert O.inner(a, b) == pytest.approx(np.vdot(a.ravel(), b.ravel()), rel=1e-13)


# --- regulariser and normal operator ---

def test_second_difference_equals_numpy_diff():
    rng = np.random.default_rng(7)
    for n in (3, 4, 9):
        v = rng.standard_normal(n)
        np.testing.assert_allclose(O.second_difference(n) @ v, np.diff(v, n=2), rtol=0, atol=1e-14)
    # Null space of D2^T D2: constant and linear sequences.
    n = 12
    d2 = O.second_difference(n)
    l = d2.T @ d2
    np.testing.assert_allclose(l @ np.ones(n), 0.0, atol=1e-13)
    np.testing.assert_allclose(l @ np.arange(n, dtype=float), 0.0, atol=1e-12)
    # A quadratic has constant second difference 2.
    t = np.arange(n, dtype=float)
    np.testing.assert_allclose(d2 @ (t * t), 2.0, atol=1e-12)


def test_normal_operator_equals_dense_matrix():
    """K x the long way equals the explicit reshaped normal matrix (Sec. 3) on a tiny B-spline case."""
    inst = synth.instance_bspline((6, 5, 7, 4), seed=11, lam=0.3, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    rng = np.random.default_rng(8)
    x = rng.standard_normal(inst.shape)
    k = O.dense_normal_matrix(mats, 0.3, inst.shape)
    np.testing.assert_allclose(O.normal_apply(x, mats, 0.3).ravel(), k @ x.ravel(), rtol=1e-11, atol=1e-11)
    # Symmetric positive definite.
    np.testing.assert_allclose(k, k.T, atol=1e-12)
    assert np.linalg.eigvalsh(k).min() > 0.0


def test_normal_operator_symmetry_random():
    inst = synth.instance_bspline((7, 6, 5), seed=12, lam=1e-2, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    rng = np.random.default_rng(9)
    x = rng.standard_normal(inst.shape)
    y = rng.standard_normal(inst.shape)
    a = O.inner(O.normal_apply(x, mats, 1e-2), y)
    b = O.inner(x, O.normal_apply(y, mats, 1e-2))
    assert abs(a - b) <= 1e-12 * abs(a)
    assert O.inner(O.normal_apply(x, mats, 1e-2), x) > 0


# --- CG of Fig. 2 ---

@pytest.mark.slow
def test_cg_matches_cholesky_dense_3d():
    """Dense 16^3 problem with 24x16 Gaussian factors: CG to 1e-10 vs Cholesky of the reshaped system."""
    inst = synth.instance_dense_3d(seed=0)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    res = O.solve(b, mats, inst.lam, rtol=1e-10)
    assert res.converged
    x_direct = O.direct_solve(b, mats, inst.lam, inst.shape)
    err = np.linalg.norm(res.x - x_direct) / np.linalg.norm(x_direct)
    assert err < 1e-8, err
    assert O.rel_residual(res.x, b, mats, inst.lam) < 1e-9


def test_cg_matches_cholesky_small_bspline():
    inst = synth.instance_bspline((8, 7, 6, 4), seed=13, lam=1e-3, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    res = O.solve(b, mats, inst.lam, rtol=1e-12)
    x_direct = O.direct_solve(b, mats, inst.lam, inst.shape)
    err = np.linalg.norm(res.x - x_direct) / np.linalg.norm(x_direct)
    assert err < 1e-9, err


def test_lambda_zero_closed_form():
    """lambda = 0: the normal-equation solution is b x_k pinv(A_k) on every mode (least squares)."""
    rng = np.random.default_rng(14)
    shape, sshape = (5, 4, 6), (8, 7, 9)
    mats = _rand_mats(rng, shape, sshape)
    b = rng.standard_normal(sshape)
    res = O.solve(b, mats, 0.0, rtol=1e-13, max_iter=5000)
    ref = b
    for k, a in enumerate(mats):
        ref = np.moveaxis(np.tensordot(np.linalg.pinv(a), ref, axes=([1], [k])), 0, k)
    np.testing.assert_allclose(res.x, ref, rtol=1e-9, atol=1e-10)


def test_identity_factors_kronecker_sum_eigensolve():
    """A_k = I: K = I + lambda sum_k L_k is solved exactly in the eigenbasis of each L_k."""
    rng = np.random.default_rng(15)
    shape = (7, 5, 6, 3)
    lam = 0.37
    mats = [np.eye(n) for n in shape]
    b = rng.standard_normal(shape)
    res = O.solve(b, mats, lam, rtol=1e-13)
    # Exact solve: rotate into each L_k's eigenbasis, divide, rotate back.
    evals, evecs = [], []
    for n in shape:
        d2 = np.diff(np.eye(n), n=2, axis=0)  # library second difference
        mu, v = linalg.eigh(d2.T @ d2)
        evals.append(mu)
        evecs.append(v)
    xh = b
    for k, v in enumerate(evecs):
        xh = np.moveaxis(np.tensordot(v.T, xh, axes=([1], [k])), 0, k)
    denom = np.ones(shape)
    for k, mu in enumerate(evals):
        sh = [1] * len(shape)
        sh[k] = shape[k]
        denom = denom + lam * mu.reshape(sh)
    xh = xh / denom
    for k, v in enumerate(evecs):
        xh = np.moveaxis(np.tensordot(v, xh, axes=([1], [k])), 0, k)
    np.testing.assert_allclose(res.x, xh, rtol=1e-10, atol=1e-11)


def test_cg_zero_rhs_and_x0():
    mats = [np.eye(3), np.eye(4)]
    r = O.solve(np.zeros((3, 4)), mats, 0.1)
    assert r.iters == 0 and np.all(r.x == 0)
    # Starting from the exact solution needs no iteration.
    rng = np.random.default_rng(16)
    b = rng.standard_normal((3, 4))
    exact = O.solve(b, mats, 0.1, rtol=1e-14).x
    r2 = O.solve(b, mats, 0.1, rtol=1e-8, x0=exact)
    assert r2.iters == 0


# --- CG preconditioned by a separable tensor inverse (Sec. 3, Eq. TensorEq) ---

def test_separable_inverse_is_the_kronecker_inverse():
    """(x)_k (G_k + s lam L_k)^-1 is the matrix inverse of (x)_k (G_k + s lam L_k) (mixed product), via np.kron."""
    rng = np.random.default_rng(23)
    shape, sshape = (5, 4, 6), (7, 6, 9)
    mats = _rand_mats(rng, shape, sshape)
    lam, shift = 0.03, 16.0
    inv = O.separable_inverse_factors(mats, lam, shift)
    blocks = []
    for a, n in zip(mats, shape):
        d2 = np.diff(np.eye(n), n=2, axis=0)  # library second difference
        blocks.append(a.T @ a + shift * lam * (d2.T @ d2))
    big = functools.reduce(np.kron, blocks)
    x = rng.standard_normal(shape)
    np.testing.assert_allclose(O.apply_separable(x, inv).ravel(), np.linalg.solve(big, x.ravel()),
                               rtol=1e-9, atol=1e-11)


def test_pcg_with_identity_is_cg_step_for_step():
    inst = synth.instance_bspline((8, 7, 6, 4), seed=24, lam=1e-3, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    kop = lambda v: O.normal_apply(v, mats, inst.lam)
    rhs = O.apply_T(O.apply(inst.x_true, mats) + inst.noise, mats)
    for k in (1, 3, 7):
        a = O.cg(kop, rhs, rtol=0.0, max_iter=k)
        b = O.pcg(kop, lambda r: r, rhs, rtol=0.0, max_iter=k)
        assert a.iters == b.iters == k
        np.testing.assert_allclose(b.x, a.x, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(b.history, a.history, rtol=1e-12)


def test_pcg_with_exact_inverse_takes_one_step():
    """M = K makes Z = K^-1 R: one PCG step lands on the Cholesky solution; a PCG that used
    <R, R> for rho (a plausible slip) would not."""
    rng = np.random.default_rng(25)
    shape, sshape = (4, 5, 3), (6, 7, 5)
    mats = _rand_mats(rng, shape, sshape)
    lam = 0.05
    b = rng.standard_normal(sshape)
    kmat = O.dense_normal_matrix(mats, lam, shape)
    kop = lambda v: O.normal_apply(v, mats, lam)
    minv = lambda r: np.linalg.solve(kmat, r.ravel()).reshape(shape)
    rhs = O.apply_T(b, mats)
    res = O.pcg(kop, minv, rhs, rtol=1e-11, max_iter=3)
    ref = O.direct_solve(b, mats, lam, shape)
    assert res.iters == 1
    np.testing.assert_allclose(res.x, ref, rtol=1e-9, atol=1e-11)


def test_pcg_iterates_are_cg_on_the_split_system():
    """With M = C C^T, preconditioned CG is plain CG on C^-1 K C^-T y = C^-1 rhs: its k-th iterate
    is C^-T y_k (textbook identity), checked iterate by iterate with explicit matrices."""
    rng = np.random.default_rng(28)
    shape, sshape = (4, 3, 5), (6, 5, 7)
    mats = _rand_mats(rng, shape, sshape)
    lam = 0.02
    kmat = O.dense_normal_matrix(mats, lam, shape)
    inv = O.separable_inverse_factors(mats, lam, 16.0)
    m_inv = functools.reduce(np.kron, inv)           # M^-1 as a matrix
    c = np.linalg.cholesky(np.linalg.inv(m_inv))     # M = C C^T
    c_inv = np.linalg.inv(c)
    kt = c_inv @ kmat @ c_inv.T
    b = rng.standard_normal(sshape)
    rhs = O.apply_T(b, mats)
    kop = lambda v: O.normal_apply(v, mats, lam)
    for k in (1, 2, 4, 6):
        x = O.pcg(kop, lambda r: O.apply_separable(r, inv), rhs, rtol=0.0, max_iter=k).x
        y = O.cg(lambda v: (kt @ v.ravel()).reshape(v.shape), (c_inv @ rhs.ravel()).reshape(shape),
                 rtol=0.0, max_iter=k).x
        np.testing.assert_allclose(x.ravel(), c_inv.T @ y.ravel(), rtol=1e-8, atol=1e-10)


def test_pcg_separable_matches_cholesky_and_needs_fewer_iterations():
    """Dense Gaussian factors, small lambda: the separable-inverse PCG reaches the Cholesky solution
    in far fewer iterations than plain CG (the Gram part, whose condition number is the product of
    the modes', is inverted exactly)."""
    rng = np.random.default_rng(26)
    shape = (9, 8, 7)
    sshape = tuple(int(math.ceil(1.5 * n)) for n in shape)
    mats = [rng.standard_normal((m, n)) / math.sqrt(m) for m, n in zip(sshape, shape)]
    lam = 2e-4
    b = rng.standard_normal(sshape)
    kop = lambda v: O.normal_apply(v, mats, lam)
    rhs = O.apply_T(b, mats)
    inv = O.separable_inverse_factors(mats, lam, 16.0)
    pc = O.pcg(kop, lambda r: O.apply_separable(r, inv), rhs, rtol=1e-10)
    plain = O.cg(kop, rhs, rtol=1e-10)
    ref = O.direct_solve(b, mats, lam, shape)
    assert pc.converged and plain.converged
    err = np.linalg.norm(pc.x - ref) / np.linalg.norm(ref)
    assert err < 1e-7, err
    assert pc.iters * 3 < plain.iters, (pc.iters, plain.iters)


@pytest.mark.parametrize("shape,lam", [((6, 5, 7, 4), 0.3), ((5, 2, 6), 0.7), ((7, 6, 5, 1), 1e-3)])
def test_jacobi_diagonal_is_the_diagonal_of_the_explicit_normal_matrix(shape, lam):
    """diag(K) from the per-mode definition equals the diagonal of the explicit reshaped normal
    matrix (Sec. 3 matrix form), regulariser included; a mode with n < 3 carries no regulariser."""
    inst = synth.instance_bspline(shape, seed=31, lam=lam, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    k = O.dense_normal_matrix(mats, lam, shape)
    np.testing.assert_allclose(O.jacobi_diagonal(mats, lam, shape).ravel(), np.diag(k), rtol=1e-13, atol=1e-14)
    rng = np.random.default_rng(3)
    dense = [rng.standard_normal((n + 3, n)) for n in shape]
    kd = O.dense_normal_matrix(dense, lam, shape)
    np.testing.assert_allclose(O.jacobi_diagonal(dense, lam, shape).ravel(), np.diag(kd), rtol=1e-13)


def test_jacobi_pcg_matches_cholesky_and_fixes_a_bad_scaling():
    """Factors whose columns differ in scale by 10^4: K is badly scaled, point Jacobi removes the
    scaling, and the Jacobi-preconditioned CG of Fig. 2 reaches the Cholesky solution in a fraction
    of plain CG's iterations."""
    rng = np.random.default_rng(27)
    shape = (9, 8, 7)
    sshape = tuple(int(math.ceil(1.5 * n)) for n in shape)
    mats = [(rng.standard_normal((m, n)) / math.sqrt(m)) * 10.0 ** rng.uniform(-1, 1, n)
            for m, n in zip(sshape, shape)]
    lam = 1e-4
    b = rng.standard_normal(sshape)
    kop = lambda v: O.normal_apply(v, mats, lam)
    rhs = O.apply_T(b, mats)
    dia = O.jacobi_diagonal(mats, lam, shape)
    pc = O.pcg(kop, lambda r: r / dia, rhs, rtol=1e-10)
    plain = O.cg(kop, rhs, rtol=1e-10, max_iter=20000)
    ref = O.direct_solve(b, mats, lam, shape)
    assert pc.converged
    err = np.linalg.norm(pc.x - ref) / np.linalg.norm(ref)
    assert err < 1e-7, err
    assert pc.iters * 2 < plain.iters, (pc.iters, plain.iters)


def test_banded_separable_inverse_is_symmetric_positive_and_still_preconditions():
    """The 7-band truncation of each per-mode inverse (B-spline factors) is symmetric and positive
    definite (eigh), equals the full inverse inside the band, and still cuts the CG count."""
    inst = synth.instance_bspline((24, 22, 20, 8), seed=27, lam=1e-3, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    full = O.separable_inverse_factors(mats, inst.lam, 32.0)
    band = O.separable_inverse_factors(mats, inst.lam, 32.0, half_band=3)
    for f, bnd in zip(full, band):
        n = len(f)
        i, j = np.indices((n, n))
        assert np.array_equal(bnd[np.abs(i - j) <= 3], f[np.abs(i - j) <= 3])
        assert np.all(bnd[np.abs(i - j) > 3] == 0.0)
        np.testing.assert_array_equal(bnd, bnd.T)
        assert linalg.eigh(bnd, eigvals_only=True).min() > 0.0
    kop = lambda v: O.normal_apply(v, mats, inst.lam)
    rhs = O.apply_T(O.apply(inst.x_true, mats) + inst.noise, mats)
    plain = O.cg(kop, rhs, rtol=1e-6)
    banded = O.pcg(kop, lambda r: O.apply_separable(r, band), rhs, rtol=1e-6)
    assert banded.converged and banded.iters * 2 < plain.iters, (banded.iters, plain.iters)


# --- B-spline factors (inputs of the spline reconstruction, Sec. 5) ---

def test_bspline3_golden_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "bspline3_values.txt")) if l.strip() and not l.startswith("#")]
    for u, num, den in rows:
        assert synth.bspline3(float(u)) == pytest.approx(int(num) / int(den), abs=1e-15)


def test_bspline3_equals_scipy_basis():
    basis = interpolate.BSpline.basis_element([-2.0, -1.0, 0.0, 1.0, 2.0], extrapolate=False)
    u = np.linspace(-1.999, 1.999, 401)
    np.testing.assert_allclose(synth.bspline3(u), basis(u), rtol=1e-12, atol=1e-14)


def test_bspline_factor_partition_of_unity_and_band():
    rng = np.random.default_rng(17)
    n, m = 40, 60
    col0, w, t = synth.bspline_factor_ell4(n, m, rng)
    a = synth.ell4_to_dense(col0, w, n)
    interior = (t >= 1.0) & (t <= n - 2.0)
    np.testing.assert_allclose(a[interior].sum(axis=1), 1.0, atol=1e-14)
    assert np.all(np.diff(t) > 0)
    # At most 4 nonzeros per row, contiguous.
    assert (np.count_nonzero(a, axis=1) <= 4).all()
    # Gram of a 4-wide band is 7-banded.
    g = a.T @ a
    i, j = np.nonzero(np.abs(g) > 0)
    assert np.max(np.abs(i - j)) <= 3


def test_bspline_positions_at_integers():
    """Row of a sample sitting on grid point j reads [1/6, 2/3, 1/6] at j-1, j, j+1."""
    t = np.array([3.0, 7.0])
    col0 = (np.floor(t) - 1).astype(np.int32)
    cols = col0[:, None] + np.arange(4)
    w = synth.bspline3(t[:, None] - cols)
    np.testing.assert_allclose(w, [[1 / 6, 2 / 3, 1 / 6, 0.0]] * 2, atol=1e-15)


# --- the pins catch planted mistakes in the oracle (mutation checks, CPU only) ---

def test_pin_catches_transposed_factor(monkeypatch):
    rng = np.random.default_rng(18)
    shape = (3, 3, 3)
    mats = [rng.standard_normal((3, 3)) for _ in range(3)]
    x = rng.standard_normal(shape)
    good = O.apply(x, mats)
    orig = O.mode_product
    monkeypatch.setattr(O, "mode_product", lambda x_, a, k: orig(x_, np.asarray(a).T, k))
    bad = O.apply(x, mats)
    big = np.kron(np.kron(mats[0], mats[1]), mats[2])
    ref = (big @ x.ravel()).reshape(shape)
    assert np.allclose(good, ref) and not np.allclose(bad, ref)


def test_pin_catches_dropped_regulariser_term(monkeypatch):
    shape = (5, 4, 6)
    lam = 0.5
    mats = [np.eye(n) for n in shape]
    rng = np.random.default_rng(19)
    x = rng.standard_normal(shape)
    k = O.dense_normal_matrix(mats, lam, shape)
    assert np.allclose(O.normal_apply(x, mats, lam).ravel(), k @ x.ravel())
    monkeypatch.setattr(O, "regulariser", lambda v, l: l * O.mode_product(v, O.second_difference(v.shape[0]).T @ O.second_difference(v.shape[0]), 0))
    assert not np.allclose(O.normal_apply(x, mats, lam).ravel(), k @ x.ravel())


def test_pin_catches_wrong_cg_sign():
    """A CG with the residual update sign flipped stops matching the direct solve."""
    rng = np.random.default_rng(20)
    shape = (4, 5)
    mats = [rng.standard_normal((6, 4)), rng.standard_normal((7, 5))]
    b = rng.standard_normal((6, 7))
    lam = 0.1
    kop = lambda v: O.normal_apply(v, mats, lam)
    rhs = O.apply_T(b, mats)
    ref = O.direct_solve(b, mats, lam, shape)
    good = O.cg(kop, rhs, rtol=1e-12).x
    assert np.allclose(good, ref, rtol=1e-8, atol=1e-10)
    # Planted mistake: R = R + alpha Q.
    c = np.zeros(shape); r = rhs.copy(); p = r.copy(); rho = O.inner(r, r)
    for _ in range(50):
        q = kop(p); alpha = rho / O.inner(p, q); c = c + alpha * p; r = r + alpha * q
        rho1 = O.inner(r, r); p = r + (rho1 / rho) * p; rho = rho1
    assert not np.allclose(c, ref, rtol=1e-4)


def test_sampled_oracle_matches_full():
    """Point-wise (A x)[s] and (K x)[i] agree with the full oracle evaluations."""
    inst = synth.instance_bspline((9, 8, 10, 4), seed=21, lam=0.2, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    rng = np.random.default_rng(22)
    x = rng.standard_normal(inst.shape)
    ax = O.apply(x, mats)
    kx = O.normal_apply(x, mats, 0.2)
    for _ in range(12):
        s = tuple(int(rng.integers(0, m)) for m in inst.sample_shape)
        i = tuple(int(rng.integers(0, n)) for n in inst.shape)
        assert O.apply_at(x, mats, s) == pytest.approx(ax[s], rel=1e-12, abs=1e-12)
        assert O.normal_apply_at(x, mats, 0.2, i) == pytest.approx(kx[i], rel=1e-12, abs=1e-12)
    # dense factors too
    mats = [rng.standard_normal((5, 4)), rng.standard_normal((6, 3)), rng.standard_normal((4, 5))]
    x = rng.standard_normal((4, 3, 5))
    kx = O.normal_apply(x, mats, 0.3)
    for i in [(0, 0, 0), (3, 2, 4), (1, 1, 2)]:
        assert O.normal_apply_at(x, mats, 0.3, i) == pytest.approx(kx[i], rel=1e-12)


# ---- scattered samples (row-wise / face-splitting product of the per-mode rows) ----

@pytest.mark.parametrize("shape,m", [((5, 4, 6), 37), ((4, 5, 3, 4), 29)])
def test_scattered_apply_equals_explicit_kronecker_rows(shape, m):
    """Row s of the scattered system tensor is the Kronecker product of the sample's dense
    per-mode rows; the windowed sums equal that explicit matrix, and the transpose is its
    adjoint."""
    inst = synth.instance_scattered(shape, m, seed=40 + m)
    a = O.scattered_rows_matrix(inst.col0, inst.w, shape)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(shape)
    y = rng.standard_normal(m)
    np.testing.assert_allclose(O.scattered_apply(x, inst.col0, inst.w), a @ x.ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(O.scattered_apply_T(y, inst.col0, inst.w, shape).ravel(), a.T @ y,
                               rtol=1e-12, atol=1e-13)
    k = a.T @ a + O.dense_normal_matrix([np.zeros((1, n)) for n in shape], inst.lam, shape)
    np.testing.assert_allclose(O.scattered_normal_apply(x, inst.col0, inst.w, inst.lam).ravel(), k @ x.ravel(),
                               rtol=1e-11, atol=1e-12)


def test_scattered_on_a_tensor_grid_equals_the_separable_operator():
    """Samples that lie on a tensor grid of per-mode positions are the rows of A_1 x ... x A_d:
    the scattered operator must then equal the separable one (Eq. separable_transf)."""
    rng = np.random.default_rng(12)
    shape = (6, 5, 7, 4)
    facs = [synth.bspline_factor_ell4(n, int(round(1.5 * n)), rng) for n in shape]
    mats = [synth.ell4_to_dense(c0, w, n) for (c0, w, _), n in zip(facs, shape)]
    ms = [f[0].shape[0] for f in facs]
    grid = np.array(list(itertools.product(*[range(mm) for mm in ms])))  # C order of the sample tensor
    col0s = [facs[k][0][grid[:, k]] for k in range(4)]
    ws = [facs[k][1][grid[:, k]] for k in range(4)]
    x = rng.standard_normal(shape)
    np.testing.assert_allclose(O.scattered_apply(x, col0s, ws), O.apply(x, mats).ravel(), rtol=1e-12, atol=1e-13)
    y = rng.standard_normal(len(grid))
    np.testing.assert_allclose(O.scattered_apply_T(y, col0s, ws, shape), O.apply_T(y.reshape(ms), mats),
                               rtol=1e-12, atol=1e-13)


def test_scattered_cg_matches_direct_solve():
    shape = (5, 6, 4)
    inst = synth.instance_scattered(shape, 300, seed=9, lam=1e-2)
    a = O.scattered_rows_matrix(inst.col0, inst.w, shape)
    b = a @ inst.x_true.ravel() + inst.noise
    k = a.T @ a + O.dense_normal_matrix([np.zeros((1, n)) for n in shape], inst.lam, shape)
    ref = np.linalg.solve(k, a.T @ b).reshape(shape)
    res = O.cg(lambda v: O.scattered_normal_apply(v, inst.col0, inst.w, inst.lam),
               O.scattered_apply_T(b, inst.col0, inst.w, shape), rtol=1e-12)
    assert res.converged
    np.testing.assert_allclose(res.x, ref, rtol=1e-8, atol=1e-9)


# ---- tensor multigrid (two-grid V-cycle as a CG preconditioner) ----

def _tmg_case():
    inst = synth.instance_bspline((9, 8, 7, 4), seed=33, lam=1e-2, with_truth=False)
    mats = [f.dense() for f in inst.factors]
    shape = inst.shape
    kop = lambda v: O.normal_apply(v, mats, inst.lam)
    dia = O.jacobi_diagonal(mats, inst.lam, shape)
    prol = [O.tmg_prolongation(n) if k < 3 else np.eye(n) for k, n in enumerate(shape)]
    return inst, mats, shape, kop, dia, prol


def test_tmg_prolongation_interpolates_linear_functions():
    """Linear interpolation reproduces linear functions exactly on the fine points the coarse
    points span (the coarse points are the even fine points; an even n leaves one last fine point
    with half the last coarse value), and its interior columns sum to 2 (restriction = transpose,
    full weighting x 2)."""
    for n in (7, 8, 9):
        p = O.tmg_prolongation(n)
        nc = p.shape[1]
        xc = np.arange(nc) * 2.0
        span = 2 * (nc - 1) + 1
        np.testing.assert_allclose((p @ xc)[:span], np.arange(span), atol=1e-15)
        np.testing.assert_allclose((p.T @ np.ones(n))[1:-1], 2.0)


def test_tmg_coarse_correction_is_the_galerkin_projection():
    """With no smoothing, the cycle is z = P (P^T K P)^-1 P^T r: checked against the explicit
    matrices (np.kron transfers, explicit normal matrix, dense inverse)."""
    inst, mats, shape, kop, dia, prol = _tmg_case()
    k = O.dense_normal_matrix(mats, inst.lam, shape)
    pm = O.kron_matrix(prol)
    ref_op = pm @ np.linalg.inv(pm.T @ k @ pm) @ pm.T
    rng = np.random.default_rng(1)
    r = rng.standard_normal(shape)
    z = O.tmg_vcycle(r, kop, dia, prol, nu=0, lam_lo=1.0, lam_hi=2.0, coarse_rtol=1e-13)
    np.testing.assert_allclose(z.ravel(), ref_op @ r.ravel(), rtol=1e-8, atol=1e-10)


def test_tmg_vcycle_is_symmetric_positive_and_preconditions():
    """With Chebyshev smoothing the cycle is a symmetric positive definite operator (what PCG needs),
    and PCG with it reaches the Cholesky solution in fewer iterations than plain CG."""
    inst, mats, shape, kop, dia, prol = _tmg_case()
    v = np.random.default_rng(0).standard_normal(shape)
    for _ in range(30):
        v = kop(v) / dia
        lmax = np.linalg.norm(v)
        v /= lmax
    cyc = lambda r: O.tmg_vcycle(r, kop, dia, prol, nu=2, lam_lo=lmax / 30, lam_hi=1.05 * lmax, coarse_rtol=1e-13)
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    assert abs(O.inner(cyc(a), b) - O.inner(a, cyc(b))) < 1e-9 * np.linalg.norm(a) * np.linalg.norm(b)
    assert O.inner(cyc(a), a) > 0 and O.inner(cyc(b), b) > 0
    rhs = rng.standard_normal(shape)
    ref = np.linalg.solve(O.dense_normal_matrix(mats, inst.lam, shape), rhs.ravel()).reshape(shape)
    pc = O.pcg(kop, cyc, rhs, rtol=1e-10)
    plain = O.cg(kop, rhs, rtol=1e-10)
    assert pc.converged
    np.testing.assert_allclose(pc.x, ref, rtol=1e-7, atol=1e-8)
    assert pc.iters < plain.iters, (pc.iters, plain.iters)


# ---- corner model of the preconditioner's shift ------------------------------------

def test_corner_model_shift_special_cases():
    """One mode: every corner's ratio K/M is 1 at s = 1, the first grid point; lambda = 0: K = M at
    every corner for every s, so the first grid point again."""
    rng = np.random.default_rng(40)
    a = rng.standard_normal((9, 7))
    assert O.corner_model_shift([a], 1e-2) == 1.0
    mats = [rng.standard_normal((m, n)) for m, n in ((8, 6), (7, 5), (9, 4))]
    assert O.corner_model_shift(mats, 0.0) == 1.0


def _pcg_iters(mats, lam, shift, rhs):
    f = O.separable_inverse_factors(mats, lam, shift)
    res = O.pcg(lambda v: O.normal_apply(v, mats, lam), lambda r: O.apply_separable(r, f), rhs, rtol=1e-6,
                max_iter=4000)
    assert res.converged
    return res.iters


@pytest.mark.parametrize("kind,lam", [("bspline", 1e-4), ("bspline", 1e-3), ("bspline", 1e-2), ("dense", 1e-3)])
def test_corner_model_shift_is_near_the_best_shift(kind, lam):
    """The model's shift takes at most two PCG iterations more than the best shift of the grid
    s = 1, 2, 4, .. 256 (oracle PCG to 1e-6), on B-spline instances over two decades of lambda
    (the best shift moves from 8 to 128 there) and on a dense instance."""
    if kind == "bspline":
        inst = synth.instance_bspline((16, 16, 16, 4), seed=3, lam=lam)
    else:
        inst = synth.instance_dense_3d(seed=1, n=12, m=18, lam=lam)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise.reshape(tuple(m.shape[0] for m in mats))
    rhs = O.apply_T(b, mats)
    s_model = O.corner_model_shift(mats, lam)
    best = min(_pcg_iters(mats, lam, 2.0 ** j, rhs) for j in range(9))
    assert _pcg_iters(mats, lam, s_model, rhs) <= best + 2


# ---- one-dimensional shear transforms (Table 1 rotation) ------------------------------

@pytest.mark.parametrize("kind", [1, 3])
def test_shear_by_integer_steps_moves_lines_exactly(kind):
    """Slope 1 about an integer centre moves line i_b by i_b - centre whole points: an exact shift
    with zeros entering (both kernels interpolate: h(0) = 1, h = 0 at the other integers)."""
    x = np.random.default_rng(50).standard_normal((7, 6, 3))
    y = O.shear(x, 0, 1, slope=1.0, center=2.0, kind=kind)
    ref = np.zeros_like(x)
    for ib in range(6):
        k = ib - 2
        for ia in range(7):
            if 0 <= ia - k < 7:
                ref[ia, ib] = x[ia - k, ib]
    np.testing.assert_allclose(y, ref, atol=1e-15)


def test_shear_reproduces_low_order_polynomials_inside():
    """Linear interpolation reproduces linear lines and cubic convolution (a = -1/2) quadratic ones
    exactly wherever every tap lies on the line; the resampling point is i_a - slope (i_b - c)."""
    n_a, n_b, slope, c = 24, 5, 0.37, 1.5
    ia = np.arange(n_a, dtype=np.float64)
    for kind, f, reach in ((1, lambda p: 2.0 * p + 1.0, 1), (3, lambda p: 0.5 * p * p - p + 3.0, 2)):
        x = np.stack([f(ia)] * n_b, axis=1)
        y = O.shear(x, 0, 1, slope=slope, center=c, kind=kind)
        for ib in range(n_b):
            pos = ia - slope * (ib - c)
            inside = (np.floor(pos) - (reach - 1) >= 0) & (np.floor(pos) + reach <= n_a - 1)
            np.testing.assert_allclose(y[inside, ib], f(pos[inside]), rtol=1e-12, atol=1e-12)


def test_three_shears_rotate_a_linear_image():
    """Shears with slopes tan(t/2) (mode 0 by mode 1), -sin t (mode 1 by mode 0), tan(t/2) (mode 0
    by mode 1), each about the centre, compose to sampling at c + R(t)(i - c) with R the rotation
    by t: exact for a linear image (linear interpolation) near the centre, where no tap leaves the
    grid in any of the three passes."""
    n, t = 41, np.deg2rad(30.0)
    c = (n - 1) / 2.0
    g = np.arange(n, dtype=np.float64)
    xx, yy = np.meshgrid(g, g, indexing="ij")
    f = lambda u, v: 0.7 * u - 1.3 * v + 4.0
    img = f(xx, yy)
    out = O.shear(img, 0, 1, np.tan(t / 2), c, kind=1)
    out = O.shear(out, 1, 0, -np.sin(t), c, kind=1)
    out = O.shear(out, 0, 1, np.tan(t / 2), c, kind=1)
    u = c + np.cos(t) * (xx - c) - np.sin(t) * (yy - c)
    v = c + np.sin(t) * (xx - c) + np.cos(t) * (yy - c)
    near = (xx - c) ** 2 + (yy - c) ** 2 <= 6.0 ** 2
    np.testing.assert_allclose(out[near], f(u, v)[near], rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("kind", [1, 3])
def test_three_shears_by_ninety_degrees_permute_exactly(kind):
    """At t = 90 degrees the slopes are 1, -1, 1 and every shift is whole: the three passes move
    point (i, j) to (2c - j, i) exactly near the centre, for either kernel."""
    n = 41
    c = (n - 1) // 2
    x = np.random.default_rng(51).standard_normal((n, n))
    out = O.shear(x, 0, 1, 1.0, c, kind=kind)
    out = O.shear(out, 1, 0, -1.0, c, kind=kind)
    out = O.shear(out, 0, 1, 1.0, c, kind=kind)
    for i in range(c - 4, c + 5):
        for j in range(c - 4, c + 5):
            if (i - c) ** 2 + (j - c) ** 2 <= 16:
                assert out[i, j] == x[2 * c - j, i]


# ---- discrete Fourier transform over several modes (Table 1) -----------------------------

@pytest.mark.parametrize("modes", [(0,), (1, 2), (0, 1, 2, 3), (3, 1)])
def test_dft_equals_numpy_fft(modes):
    """The separable DFT (one DFT matrix per listed mode) equals numpy's FFT over those axes, for a
    complex input and for a real one; the inverse equals numpy's ifftn and undoes the forward."""
    rng = np.random.default_rng(70)
    shape = (6, 5, 8, 3)
    re, im = rng.standard_normal(shape), rng.standard_normal(shape)
    fr, fi = O.dft(re, im, modes)
    ref = np.fft.fftn(re + 1j * im, axes=modes)
    np.testing.assert_allclose(fr + 1j * fi, ref, rtol=1e-12, atol=1e-12)
    fr0, fi0 = O.dft(re, None, modes)
    np.testing.assert_allclose(fr0 + 1j * fi0, np.fft.fftn(re, axes=modes), rtol=1e-12, atol=1e-12)
    br, bi = O.dft(fr, fi, modes, inverse=True)
    np.testing.assert_allclose(br + 1j * bi, np.fft.ifftn(fr + 1j * fi, axes=modes), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(br, re, atol=1e-12)
    np.testing.assert_allclose(bi, im, atol=1e-12)


def test_pin_catches_wrong_cubic_coefficient(monkeypatch):
    """Cubic convolution with a = -3/4 instead of -1/2 no longer reproduces quadratics, so the
    shear's reproduction pin would fail on it."""
    n_a, slope, c = 24, 0.37, 1.5
    ia = np.arange(n_a, dtype=np.float64)
    x = np.stack([0.5 * ia * ia - ia + 3.0] * 3, axis=1)
    pos = ia - slope * (2 - c)
    inside = (np.floor(pos) - 1 >= 0) & (np.floor(pos) + 2 <= n_a - 1)
    want = 0.5 * pos * pos - pos + 3.0
    good = O.shear(x, 0, 1, slope, c, kind=3)[:, 2]
    assert np.allclose(good[inside], want[inside], atol=1e-12)

    def keys_wrong(u, kind):
        u = np.abs(np.asarray(u, dtype=np.float64))
        a = -0.75
        near = (a + 2.0) * u**3 - (a + 3.0) * u**2 + 1.0
        far = a * u**3 - 5.0 * a * u**2 + 8.0 * a * u - 4.0 * a
        return np.where(u <= 1.0, near, np.where(u < 2.0, far, 0.0))

    monkeypatch.setattr(O, "shear_kernel", keys_wrong)
    bad = O.shear(x, 0, 1, slope, c, kind=3)[:, 2]
    assert not np.allclose(bad[inside], want[inside], atol=1e-6)


def test_pin_catches_conjugated_dft(monkeypatch):
    """A DFT with the exponent's sign flipped (the conjugate transform) fails the numpy pin."""
    rng = np.random.default_rng(71)
    re, im = rng.standard_normal((5, 6)), rng.standard_normal((5, 6))
    ref = np.fft.fftn(re + 1j * im, axes=(0, 1))
    r, i = O.dft(re, im, (0, 1))
    assert np.allclose(r + 1j * i, ref)
    rb, ib = O.dft(re, im, (0, 1), inverse=True)  # the conjugate kernel, divided by n
    assert not np.allclose((rb + 1j * ib) * re.size, ref)
