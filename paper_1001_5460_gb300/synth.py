"""Seeded synthetic inputs for the separable tensor-operator solve.

This module only draws and shapes inputs: factor matrices, ground-truth fields
and measurement noise.  It holds none of the method's arithmetic (no mode
product, no Gram factor, no regulariser, no solver), so both the CPU oracle and
the CUDA path can consume what it produces without sharing any of the method.

The workloads follow the paper's 4D spline reconstruction (Sec. 5): a field on a
regular 4D grid observed through a separable cubic B-spline sampling operator
(one 1D collocation matrix per mode, Eq. separable_transf), plus the small
dense-factor and batched variants used as test cases.

Conventions
-----------
* Tensors are dense C-order arrays, last mode fastest.
* A factor for mode k is an m_k x n_k matrix A_k (samples x unknowns).
* Banded B-spline factors are returned in "ELL-4" form: for each sample row i,
  ``col0[i]`` is the first column touched and ``w[i, c]`` the weight of column
  ``col0[i] + c`` (c = 0..3).  Columns outside [0, n) carry weight exactly 0.
* Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "bspline3",
    "sample_positions",
    "bspline_factor_ell4",
    "ell4_to_dense",
    "dense_gaussian_factor",
    "gaussian_blobs",
    "smooth_random_field",
    "Factor",
    "Instance",
    "instance_dense_3d",
    "instance_bspline",
    "instance_batched",
    "net_init_params",
]


def bspline3(u):
    """Centred cubic B-spline beta^3(u) (textbook piecewise cubic, support |u| < 2).

    beta^3(u) = 2/3 - u^2 + |u|^3 / 2      for |u| < 1
              = (2 - |u|)^3 / 6            for 1 <= |u| < 2
              = 0                          otherwise
    """
    a = np.abs(np.asarray(u, dtype=np.float64))
    out = np.zeros_like(a)
    inner = a < 1.0
    outer = (a >= 1.0) & (a < 2.0)
    out[inner] = 2.0 / 3.0 - a[inner] ** 2 + 0.5 * a[inner] ** 3
    out[outer] = (2.0 - a[outer]) ** 3 / 6.0
    return out


def sample_positions(n: int, m: int, rng: np.random.Generator, jitter: float = 0.3) -> np.ndarray:
    """Per-axis sample positions in grid units for m samples over n unknowns.

    Samples are spread uniformly with spacing h = n / m, each moved by a uniform
    jitter of +-``jitter`` sample spacings, and clipped to the grid [0, n-1]:
        t_i = clip((i + 0.5) h - 0.5 + u_i h, 0, n - 1),  u_i ~ U(-jitter, jitter).
    The positions are sorted by construction when jitter < 0.5.
    """
    h = n / m
    u = rng.uniform(-jitter, jitter, size=m)
    t = (np.arange(m) + 0.5) * h - 0.5 + u * h
    return np.clip(t, 0.0, n - 1.0)


def bspline_factor_ell4(n: int, m: int, rng: np.random.Generator, jitter: float = 0.3):
    """Cubic B-spline collocation factor A[i, j] = beta^3(t_i - j) in ELL-4 form.

    Returns ``(col0, w, t)``: int32 first column per row, float64 weights
    (m x 4) and the float64 sample positions.  The basis is truncated at the
    grid ends: columns outside [0, n) get weight 0.
    """
    t = sample_positions(n, m, rng, jitter)
    col0 = np.floor(t).astype(np.int64) - 1
    cols = col0[:, None] + np.arange(4)[None, :]
    w = bspline3(t[:, None] - cols)
    w[(cols < 0) | (cols >= n)] = 0.0
    return col0.astype(np.int32), w, t


def ell4_to_dense(col0: np.ndarray, w: np.ndarray, n: int) -> np.ndarray:
    """Expand an ELL-4 factor to its dense m x n matrix (weights outside [0, n) dropped)."""
    m = col0.shape[0]
    a = np.zeros((m, n), dtype=np.float64)
    for c in range(w.shape[1]):
        j = col0.astype(np.int64) + c
        ok = (j >= 0) & (j < n)
        a[np.nonzero(ok)[0], j[ok]] += w[ok, c]
    return a


def dense_gaussian_factor(m: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """Dense m x n factor with i.i.d. entries N(0, 1) / sqrt(m)."""
    return rng.standard_normal((m, n)) / math.sqrt(m)


def gaussian_blobs(shape, count: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Sum of ``count`` isotropic Gaussians on the integer grid of ``shape``.

    Centres are uniform over the grid box [0, n_k) per axis, amplitudes U(0.5, 1.5).
    """
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    out = np.zeros(shape, dtype=np.float64)
    for _ in range(count):
        c = [rng.uniform(0.0, s) for s in shape]
        amp = rng.uniform(0.5, 1.5)
        r2 = sum((g - ci) ** 2 for g, ci in zip(grids, c))
        out += amp * np.exp(-0.5 * r2 / sigma ** 2)
    return out


def smooth_random_field(shape, sigma: float, rng: np.random.Generator, dtype=np.float32) -> np.ndarray:
    """Gaussian-filtered N(0, 1) noise on every mode, normalised to unit RMS.

    The filter is ``scipy.ndimage.gaussian_filter`` with reflecting boundaries,
    truncated at 4 sigma.
    """
    from scipy import ndimage

    z = rng.standard_normal(shape, dtype=np.float32 if dtype == np.float32 else np.float64)
    f = ndimage.gaussian_filter(z, sigma=sigma, mode="reflect", truncate=4.0)
    rms = float(np.sqrt(np.mean(np.square(f, dtype=np.float64))))
    return (f / rms).astype(dtype)


@dataclasses.dataclass
class Factor:
    """One mode's factor: dense ``a`` (m x n), or ELL-4 ``col0``/``w``."""

    kind: str  # "dense" | "ell4"
    m: int
    n: int
    a: np.ndarray | None = None
    col0: np.ndarray | None = None
    w: np.ndarray | None = None

    def dense(self) -> np.ndarray:
        if self.kind == "dense":
            return np.asarray(self.a, dtype=np.float64)
        return ell4_to_dense(self.col0, self.w, self.n)


@dataclasses.dataclass
class Instance:
    """A synthetic problem: factors, ground truth, sample-space noise and lambda.

    The data is b = A x_true + noise; forming A x_true is the method's forward
    operator and is left to the caller (the oracle in tests, the library on the
    GPU), so this module stays free of the method's arithmetic.
    """

    shape: tuple
    factors: list
    x_true: np.ndarray
    noise: np.ndarray
    lam: float
    seed: int

    @property
    def sample_shape(self) -> tuple:
        return tuple(f.m for f in self.factors)


def instance_dense_3d(seed: int = 0, n: int = 16, m: int = 24, lam: float = 1e-3) -> Instance:
    """Tiny 3D problem with dense Gaussian factors (n^3 unknowns, m x n factors).

    X_true is a sum of 5 isotropic Gaussians (sigma = 3 voxels); the noise is
    N(0, 0.01^2) per sample.  Draw order: factors for modes 1..3, blobs, noise.
    """
    rng = np.random.default_rng(seed)
    factors = [Factor("dense", m, n, a=dense_gaussian_factor(m, n, rng)) for _ in range(3)]
    x_true = gaussian_blobs((n, n, n), 5, 3.0, rng)
    noise = 0.01 * rng.standard_normal((m, m, m))
    return Instance((n, n, n), factors, x_true, noise, lam, seed)


def instance_bspline(shape, seed: int, oversample: float = 1.5, lam: float = 1e-3,
                     sigma: float = 4.0, dtype=np.float32, with_truth: bool = True) -> Instance:
    """Banded problem: cubic B-spline collocation factors at jittered positions.

    ``m_k = round(oversample * n_k)`` samples per mode; X_true is a smooth random
    field (Gaussian-filtered noise, ``sigma`` voxels, unit RMS); noise N(0, 0.01^2).
    Draw order: factors for modes 1..d, field, noise.
    """
    rng = np.random.default_rng(seed)
    factors = []
    for n in shape:
        m = int(round(oversample * n))
        col0, w, _ = bspline_factor_ell4(n, m, rng)
        factors.append(Factor("ell4", m, n, col0=col0, w=w))
    ms = tuple(f.m for f in factors)
    if with_truth:
        x_true = smooth_random_field(tuple(shape), sigma, rng, dtype=dtype)
        noise = (0.01 * rng.standard_normal(ms, dtype=np.float32)).astype(dtype, copy=False)
    else:
        x_true = None
        noise = None
    return Instance(tuple(shape), factors, x_true, noise, lam, seed)


def instance_batched(index: int, base_seed: int = 100, lo: int = 24, hi: int = 96) -> Instance:
    """One of the uneven batched instances (seed = base_seed + index).

    Sizes n_k ~ U{lo..hi} (24..96 by default) for three modes and a 4th mode in
    {1, 4, 8} (1 means a 3D instance).  Even indices use dense Gaussian factors, odd ones B-spline
    factors; m_k = ceil(1.5 n_k); lambda is log-uniform in [1e-4, 1e-2].
    """
    seed = base_seed + index
    rng = np.random.default_rng(seed)
    dims = [int(rng.integers(lo, hi + 1)) for _ in range(3)]
    n4 = int(rng.choice([1, 4, 8]))
    if n4 > 1:
        dims.append(n4)
    lam = float(10.0 ** rng.uniform(-4.0, -2.0))
    dense = (index % 2) == 0
    factors = []
    for n in dims:
        m = int(math.ceil(1.5 * n))
        if dense:
            factors.append(Factor("dense", m, n, a=dense_gaussian_factor(m, n, rng)))
        else:
            col0, w, _ = bspline_factor_ell4(n, m, rng)
            factors.append(Factor("ell4", m, n, col0=col0, w=w))
    x_true = smooth_random_field(tuple(dims), 4.0, rng, dtype=np.float32)
    noise = 0.01 * rng.standard_normal(tuple(f.m for f in factors), dtype=np.float32)
    return Instance(tuple(dims), factors, x_true, noise, lam, seed)


@dataclasses.dataclass
class ScatteredInstance:
    """Samples at scattered positions: per mode k the ELL-4 rows (col0[k], w[k]) of an
    m x n_k matrix (row s: the cubic B-spline weights of sample s along mode k)."""

    shape: tuple
    col0: list
    w: list
    x_true: np.ndarray
    noise: np.ndarray
    lam: float
    seed: int

    @property
    def m(self) -> int:
        return int(self.col0[0].shape[0])


def instance_scattered(shape, m: int, seed: int, lam: float = 1e-3, sigma: float = 4.0) -> ScatteredInstance:
    """m samples at independent uniform positions in the grid box [0, n_k - 1] per axis (off the
    grid, in random order), cubic B-spline weights per mode with the truncated basis; x_true a
    smooth random field (unit RMS), noise N(0, 0.01^2).  Draw order: positions (m x d), field, noise."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, 1.0, size=(m, len(shape))) * (np.asarray(shape, dtype=np.float64) - 1.0)
    col0, w = [], []
    for k, n in enumerate(shape):
        c0 = np.floor(t[:, k]).astype(np.int64) - 1
        cols = c0[:, None] + np.arange(4)[None, :]
        wk = bspline3(t[:, k][:, None] - cols)
        wk[(cols < 0) | (cols >= n)] = 0.0
        col0.append(c0.astype(np.int32))
        w.append(wk)
    x_true = smooth_random_field(tuple(shape), sigma, rng, dtype=np.float64)
    noise = 0.01 * rng.standard_normal(m)
    return ScatteredInstance(tuple(shape), col0, w, x_true, noise, lam, seed)


NET_LAYERS = ((1, 32), (32, 32), (32, 32), (32, 1))  # (c_in, c_out) of the 4 convolution layers


def net_init_params(seed: int) -> np.ndarray:
    """Packed FP32 initial parameters of the 4-layer 3x3x3 network.

    Per layer: W[c_out][c_in][3][3][3] ~ N(0, 2 / (27 c_in)) (He-normal), the
    last layer scaled by 0.1, then b[c_out] = 0.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for li, (ci, co) in enumerate(NET_LAYERS):
        w = rng.standard_normal((co, ci, 3, 3, 3)) * math.sqrt(2.0 / (27 * ci))
        if li == len(NET_LAYERS) - 1:
            w *= 0.1
        parts += [w.ravel(), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)
