"""CPU FP64 oracle for the separable tensor-operator solve.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
definition that the CUDA library is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library itself never does, and this module imports nothing from the
library (it takes plain NumPy arrays).

Everything is NumPy float64.  Tensors are C-order arrays (last mode fastest),
so with the mode product below  vec(X x_1 A_1 ... x_d A_d) = (A_1 kron ... kron A_d) vec(X).

What each function follows in the paper (Morozov & Hunziker, "Solving Tensor
Structured Problems with Computational Tensor Algebra"):

* ``mode_product`` - tensor multiplication of a tensor by a one-dimensional
  transformation acting on one index: outer product then contraction
  (Sec. 2, Eq. first_product), restricted to one index pair.
* ``apply`` / ``apply_T`` - the separable transformation as a chain of
  one-dimensional transformations (Sec. 2.1, Eq. separable_transf), and its
  transpose (App. "Tensor transposition": A^T A patterns are a change of
  variance, i.e. each factor transposed).
* ``regulariser`` - a sum of single-mode finite-difference filters, the same
  structure as the separable Poisson operator of Sec. 4.1; the finite
  difference is one of the separable building blocks of Table 1.
* ``normal_apply`` - the normal-equations operator A^T A + lambda R obtained
  from differentiating the least-squares functional (App. "Differentiation in
  respect to a tensor", Eqs. A15-A17).  It is computed the long way, through
  sample space, and never through per-mode Gram factors.
* ``cg`` - the tensor conjugate-gradient iteration of Fig. 2, with the inner
  product of App. "Inner product" (Eq. A14).
* ``separable_inverse_factors`` / ``apply_separable`` / ``pcg`` - the same
  iteration preconditioned by a tensor inverse (Sec. 3, Eq. TensorEq): for a
  separable transformation the tensor inverse is the separable transformation
  of the per-mode inverses, so the inverse of the separable approximation
  (A_1^T A_1 + s lambda L_1) x ... x (A_d^T A_d + s lambda L_d) of K is applied
  mode by mode.  The approximation keeps the Gram part of K exactly and spreads
  the regulariser over the modes with weight s (a reading: the paper fixes no
  preconditioner).
* ``scattered_apply`` / ``scattered_apply_T`` / ``scattered_normal_apply`` - the
  system tensor of scattered (off-grid) samples (Sec. 2.2, repeated indices; the
  real 4D problem of Sec. 5): sample s weights unknown (i_1..i_d) by the product
  of its per-mode weights A_k[s, i_k], i.e. the rows of A are the Kronecker
  products of the rows of the A_k (the row-wise, face-splitting product), and
  A^T A is a sum over samples of rank-1 tensor products.  Written out term by
  term over each sample's non-zero window.
* ``corner_model_shift`` - the shift s of that preconditioner from a model of the
  spectrum of M^-1 K (a reading: the paper fixes no preconditioner): each mode
  either at its smooth corner (Gram at its top eigenvalue, regulariser at zero)
  or at its rough corner (Gram at its bottom eigenvalue, regulariser at its
  top), and s minimises the spread max/min of K/M over the 2^d corners.
* ``tmg_prolongation`` / ``tmg_vcycle`` - a two-grid tensor multigrid cycle as a CG
  preconditioner (Sec. 4.2, Fig. 3): separable linear-interpolation transfers (Table 1
  upsampling and its transpose), Galerkin coarse operator, Chebyshev smoothing on the
  Jacobi-scaled operator (the smoother is a reading: the paper names none).
* ``shear_kernel`` / ``shear`` - the one-dimensional shear transform of Table 1's rotation
  row: every line along one mode resampled at positions moved in proportion to the index of
  another mode, by linear interpolation or cubic convolution (the interpolation is a reading:
  the paper names none).
* ``dft`` - the discrete Fourier transform of Table 1 over several modes: the complex
  tensor multiplied along each mode by its DFT matrix (the definition, not an FFT).
* ``kron_matrix`` / ``dense_normal_matrix`` / ``direct_solve`` - the
  equivalent matrix form of a tensor equation "with proper reshaping" (Sec. 3,
  after Eq. TensorEq), solved by a direct (Cholesky) method - the direct-solver
  class of Sec. 4.1.  For tiny cases only.

Readings where the paper is silent or garbled (also listed in the design notes):
* the CG loop condition in Fig. 2 is printed inverted; CG stops when the
  relative recursive residual sqrt(rho) / ||rhs|| <= rtol;
* the second-difference operator is the "valid" (n-2) x n matrix with rows
  [1, -2, 1]; modes with n < 3 carry no regulariser;
* the same lambda weights every mode.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np

__all__ = [
    "mode_product",
    "apply",
    "apply_T",
    "second_difference",
    "regulariser",
    "normal_apply",
    "inner",
    "cg",
    "separable_inverse_factors",
    "apply_separable",
    "pcg",
    "solve",
    "rel_residual",
    "kron_matrix",
    "dense_normal_matrix",
    "direct_solve",
    "CGResult",
    "scattered_apply",
    "scattered_apply_T",
    "scattered_normal_apply",
    "scattered_rows_matrix",
    "jacobi_diagonal",
    "corner_model_shift",
    "tmg_prolongation",
    "tmg_vcycle",
    "shear_kernel",
    "shear",
    "dft",
]


def mode_product(x: np.ndarray, a: np.ndarray, k: int) -> np.ndarray:
    """Y = X x_k A:  Y[..., j, ...] = sum_i A[j, i] X[..., i, ...] on index k.

    Outer product of A with X followed by contraction of A's second index with
    X's k-th index (Sec. 2, Eq. first_product for a single index pair).  The new
    index takes the place of the contracted one (ordered spaces, Sec. 2.1).
    """
    x = np.asarray(x, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    if a.shape[1] != x.shape[k]:
        raise ValueError(f"factor {a.shape} does not match mode {k} of {x.shape}")
    y = np.tensordot(a, x, axes=([1], [k]))  # new index first
    return np.moveaxis(y, 0, k)


def apply(x: np.ndarray, mats, order=None) -> np.ndarray:
    """Separable transformation A x = X x_1 A_1 x_2 A_2 ... x_d A_d (Eq. separable_transf).

    ``order`` is the sequence in which the one-dimensional transformations are
    applied; by commutativity on ordered spaces (Sec. 2.1) any order gives the
    same result.
    """
    y = np.asarray(x, dtype=np.float64)
    for k in (range(len(mats)) if order is None else order):
        y = mode_product(y, mats[k], k)
    return y


def apply_T(y: np.ndarray, mats, order=None) -> np.ndarray:
    """Transpose A^T y = Y x_1 A_1^T ... x_d A_d^T (App. "Tensor transposition")."""
    x = np.asarray(y, dtype=np.float64)
    for k in (range(len(mats)) if order is None else order):
        x = mode_product(x, np.asarray(mats[k], dtype=np.float64).T, k)
    return x


def second_difference(n: int) -> np.ndarray:
    """(n-2) x n second-difference matrix with rows [1, -2, 1] (Table 1, finite difference)."""
    d = np.zeros((max(n - 2, 0), n), dtype=np.float64)
    for i in range(n - 2):
        d[i, i] = 1.0
        d[i, i + 1] = -2.0
        d[i, i + 2] = 1.0
    return d


def regulariser(x: np.ndarray, lam: float) -> np.ndarray:
    """lambda * sum_k X x_k (D2_k^T D2_k), skipping modes with n_k < 3.

    A sum of single-mode filters, as in the separable Poisson operator (Sec. 4.1).
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for k, n in enumerate(x.shape):
        if n < 3:
            continue
        d2 = second_difference(n)
        out += mode_product(x, d2.T @ d2, k)
    return lam * out


def normal_apply(x: np.ndarray, mats, lam: float) -> np.ndarray:
    """K x = A^T (A x) + lambda R x, the long way through sample space.

    K is the normal-equations operator of the regularised least-squares
    functional ||A x - b||^2 + lambda sum_k ||X x_k D2_k||^2 (App., Eqs. A15-A17).
    """
    return apply_T(apply(x, mats), mats) + regulariser(x, lam)


def inner(a: np.ndarray, b: np.ndarray) -> float:
    """<A, B> = sum of the elementwise product (App. "Inner product", Eq. A14)."""
    return float(np.sum(np.asarray(a, np.float64) * np.asarray(b, np.float64)))


class CGResult:
    """Outcome of ``cg``: solution, iteration count and relative-residual history."""

    def __init__(self, x, iters, history, converged):
        self.x = x
        self.iters = iters
        self.history = history
        self.converged = converged


def cg(kop, rhs: np.ndarray, x0: np.ndarray | None = None, rtol: float = 1e-10,
       max_iter: int = 10000) -> CGResult:
    """Tensor conjugate gradients of Fig. 2 for K x = rhs with SPD K.

    Steps, in the figure's order and names (C is the solution, B the data):
        R = B - K C;  P = R;  rho = <R, R>
        repeat:  Q = K P;  alpha = rho / <P, Q>;  C = C + alpha P;
                 R = R - alpha Q;  rho1 = <R, R>;  P = R + (rho1 / rho) P;  rho = rho1
    stopping when sqrt(rho) / ||B|| <= rtol (the figure prints this test inverted).
    """
    b = np.asarray(rhs, dtype=np.float64)
    c = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.sqrt(inner(b, b))
    if bnorm == 0.0:
        return CGResult(np.zeros_like(b), 0, [0.0], True)
    r = b - kop(c)
    p = r.copy()
    rho = inner(r, r)
    history = [np.sqrt(rho) / bnorm]
    it = 0
    while history[-1] > rtol and it < max_iter:
        q = kop(p)
        alpha = rho / inner(p, q)
        c = c + alpha * p
        r = r - alpha * q
        rho1 = inner(r, r)
        p = r + (rho1 / rho) * p
        rho = rho1
        it += 1
        history.append(np.sqrt(rho) / bnorm)
    return CGResult(c, it, history, history[-1] <= rtol)


def separable_inverse_factors(mats, lam: float, shift: float, half_band: int | None = None) -> list:
    """Per-mode factors (A_k^T A_k + shift * lam * D2_k^T D2_k)^-1 of the preconditioner.

    The tensor inverse of a separable transformation (Sec. 3, Eq. TensorEq with
    A = A_1 x ... x A_d) is the separable transformation of the per-mode
    inverses; modes with n_k < 3 carry no regulariser, as in ``regulariser``.
    With ``half_band`` h, each inverse keeps only its entries with |i - j| <= h
    (a symmetric band; for banded factors the inverses decay away from the
    diagonal, so a band as wide as the Gram band keeps most of the effect).
    """
    out = []
    for a in mats:
        a = np.asarray(a, dtype=np.float64)
        n = a.shape[1]
        m = a.T @ a
        if n >= 3:
            d2 = second_difference(n)
            m = m + (shift * lam) * (d2.T @ d2)
        inv = np.linalg.inv(m)
        inv = 0.5 * (inv + inv.T)  # the inverse of the SPD M_k is symmetric; drop rounding asymmetry
        if half_band is not None:
            idx = np.arange(n)
            inv = np.where(np.abs(idx[:, None] - idx[None, :]) <= half_band, inv, 0.0)
        out.append(inv)
    return out


def corner_model_shift(mats, lam: float, steps: int = 16) -> float:
    """The shift s of M = (x)_k (G_k + s lam L_k) (``separable_inverse_factors``) chosen on the
    grid s = 2^(j/2), j = 0 .. steps, from a corner model of the spectrum of M^-1 K.

    Mode k contributes one of two corners: (g_max, 0), its Gram G_k = A_k^T A_k at its top
    eigenvalue and the regulariser at zero (smooth components), or (g_min, lam l_max), the
    Gram at its bottom eigenvalue and lam L_k = lam D2^T D2 at its top (rough components; a
    mode with n_k < 3 has l_max = 0).  At a corner c the operator K = (x)G_k + lam sum L_k
    is modelled by prod g + sum l and M by prod (g + s l); s minimises
    max_c (K_c / M_c) / min_c (K_c / M_c) (the first grid point of the minimum; corners with
    M_c = 0 are left out).
    """
    corners = []
    for a in mats:
        a = np.asarray(a, dtype=np.float64)
        n = a.shape[1]
        g = np.linalg.eigvalsh(a.T @ a)
        l_max = 0.0
        if n >= 3:
            d2 = second_difference(n)
            l_max = float(np.linalg.eigvalsh(d2.T @ d2)[-1])
        corners.append(((float(g[-1]), 0.0), (float(g[0]), lam * l_max)))
    best_s, best_k = 1.0, None
    for j in range(steps + 1):
        shift = 2.0 ** (j / 2)
        ratios = []
        for c in itertools.product(*corners):
            k_c = float(np.prod([g for g, _ in c])) + sum(l for _, l in c)
            m_c = float(np.prod([g + shift * l for g, l in c]))
            if m_c > 0.0:
                ratios.append(k_c / m_c)
        spread = max(ratios) / min(ratios)
        if best_k is None or spread < best_k:
            best_s, best_k = shift, spread
    return best_s


def jacobi_diagonal(mats, lam: float, shape) -> np.ndarray:
    """diag(K) of K = A^T A + lam R as an n-shaped tensor: the point-Jacobi
    preconditioner of the Fig. 1 solver family.

    Written from the definitions: the diagonal entry of the Kronecker product
    A_1^T A_1 x ... x A_d^T A_d at (i_1, ..., i_d) is the product of the
    per-mode diagonal entries, and the regulariser sum_k I x .. x D2_k^T D2_k x
    .. x I adds the k-th mode's diagonal entry of D2_k^T D2_k (modes with
    n_k < 3 carry none, as in ``regulariser``).
    """
    d = len(shape)
    diag = np.ones(tuple(shape), dtype=np.float64)
    for k, a in enumerate(mats):
        a = np.asarray(a, dtype=np.float64)
        g = np.sum(a * a, axis=0)  # (A^T A)[i, i] = sum over rows of A[:, i]^2
        view = [1] * d
        view[k] = shape[k]
        diag = diag * g.reshape(view)
    for k in range(d):
        n = shape[k]
        if n < 3:
            continue
        d2 = second_difference(n)
        l = np.sum(d2 * d2, axis=0)
        view = [1] * d
        view[k] = n
        diag = diag + lam * l.reshape(view)
    return diag


def apply_separable(x: np.ndarray, factors) -> np.ndarray:
    """X x_1 F_1 ... x_d F_d for square per-mode factors (Sec. 2.1, Eq. separable_transf)."""
    x = np.asarray(x, dtype=np.float64)
    for k, f in enumerate(factors):
        x = mode_product(x, f, k)
    return x


def pcg(kop, minv, rhs: np.ndarray, x0: np.ndarray | None = None, rtol: float = 1e-10,
        max_iter: int = 10000) -> CGResult:
    """Fig. 2's CG for K x = rhs preconditioned by the SPD operator ``minv`` (Z = M^-1 R).

    Steps, in the figure's order, with rho = <R, Z> in place of <R, R>:
        R = B - K C;  Z = M^-1 R;  P = Z;  rho = <R, Z>
        repeat:  Q = K P;  alpha = rho / <P, Q>;  C = C + alpha P;  R = R - alpha Q;
                 (stop when ||R|| / ||B|| <= rtol)
                 Z = M^-1 R;  rho1 = <R, Z>;  P = Z + (rho1 / rho) P;  rho = rho1
    With ``minv`` the identity this is ``cg`` step for step.  The history holds
    ||R|| / ||B|| (the recursive residual), as in ``cg``.
    """
    b = np.asarray(rhs, dtype=np.float64)
    c = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.sqrt(inner(b, b))
    if bnorm == 0.0:
        return CGResult(np.zeros_like(b), 0, [0.0], True)
    r = b - kop(c)
    history = [np.sqrt(inner(r, r)) / bnorm]
    if history[-1] <= rtol:
        return CGResult(c, 0, history, True)
    z = minv(r)
    p = z.copy()
    rho = inner(r, z)
    it = 0
    while it < max_iter:
        q = kop(p)
        alpha = rho / inner(p, q)
        c = c + alpha * p
        r = r - alpha * q
        it += 1
        history.append(np.sqrt(inner(r, r)) / bnorm)
        if history[-1] <= rtol:
            break
        z = minv(r)
        rho1 = inner(r, z)
        p = z + (rho1 / rho) * p
        rho = rho1
    return CGResult(c, it, history, history[-1] <= rtol)


def solve(b: np.ndarray, mats, lam: float, rtol: float = 1e-10, max_iter: int = 10000,
          x0: np.ndarray | None = None) -> CGResult:
    """Solve (A^T A + lambda R) x = A^T b by the CG of Fig. 2, from x0 = 0 unless given."""
    rhs = apply_T(b, mats)
    return cg(lambda v: normal_apply(v, mats, lam), rhs, x0=x0, rtol=rtol, max_iter=max_iter)


def rel_residual(x: np.ndarray, b: np.ndarray, mats, lam: float) -> float:
    """True relative residual ||A^T b - K x|| / ||A^T b|| of the normal equations."""
    rhs = apply_T(b, mats)
    r = rhs - normal_apply(x, mats, lam)
    return float(np.sqrt(inner(r, r)) / np.sqrt(inner(rhs, rhs)))


def _window_terms(col0s, ws, shape):
    """For each combination of per-mode taps (a_1..a_d): the weight product over samples and the
    flat grid index (-1 where a tap falls outside the grid)."""
    d = len(shape)
    m = col0s[0].shape[0]
    width = [w.shape[1] for w in ws]
    for taps in itertools.product(*[range(t) for t in width]):
        wt = np.ones(m)
        flat = np.zeros(m, dtype=np.int64)
        ok = np.ones(m, dtype=bool)
        for k in range(d):
            idx = np.asarray(col0s[k], dtype=np.int64) + taps[k]
            wt = wt * np.asarray(ws[k], dtype=np.float64)[:, taps[k]]
            ok &= (idx >= 0) & (idx < shape[k])
            flat = flat * shape[k] + np.where(ok, idx, 0)
        yield wt, np.where(ok, flat, -1)


def scattered_apply(x: np.ndarray, col0s, ws) -> np.ndarray:
    """(A x)_s = sum over the taps a_k of prod_k w_k[s, a_k] * x[col0_1[s] + a_1, ..., col0_d[s] + a_d]
    for scattered samples: mode k's weights of sample s sit in columns col0_k[s] .. col0_k[s] + 3
    (a row of an m x n_k ELL-4 matrix); taps outside the grid are dropped."""
    x = np.asarray(x, dtype=np.float64)
    xf = x.ravel()
    y = np.zeros(col0s[0].shape[0])
    for wt, flat in _window_terms(col0s, ws, x.shape):
        ok = flat >= 0
        y[ok] += wt[ok] * xf[flat[ok]]
    return y


def scattered_apply_T(y: np.ndarray, col0s, ws, shape) -> np.ndarray:
    """x = A^T y for scattered samples: every sample adds y_s times its weight product to each
    unknown of its window."""
    y = np.asarray(y, dtype=np.float64)
    xf = np.zeros(int(np.prod(shape)))
    for wt, flat in _window_terms(col0s, ws, shape):
        ok = flat >= 0
        np.add.at(xf, flat[ok], wt[ok] * y[ok])
    return xf.reshape(shape)


def scattered_normal_apply(x: np.ndarray, col0s, ws, lam: float) -> np.ndarray:
    """(A^T A + lam R) x for scattered samples, through sample space (as ``normal_apply``)."""
    x = np.asarray(x, dtype=np.float64)
    return scattered_apply_T(scattered_apply(x, col0s, ws), col0s, ws, x.shape) + regulariser(x, lam)


def scattered_rows_matrix(col0s, ws, shape) -> np.ndarray:
    """Explicit m x N matrix of the scattered system tensor: row s is the Kronecker product of
    the samples' dense per-mode rows (tiny cases only)."""
    m = col0s[0].shape[0]
    rows = []
    for s_ in range(m):
        dense_rows = []
        for k, n in enumerate(shape):
            r = np.zeros(n)
            for a in range(ws[k].shape[1]):
                j = int(col0s[k][s_]) + a
                if 0 <= j < n:
                    r[j] += ws[k][s_, a]
            dense_rows.append(r)
        rows.append(functools.reduce(np.kron, dense_rows))
    return np.array(rows)


def tmg_prolongation(n: int) -> np.ndarray:
    """Linear interpolation from ceil(n / 2) coarse points (the even fine points) to n fine points:
    the upsampling building block of Table 1; its transpose is the restriction."""
    nc = (n + 1) // 2
    p = np.zeros((n, nc))
    for i in range(nc):
        p[2 * i, i] = 1.0
        if 2 * i + 1 < n:
            p[2 * i + 1, i] += 0.5
            if i + 1 < nc:
                p[2 * i + 1, i + 1] += 0.5
    return p


def tmg_vcycle(r: np.ndarray, kop, diag: np.ndarray, prolongs, nu: int, lam_lo: float, lam_hi: float,
               coarse_rtol: float = 1e-12) -> np.ndarray:
    """One two-grid tensor multigrid cycle (Sec. 4.2, Fig. 3) as a CG preconditioner z = V r.

    The transfers are separable (P = P_1 x ... x P_d, one one-dimensional interpolation per mode;
    restriction = P^T), the coarse operator is Galerkin, K_c = P^T K P (applied matrix-free), and
    the coarse system is solved to coarse_rtol by ``cg``.  Smoothing: nu steps of Chebyshev
    iteration on D^-1 K (D = diag(K)) over the interval [lam_lo, lam_hi], before and after the
    coarse correction (the same polynomial, so V is symmetric).
    """
    def smooth(z):
        theta, delta = 0.5 * (lam_hi + lam_lo), 0.5 * (lam_hi - lam_lo)
        res = r - kop(z)
        d = res / diag / theta
        z = z + d
        sigma = theta / delta
        rho = 1.0 / sigma
        for _ in range(nu - 1):
            res = r - kop(z)
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * (res / diag)
            z = z + d
            rho = rho_new
        return z

    z = smooth(np.zeros_like(r)) if nu > 0 else np.zeros_like(r)
    rc = apply_T(r - kop(z), prolongs)
    zc = cg(lambda v: apply_T(kop(apply(v, prolongs)), prolongs), rc, rtol=coarse_rtol, max_iter=100000).x
    z = z + apply(zc, prolongs)
    return smooth(z) if nu > 0 else z


def shear_kernel(u, kind: int) -> np.ndarray:
    """Interpolation kernel h(u) of a one-dimensional shear transform: kind 1 the linear (hat)
    kernel max(0, 1 - |u|); kind 3 cubic convolution with a = -1/2 (Keys 1981):
    (a + 2)|u|^3 - (a + 3)|u|^2 + 1 on |u| <= 1, a|u|^3 - 5a|u|^2 + 8a|u| - 4a on 1 < |u| < 2,
    0 beyond.  Both are interpolating: h(0) = 1 and h vanishes at the other integers."""
    u = np.abs(np.asarray(u, dtype=np.float64))
    if kind == 1:
        return np.maximum(0.0, 1.0 - u)
    if kind == 3:
        a = -0.5
        near = (a + 2.0) * u**3 - (a + 3.0) * u**2 + 1.0
        far = a * u**3 - 5.0 * a * u**2 + 8.0 * a * u - 4.0 * a
        return np.where(u <= 1.0, near, np.where(u < 2.0, far, 0.0))
    raise ValueError("kind must be 1 (linear) or 3 (cubic convolution)")


def shear(x: np.ndarray, mode_a: int, mode_b: int, slope: float, center: float, kind: int = 1) -> np.ndarray:
    """One-dimensional shear transform along mode a driven by mode b (Table 1: rotation as a
    product of 1D shear transforms).  Each line along mode a is resampled at positions moved by
    slope * (i_b - center):

        Y[.., i_a, .., i_b, ..] = sum_j h(i_a - slope * (i_b - center) - j) X[.., j, .., i_b, ..]

    with j over the line's n_a points (nothing outside them) and h = ``shear_kernel``.  Written
    as one explicit n_a x n_a matrix per value of i_b."""
    x = np.asarray(x, dtype=np.float64)
    if mode_a == mode_b:
        raise ValueError("a shear needs two different modes")
    xm = np.moveaxis(x, (mode_a, mode_b), (0, 1))
    n_a, n_b = xm.shape[0], xm.shape[1]
    y = np.zeros_like(xm)
    idx = np.arange(n_a, dtype=np.float64)
    for ib in range(n_b):
        pos = idx - slope * (ib - center)
        h = shear_kernel(pos[:, None] - idx[None, :], kind)
        y[:, ib] = np.tensordot(h, xm[:, ib], axes=(1, 0))
    return np.moveaxis(y, (0, 1), (mode_a, mode_b))


def dft(re: np.ndarray, im: np.ndarray | None, modes, inverse: bool = False):
    """Discrete Fourier transform over the given modes as a separable transformation (Table 1:
    F = E G H C with one-dimensional DFT transforms): the complex tensor re + i im multiplied along
    each listed mode k by the n_k x n_k matrix F_k[j, i] = exp(-2 pi i j i / n_k) (inverse:
    exp(+2 pi i j i / n_k) / n_k).  Returns the real and imaginary parts."""
    z = np.asarray(re, dtype=np.float64) + (0.0 if im is None else 1j * np.asarray(im, dtype=np.float64))
    z = z.astype(np.complex128)
    for k in modes:
        n = z.shape[k]
        jk = np.outer(np.arange(n), np.arange(n))
        f = np.exp((2j if inverse else -2j) * np.pi * jk / n)
        if inverse:
            f = f / n
        z = np.moveaxis(np.tensordot(f, np.moveaxis(z, k, 0), axes=(1, 0)), 0, k)
    return z.real.copy(), z.imag.copy()


def kron_matrix(mats) -> np.ndarray:
    """Explicit matrix A_1 kron ... kron A_d of the separable operator (Sec. 3, matrix form)."""
    return functools.reduce(np.kron, [np.asarray(a, np.float64) for a in mats])


def dense_normal_matrix(mats, lam: float, shape) -> np.ndarray:
    """Explicit K = A^T A + lambda sum_k (I kron .. D2_k^T D2_k .. kron I) for tiny cases."""
    a = kron_matrix(mats)
    k = a.T @ a
    for mode, n in enumerate(shape):
        if n < 3:
            continue
        d2 = second_difference(n)
        parts = [np.eye(s) for s in shape]
        parts[mode] = d2.T @ d2
        k = k + lam * functools.reduce(np.kron, parts)
    return k


def direct_solve(b: np.ndarray, mats, lam: float, shape) -> np.ndarray:
    """Direct solve of the reshaped normal equations by Cholesky (Sec. 4.1 direct solvers)."""
    from scipy import linalg

    a = kron_matrix(mats)
    k = dense_normal_matrix(mats, lam, shape)
    rhs = a.T @ np.asarray(b, np.float64).ravel()
    x = linalg.cho_solve(linalg.cho_factor(k), rhs)
    return x.reshape(shape)


def _support(a: np.ndarray, rows=None, cols=None):
    """Nonzero columns of the given rows (or nonzero rows of the given columns) of a."""
    a = np.asarray(a, np.float64)
    if rows is not None:
        return np.nonzero(np.any(a[rows, :] != 0.0, axis=0))[0]
    return np.nonzero(np.any(a[:, cols] != 0.0, axis=1))[0]


def apply_at(x: np.ndarray, mats, s_idx) -> float:
    """(A x)[s] for one sample multi-index s, from Eq. separable_transf restricted
    to the columns the rows s_k touch (all other terms are exact zeros)."""
    cols = [_support(a, rows=[sk]) for a, sk in zip(mats, s_idx)]
    blk = np.asarray(x, np.float64)[np.ix_(*cols)]
    rows = [np.asarray(a, np.float64)[[sk]][:, c] for a, sk, c in zip(mats, s_idx, cols)]
    return float(apply(blk, rows).reshape(()))


def normal_apply_at(x: np.ndarray, mats, lam: float, idx) -> float:
    """(K x)[i] for one unknown multi-index i, the long way through sample space:
    (A^T A x)[i] = sum_s (kron_k A_k[s_k, i_k]) (A x)[s] over the samples s whose
    rows touch i, plus lambda sum_k (x x_k D2_k^T D2_k)[i]."""
    x = np.asarray(x, np.float64)
    srows = [_support(a, cols=[ik]) for a, ik in zip(mats, idx)]          # samples touching i
    ccols = [_support(a, rows=sr) for a, sr in zip(mats, srows)]          # columns those samples read
    blk = x[np.ix_(*ccols)]
    sub = [np.asarray(a, np.float64)[np.ix_(sr, cc)] for a, sr, cc in zip(mats, srows, ccols)]
    ax = apply(blk, sub)                                                  # (A x) on the touching samples
    wi = [np.asarray(a, np.float64)[sr, ik][None, :] for a, sr, ik in zip(mats, srows, idx)]
    val = float(apply(ax, wi).reshape(()))                                # contract with A_k[s_k, i_k]
    for k, n in enumerate(x.shape):
        if n < 3:
            continue
        d2 = second_difference(n)
        row = (d2.T @ d2)[idx[k]]
        line = x[tuple(idx[:k]) + (slice(None),) + tuple(idx[k + 1:])]
        val += lam * float(row @ line)
    return val


def all_mode_orders(d: int):
    """Every order of the d one-dimensional transformations (for commutativity checks)."""
    return list(itertools.permutations(range(d)))
