/*
 * tca.h - C ABI of the GB300 separable tensor-operator solver.
 *
 * The library computes with tensors on ordered vector spaces as in Morozov &
 * Hunziker, "Solving Tensor Structured Problems with Computational Tensor
 * Algebra":
 *   - a tensor is a dense array of components on an ordered set of spaces
 *     (Sec. 2, Sec. 2.1; App. "Tensor notation");
 *   - the system tensor is separable, A = A_1 . A_2 . A_3 (. A_4): one
 *     one-dimensional transformation per space, applied as chained mode
 *     products in any order (Sec. 2.1, Eq. separable_transf and the
 *     commutativity statement that follows it);
 *   - the tensor equation A . U = B (Sec. 3, Eq. TensorEq) is solved in the
 *     least-squares sense through the normal equations
 *     (A^T A + lambda R) x = A^T b (App. "Tensor transposition", App.
 *     "Differentiation in respect to a tensor", Eqs. A15-A17) by the tensor
 *     conjugate gradient of Sec. 4.1, Fig. 2.
 *
 * Layout.  Every tensor is a dense C-order array (last mode fastest).  An
 * order-d unknown tensor has shape n[0..d-1]; the data (sample) tensor has
 * shape m[0..d-1], where m[k] is the row count of factor k.  With this layout
 * vec(X x_1 A_1 ... x_d A_d) = (A_1 kron ... kron A_d) vec(X).
 *
 * Element type.  Data buffers hold double for a TCA_F64 plan and float for
 * every other precision.
 *
 * Pointers.  Data pointers passed to tca_apply, tca_apply_T, tca_apply_normal,
 * tca_apply_mode and tca_solve may be device pointers (cudaMalloc, torch) or
 * host pointers (pageable or pinned).  Host buffers are staged through the
 * plan's own device buffers on the given stream, and the call then returns
 * only after the result is back in host memory.  Device-pointer calls are
 * asynchronous on the stream, except tca_solve, which synchronises the stream
 * to fill its info record.
 *
 * Ownership.  The caller owns every data buffer.  tca_plan copies the factors
 * it is given (host memory) and owns its device copies and workspace;
 * tca_destroy frees them.  A plan may be used by one stream at a time.
 *
 * Errors.  No call aborts or throws across this boundary: every failure comes
 * back as a tca_status.  A CUDA error is reported as TCA_ERR_CUDA and
 * tca_last_error_string() gives the CUDA message.  Device-side waits are
 * bounded: a wait that gives up sets a device flag and its kernel finishes
 * without waiting further (its output is then invalid); tca_solve,
 * tca_solve_batched and tca_solve_net report the flag as TCA_ERR_TIMEOUT, and
 * tca_check_timeout reads it after asynchronous calls.
 */
#ifndef TCA_H
#define TCA_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define TCA_API __attribute__((visibility("default")))
#else
#define TCA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TCA_OK = 0,
  TCA_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, negative size */
  TCA_ERR_SHAPE = 2,         /* factor or tensor shapes do not match */
  TCA_ERR_UNSUPPORTED = 3,   /* valid request this build does not implement */
  TCA_ERR_ALLOC = 4,         /* device allocation failed */
  TCA_ERR_CUDA = 5,          /* a CUDA runtime/driver call failed */
  TCA_ERR_NOT_CONVERGED = 6, /* solve hit max_iter; x holds the last iterate */
  TCA_ERR_BREAKDOWN = 7,     /* CG met <p, Kp> <= 0 or a non-finite scalar */
  TCA_ERR_TIMEOUT = 8        /* a bounded device wait gave up */
} tca_status;

/* Arithmetic of a plan.  TCA_F64: double data, double arithmetic.  TCA_F32:
 * float data and arithmetic, inner products accumulated to double (dense
 * factors: 3xTF32 tensor-core products, about FP32 accuracy).  The _IR forms
 * keep float data at the boundary and solve by iterative refinement: an
 * outer loop on the FP64-accurate (double-float) residual and an inner CG to
 * a loose tolerance with a reduced-precision operator:
 *   TCA_TF32_IR  plain TF32 tensor-core products for dense factors; banded
 *                factors keep the FP32 sweep;
 *   TCA_BF16_IR  banded (ELL4) factors only: the inner CG keeps r, p and q in
 *                bfloat16 and applies the normal operator with the modes-3/4
 *                contraction (G_3 kron G_4 and its regulariser) on the tensor
 *                cores in BF16 with FP32 accumulation, modes 1-2 in FP32;
 *                tca_apply_normal rounds x to bfloat16 and returns K x through
 *                the same sweep (tca_apply / tca_apply_T stay FP32).  tca_plan
 *                returns TCA_ERR_UNSUPPORTED for dense factors, n4 > 8 or an
 *                inner axis n3*n4 (n3 for order 3) that is not a multiple of 8.
 * CG scalars and every inner product stay FP64 in all forms. */
typedef enum { TCA_F64 = 0, TCA_F32 = 1, TCA_BF16_IR = 2, TCA_TF32_IR = 3 } tca_precision;

typedef enum {
  TCA_FACTOR_DENSE = 0, /* values: m*n doubles, row-major A[i][j] */
  TCA_FACTOR_ELL4 = 1   /* values: m*4 doubles, col0: m int32; row i holds
                           A[i][col0[i]+c] = values[4*i+c], c = 0..3.  Columns
                           outside [0, n) are ignored.  col0 must be
                           non-decreasing in i. */
} tca_factor_kind;

/* One mode's one-dimensional transformation A_k (m x n), in host memory. */
typedef struct {
  int32_t kind;          /* tca_factor_kind */
  int32_t reserved;      /* must be 0 */
  int64_t m;             /* rows: samples along this mode */
  int64_t n;             /* columns: unknowns along this mode */
  const double* values;  /* host */
  const int32_t* col0;   /* host, ELL4 only (NULL for DENSE) */
} tca_factor;

/* Regulariser lambda * sum_k (I x .. x D2_k^T D2_k x .. x I) with D2_k the
 * (n_k-2) x n_k second difference; a mode takes part when its bit is set in
 * reg_mode_mask and n_k >= 3.  This is a sum of single-mode finite-difference
 * filters, the structure of the separable Poisson operator of Sec. 4.1. */
typedef struct {
  double lambda;
  uint32_t reg_mode_mask;
  uint32_t reserved;
} tca_reg;

typedef struct tca_plan_s* tca_plan_t;

/* Build a plan: define the ordered spaces (sizes n[0..order-1], as with
 * World.DefineSpace in Sec. 4.1, Fig. 1c) and the separable system tensor
 * (Eq. separable_transf).  Copies the factors to the device, forms each
 * mode's Gram factor G_k = A_k^T A_k in FP64 on the device (7-banded for ELL4
 * factors, dense otherwise; the mixed-product property makes
 * A^T A = G_1 kron .. kron G_d) and the regulariser bands, picks the mode
 * order of apply / apply_T by cost (Sec. 2.1: reorder commuting products to
 * minimise work and intermediate storage) and allocates the workspace.
 * order: 3 or 4.  Returns TCA_ERR_SHAPE if factor k's n differs from n[k].
 * The stream orders the set-up copies and kernels; tca_plan synchronises it. */
TCA_API tca_status tca_plan(tca_plan_t* out, int order, const int64_t* n, const tca_factor* factors,
                    const tca_reg* reg, tca_precision prec, cudaStream_t stream);

/* Build a plan for scattered (off-grid) samples: the same unknown grid
 * (sizes n[0..order-1]) and regulariser, but a system tensor whose rows are
 * Kronecker products of per-sample, per-mode rows - sample s weights unknown
 * (i_1..i_d) by prod_k A_k[s][i_k] (the row-wise or face-splitting product of
 * the A_k; a tensor multiplication with a repeated index, Sec. 2.2, and the
 * structure of the paper's 4D reconstruction from scattered measurements,
 * Sec. 5).  rows[k]: an ELL4 factor with m rows (one per sample, the same
 * sample order in every mode) and n[k] columns, in host memory (copied).
 * The data tensor is a vector of m samples in that order.  A^T A is a sum of
 * rank-1 tensor products, not separable: tca_apply gathers each sample's
 * 4^d window, tca_apply_T scatters it back (atomic additions, so the last
 * bits of a sum may vary between runs), tca_apply_normal and the CG
 * iterations of tca_solve go through sample space, and the regulariser is
 * the separable one of tca_plan.  The samples are grouped on the device by
 * the grid tile that holds their window (the caller's order is kept at the
 * boundary).  prec: TCA_F64 (FP64 data and arithmetic) or TCA_F32 (FP32
 * data and arithmetic; tca_solve forms A^T b and checks the true residual
 * with the FP64 operator, so its stopping test is FP64-accurate as for
 * separable FP32 plans; the plan holds the weights in both precisions);
 * TCA_ERR_UNSUPPORTED otherwise.  No preconditioner, no tca_apply_mode, no
 * batched solve.  Returns TCA_ERR_SHAPE if a factor's m or n does not match. */
TCA_API tca_status tca_plan_scattered(tca_plan_t* out, int order, const int64_t* n, int64_t m,
                                      const tca_factor* rows, const tca_reg* reg, tca_precision prec,
                                      cudaStream_t stream);

/* y = A x = X x_1 A_1 ... x_d A_d (Sec. 2.1, Eq. separable_transf).
 * x: n-shaped, y: m-shaped, both C-order, element type of the plan. */
TCA_API tca_status tca_apply(tca_plan_t plan, const void* x, void* y, cudaStream_t stream);

/* x = A^T y = Y x_1 A_1^T ... x_d A_d^T (App. "Tensor transposition").
 * y: m-shaped, x: n-shaped. */
TCA_API tca_status tca_apply_T(tca_plan_t plan, const void* y, void* x, cudaStream_t stream);

/* y = (A^T A + lambda R) x, the normal operator of the regularised
 * least-squares problem (App. Eqs. A15-A17), evaluated matrix-free as
 * (G_1 kron .. kron G_d) x + lambda R x - the "iterative application of the
 * tensor multiplication" each CG step performs (Sec. 4.1, Fig. 2, Q = A.P).
 * x and y: n-shaped, must not alias. */
TCA_API tca_status tca_apply_normal(tca_plan_t plan, const void* x, void* y, cudaStream_t stream);

/* One mode product of the plan's operator on mode k (0-based) - a single
 * one-dimensional transformation of Eq. separable_transf:
 *   op TCA_OP_FACTOR:   y = x x_k A_k     (x has n_k on mode k, y has m_k)
 *   op TCA_OP_FACTOR_T: y = x x_k A_k^T   (x has m_k on mode k, y has n_k)
 *   op TCA_OP_GRAM:     y = x x_k G_k     (n_k -> n_k)
 * dims[0..order-1] is the shape of x (other modes may hold either n or m
 * sizes).  x and y must not alias. */
typedef enum { TCA_OP_FACTOR = 0, TCA_OP_FACTOR_T = 1, TCA_OP_GRAM = 2 } tca_mode_op;
TCA_API tca_status tca_apply_mode(tca_plan_t plan, int mode, int op, const int64_t* dims, const void* x,
                          void* y, cudaStream_t stream);

typedef struct {
  double rtol;          /* stop at ||A^T b - K x|| / ||A^T b|| <= rtol (true residual) */
  int32_t max_iter;     /* cap on CG iterations, all restarts and refinements counted */
  int32_t x0_given;     /* 1: x holds the initial guess; 0: start from x = 0 */
  double inner_rtol;    /* _IR plans: relative tolerance of each inner solve (0: default 1e-3) */
  int32_t max_refine;   /* _IR plans: cap on refinement steps (0: default 30) */
  int32_t check_every;  /* CG iterations per pass of the device loop; the stop flags are tested between passes (0: default 8, 16 for tca_solve_batched; rounded up to a multiple of 4) */
  int32_t profile;      /* 1: time every normal-operator sweep with CUDA events (info->sweep_*) */
  int32_t precond;      /* TCA_PRECOND_NONE: the CG of Fig. 2; TCA_PRECOND_SEPARABLE: the same CG with
                           Z = M^-1 R, M = (G_1 + s lambda L_1) x ... x (G_d + s lambda L_d);
                           TCA_PRECOND_JACOBI: M = diag(K); TCA_PRECOND_SEPARABLE_BANDED: the
                           separable inverse cut to 7-band factors; TCA_PRECOND_TMG: a two-grid
                           tensor multigrid cycle (see below) */
  double precond_shift; /* s, the regulariser weight folded into each mode of M (0: the plan's
                           tca_precond_default_shift).  The best s depends on lambda and the
                           factors (32 for the B-spline workload at lambda = 1e-3, 128 at 1e-4,
                           8 at 1e-2). */
  /* TCA_PRECOND_TMG (the tensor multigrid cycle below); zero selects each default. */
  double tmg_coarse_rtol;   /* relative tolerance ||r_c|| / ||b_c|| of the coarse CG (0: 0.3) */
  double tmg_lambda_max;    /* largest eigenvalue of D^-1 K, D = diag(K), for the Chebyshev
                               smoother (0: estimated on the device by 60 power steps from a
                               fixed pseudo-random start, once per plan) */
  int32_t tmg_nu;           /* Chebyshev smoothing steps before and after the coarse correction
                               (0: 3; a negative value: none, the bare coarse-grid correction) */
  int32_t tmg_coarsen_mask; /* bit k set: mode k is coarsened by 2 (0: every mode with n_k >= 16) */
} tca_solve_opts;

/* Preconditioner choice (tca_solve_opts.precond).  TCA_PRECOND_SEPARABLE_BANDED
 * is the separable preconditioner below with each per-mode inverse
 * (G_k + s lambda L_k)^-1 cut to its 7 central diagonals (|i - j| <= 3; the
 * inverses of these banded SPD matrices decay away from the diagonal, and the
 * cut matrices are checked positive definite, TCA_ERR_UNSUPPORTED otherwise):
 * M^-1 = B_1 kron .. kron B_d then has the structure of the fused
 * normal-operator sweep with zero regulariser bands, so z costs one sweep
 * (8 B per unknown) instead of d dense mode products; plans without the fused
 * sweep apply it as band mode products.  TCA_PRECOND_JACOBI is point
 * Jacobi, M = diag(K), the diagonally scaled CG of the paper's Fig. 1 solver
 * family: diag(K) = prod_k diag(G_k) + lambda sum_k diag(L_k) is formed once
 * per plan from the per-mode diagonals (FP64, stored as 1 / diag(K) in the
 * plan's element type, one n-shaped vector) and applied with <R, Z> in one
 * pass per iteration.  TCA_PRECOND_SEPARABLE uses
 * a tensor inverse (Sec. 3, Eq. TensorEq): M is a separable approximation of
 * K = (x)_k G_k + lambda sum_k L_k that keeps the Gram part exactly (G_k =
 * A_k^T A_k) and spreads the regulariser over the modes with weight s, and its
 * inverse is the separable transformation of the per-mode inverses
 * (G_k + s lambda L_k)^-1, formed once per plan and shift in FP64 on the host
 * (Cholesky) and applied as dense mode products (tensor cores for FP32
 * plans: 3xTF32 where the operand tiles fit in shared memory, plain TF32
 * otherwise; native FP64 for FP64 plans).  CG then uses rho = <R, Z> and
 * P = Z + beta P; the stop test stays on ||R|| / ||A^T b|| and on the FP64
 * true residual, so the result meets the same tolerance.  The paper fixes no
 * preconditioner; this one is an addition.  Costs d dense mode products and
 * one inner product per iteration, and one n_k x n_k dense factor per mode;
 * the tensor-core products of an iteration that starts after the stop flags
 * are set return at entry, like the CG kernels. */
enum { TCA_PRECOND_NONE = 0, TCA_PRECOND_SEPARABLE = 1, TCA_PRECOND_JACOBI = 2, TCA_PRECOND_SEPARABLE_BANDED = 3,
       TCA_PRECOND_TMG = 4 };

/* TCA_PRECOND_TMG: one two-grid tensor multigrid cycle (Sec. 4.2, Fig. 3) per
 * iteration, z = V r, on TCA_F32 and TCA_F64 plans with Gram-form (not
 * scattered) operators.  The transfers are separable: a coarsened mode k keeps
 * its even points, ceil(n_k / 2) of them, and P_k is linear interpolation back
 * to n_k points (Table 1's up-sampling; restriction = P_k^T); the coarse
 * operator is the Galerkin K_c = P^T K P with P = P_1 kron .. kron P_d (the
 * identity on modes that are kept), applied without being formed: prolong,
 * the fine K, restrict.  The cycle:
 *   z = S(0);  z += P K_c^-1 P^T (r - K z);  z = S(z)
 * where S is nu steps of Chebyshev iteration for K z = r preconditioned by
 * D = diag(K) over the interval [lambda_max / 30, 1.05 lambda_max] of D^-1 K,
 * the same polynomial before and after (so V is symmetric), and K_c^-1 is CG
 * to tmg_coarse_rtol (the direct solve at the coarsest scale of Fig. 3,
 * reached here by iteration; a loose tolerance makes V vary slightly from one
 * call to the next).  The CG iteration around it is the preconditioned CG of
 * TCA_PRECOND_SEPARABLE; the cycle's coarse solve is steered from the host
 * (one synchronisation per coarse iteration), so these solves run without the
 * device-side loop.  Not for tca_solve_batched (TCA_ERR_UNSUPPORTED). */

typedef struct {
  int32_t iters;             /* CG iterations run (all inner solves summed) */
  int32_t refinements;       /* outer refinement steps / true-residual restarts */
  double rel_res_true;       /* FP64 ||A^T b - K x|| / ||A^T b|| at exit */
  double rel_res_recursive;  /* sqrt(rho) / ||A^T b|| of the last CG step */
  double seconds;            /* wall time of the call (host clock) */
  double sweep_ms;           /* profile: device time summed over the CG normal-operator sweeps */
  int32_t sweep_launches;    /* profile: sweeps that did work (one per CG iteration) */
  int32_t reserved;
} tca_solve_info;

/* One-dimensional shear transform (Table 1: rotation as a product of 1D shear
 * transforms).  Every line along mode_a is resampled at positions moved in
 * proportion to the index along mode_b:
 *   y[.., i_a, .., i_b, ..] = sum_j h(i_a - slope (i_b - center) - j) x[.., j, .., i_b, ..]
 * with j over the line's dims[mode_a] points (nothing is read outside them;
 * points whose taps all fall outside come out 0) and h the interpolation kernel:
 * TCA_SHEAR_LINEAR the hat max(0, 1 - |u|) (2 taps), TCA_SHEAR_CUBIC cubic
 * convolution with a = -1/2 (4 taps; reproduces quadratics; the paper names no
 * interpolation).  Three shears with slopes tan(t/2) (mode a by mode b),
 * -sin(t) (b by a), tan(t/2) (a by b) about the plane's centre sample x at
 * c + R(t)(i - c), R(t) the rotation by t.  x, y: device buffers of dims
 * (C order, order 2 to 4), float for TCA_F32 and double for TCA_F64, not
 * aliased.  TCA_ERR_INVALID_ARG for null or host pointers, x == y, an order
 * or mode out of range, mode_a == mode_b, another kind or precision or a slope
 * or centre that is not finite; TCA_ERR_SHAPE for a non-positive size;
 * TCA_ERR_UNSUPPORTED for dims[mode_b] > 65535, dims[mode_a] >= 2^30 or more
 * than 2^40 elements.  Asynchronous on the stream. */
typedef enum { TCA_SHEAR_LINEAR = 1, TCA_SHEAR_CUBIC = 3 } tca_shear_kind;
TCA_API tca_status tca_apply_shear(int order, const int64_t* dims, int mode_a, int mode_b, double slope,
                                   double center, int kind, tca_precision prec, const void* x, void* y,
                                   cudaStream_t stream);

/* Discrete Fourier transform over the modes set in mode_mask (Table 1: F = E G H C
 * with one-dimensional DFT transforms) of the complex tensor re_in + i im_in,
 * as the separable transformation itself: along each selected mode k the data
 * are multiplied by F_k[j][i] = exp(-2 pi i j i / n_k) (inverse != 0:
 * exp(+2 pi i j i / n_k) / n_k, so that the inverse undoes the forward), four
 * real dense mode products per mode (O(n_k) work per output; this is the
 * definition, not an FFT).  re_in, im_in (NULL: a real input), re_out, im_out:
 * device buffers of dims (C order, order 1 to 4), float for TCA_F32 and double
 * for TCA_F64; no output may alias an input or the other output.  Builds two
 * plans of dense factors per call and about three n-shaped scratch tensors, and
 * synchronises the stream.  TCA_ERR_INVALID_ARG for null or host pointers,
 * aliasing, an empty mask or one naming a mode past order, another precision;
 * TCA_ERR_SHAPE for a non-positive size; TCA_ERR_UNSUPPORTED for a transformed
 * mode longer than 256, another mode longer than 2^24 or more than 2^40
 * elements, and where the dense mode product takes no such shape. */
TCA_API tca_status tca_apply_dft(int order, const int64_t* dims, uint32_t mode_mask, int inverse,
                                 tca_precision prec, const void* re_in, const void* im_in, void* re_out,
                                 void* im_out, cudaStream_t stream);

/* Solve (A^T A + lambda R) x = A^T b by the tensor CG of Sec. 4.1, Fig. 2:
 * R = B - A.C, P = R, rho = <R,R>; repeat Q = A.P, alpha = rho/<P,Q>,
 * C += alpha P, R -= alpha Q, rho1 = <R,R>, P = R + (rho1/rho) P.  The
 * iteration stops when the recursive residual reaches rtol; the FP64 true
 * residual is then recomputed and, if it is still above rtol, CG restarts
 * from the current x.  b: m-shaped data, x: n-shaped solution (in: initial
 * guess when opts->x0_given).  Scalars alpha, beta and all inner products are
 * kept in FP64 on the device; one graph launch runs passes of check_every
 * iterations until the device's stop flags are set (no host round trip in
 * between; iterations of the last pass after the stop return at entry).  The update C += alpha P is applied once per four
 * iterations from the four directions kept meanwhile (the same terms in the
 * same order and rounding as one update per iteration; a group cut short by
 * the stop test is completed before the true residual is formed), so x is
 * read and written a quarter as often.  Returns TCA_ERR_NOT_CONVERGED (x and info still
 * filled) when max_iter is reached, TCA_ERR_BREAKDOWN when <P, Q> <= 0 (or,
 * preconditioned, <R, Z> <= 0) or a scalar is not finite - a NaN or Inf in b
 * or in the initial guess ends that way; x then holds the last iterate and
 * info->rel_res_true its true residual.  A singular K (lambda = 0 and a
 * factor of rank below n_k) still gives a consistent system, since A^T b
 * lies in K's range: FP64 plans converge to a least-squares solution, while
 * FP32 roundings can feed K's null space into the directions until
 * <P, Q> <= 0, which is reported as TCA_ERR_BREAKDOWN.  opts->precond
 * selects the optional preconditioner (TCA_PRECOND_* above).  info may be NULL.  Synchronises the stream. */
TCA_API tca_status tca_solve(tca_plan_t plan, const void* b, void* x, const tca_solve_opts* opts,
                     tca_solve_info* info, cudaStream_t stream);

/* The shift s that the separable preconditioners take when
 * tca_solve_opts.precond_shift is 0, from a model of the spectrum of M^-1 K
 * (the paper fixes no preconditioner; this is a heuristic of this library):
 * each mode k either at its smooth corner (G_k at its largest eigenvalue, the
 * regulariser at zero) or at its rough corner (G_k at its smallest eigenvalue,
 * lambda L_k at its largest); at a corner K is taken as prod g + sum l and M as
 * prod (g + s l), and s, on the grid 2^(j/2) for j = 0 .. 16 (1 to 256),
 * minimises max / min of K / M over the 2^d corners.  The eigenvalues come from
 * host copies of the plan's FP64 bands (Jacobi rotations); formed on the first
 * call and kept with the plan.  Modes longer than 512 are not modelled: 16.
 * Synchronises the device (copies of the bands).  TCA_ERR_UNSUPPORTED for
 * scattered-sample plans. */
TCA_API tca_status tca_precond_default_shift(tca_plan_t plan, double* shift);

/* One tensor multigrid cycle z = V r (TCA_PRECOND_TMG above) with the options'
 * tmg_* fields: r and z n-shaped device buffers of the plan's element type
 * (TCA_F32: float, TCA_F64: double), not aliased.  Builds on first use, and
 * keeps with the plan, the transfers, the cycle's vectors (three n-shaped and
 * four coarse) and 1 / diag(K).  TCA_ERR_INVALID_ARG for a null pointer, a
 * negative tolerance or lambda_max, or a mask bit for a mode the plan lacks
 * or one with n_k < 2; TCA_ERR_UNSUPPORTED for scattered-sample plans and the
 * _IR precisions.  Synchronises the stream. */
TCA_API tca_status tca_tmg_apply(tca_plan_t plan, const void* r, void* z, const tca_solve_opts* opts,
                                 cudaStream_t stream);

/* The tensor multigrid state of the plan (Sec. 4.2, Fig. 3; no counterpart in
 * the paper, which reports no cycle statistics): the lambda_max of D^-1 K its
 * smoother uses (given or estimated; 0 before the first cycle) and the coarse
 * CG iterations run since the last tca_solve started (or since the last
 * tca_tmg_apply call).  Either pointer may be NULL. */
TCA_API tca_status tca_tmg_info(tca_plan_t plan, double* lambda_max, int64_t* coarse_iters);

/* Solve `count` independent systems (A_i^T A_i + lambda_i R_i) x_i = A_i^T b_i,
 * each by the CG of Sec. 4.1, Fig. 2, in one CUDA graph launch.  Many small
 * problems of uneven shapes are the workload; the paper's method is applied
 * unchanged to each of them.  plans[i]: a distinct TCA_F32 plan per instance
 * (any order, shape and factor kinds; a plan may not appear twice).  b[i]:
 * m_i-shaped, x[i]: n_i-shaped, both device memory, x[i] 16-byte aligned;
 * host or unaligned buffers give TCA_ERR_UNSUPPORTED.  opts applies to every
 * instance (rtol, max_iter, x0_given, check_every = CG iterations per pass
 * of an instance's inner loop; profile is ignored).
 * The first call for a given set of plans, buffers and options captures one
 * graph in which every instance is an independent branch, its kernels sized
 * for a quarter of the GPU's SMs so that several instances run side by side
 * (fused-sweep chunks from the wave model at that size; tca_autotune's choice
 * applies to single solves): set-up (A^T b in double-float, scalars,
 * first residual), then a while-conditional loop of restarts whose body runs
 * a nested while-conditional loop of check_every CG iterations until the
 * recursive residual meets rtol, recomputes the true residual in
 * double-float and, while it misses rtol and iterations remain, restarts CG
 * from x.  An instance that finishes leaves its loops while the others keep
 * iterating.  Later calls with the same signature replay the graph: one
 * graph launch per call, no host round trip until every instance is done
 * (info[i].refinements counts the restarts, at most 16).  info: `count`
 * entries or NULL; seconds is the wall time of the whole batch.  Returns the
 * first non-OK instance status (TCA_ERR_NOT_CONVERGED / TCA_ERR_BREAKDOWN);
 * every x[i] and info[i] is still written.  The graph is cached per
 * process for one batch at a time.  Synchronises the stream. */
TCA_API tca_status tca_solve_batched(int count, tca_plan_t* plans, const void* const* b, void* const* x,
                                     const tca_solve_opts* opts, tca_solve_info* info, cudaStream_t stream);

/* Autotune a batch for tca_solve_batched: solve it (opts as tca_solve_batched
 * takes them) once per candidate SM share - every instance's kernels sized
 * for 1/1, 1/2, 1/3, 1/4, 1/6 or 1/8 of the GPU's SMs, which sets each
 * instance's tile counts (fused-sweep chunks, vector-kernel grids, persistent
 * tensor-core and TMA-row CTAs) - time each graph launch on the device and
 * keep the fastest share for this batch signature (the same plans, buffers
 * and options), which later tca_solve_batched calls use; batches without a
 * tuned share use a quarter.  Solves the batch 2 x 6 times (x is
 * overwritten).  share_out (may be NULL) receives the share's denominator.
 * The paper applies its method to one system at a time; this is the
 * one-launch batch's tile choice made by measurement.  Synchronises the
 * stream. */
TCA_API tca_status tca_autotune_batched(int count, tca_plan_t* plans, const void* const* b, void* const* x,
                                        const tca_solve_opts* opts, int* share_out, cudaStream_t stream);

/* Autotune the normal-operator sweep that the plan's CG iterations run (its
 * CG form: new direction, K p and <p, K p>): time it for a few tile extents
 * along mode 1 around the cost model's choice and, for TCA_BF16_IR plans,
 * for both worker layouts of the tensor-core sweep (4 or 8 core rows per
 * thread), and keep the fastest in the plan (the plan-time expression
 * analysis of Sec. 2.1 and Sec. 4, which picks evaluation orders and kernels
 * by cost, extended with a measurement on this GPU).  Results are cached per
 * precision and shape (n_1..n_4) for the life of the process, so a second plan
 * of the same kind tunes in no time.  Plans without a fused sweep (TCA_F64,
 * dense factors, order 4 with n_4 other than 4 or 8 outside TCA_BF16_IR)
 * return TCA_OK unchanged.  Overwrites the plan's solver vectors and scalars
 * (every solve sets them up again); call it before a solve, not concurrently
 * with one on this plan.  Synchronises the stream. */
TCA_API tca_status tca_autotune(tca_plan_t plan, cudaStream_t stream);

/* Tile extent the autotuner chose for the plan (chunks of mode 1), or 0 when
 * the plan uses the cost model. */
TCA_API int tca_autotuned_chunks(tca_plan_t plan);

/* Worker layout the autotuner chose for a TCA_BF16_IR plan's tensor-core sweep
 * (core rows per thread: 4 or 8), or 0 when it has not tuned the plan. */
TCA_API int tca_autotuned_rows(tca_plan_t plan);

/* Relative residual ||rhs - kx||_2 / ||rhs||_2 of two FP64 device vectors of
 * length n, written to *out (device memory, one double).  If ||rhs|| is zero
 * the absolute norm ||rhs - kx|| is written instead (0 for n = 0).
 *
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory when they check a solution - code with a fixed
 * memory budget after start-up, device memory owned by another allocator, or
 * a hook that runs while the caller's allocator is locked.  It allocates
 * nothing: its reduction scratch is a fixed 256 KiB device array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  The first call on a device looks up that array's address (set-up),
 * so make that first call before any stream capture; after a cudaDeviceReset
 * the next call on that device repeats the set-up.  n may not exceed
 * 134,217,728 (TCA_ERR_UNSUPPORTED, message in tca_last_error_string()).
 * Every call shares the scratch, which keeps the last call's contents; calls
 * that overlap on the GPU (unordered streams) race and give undefined
 * results.  Asynchronous on the stream. */
TCA_API tca_status tca_rel_residual_noalloc(const double* rhs, const double* kx, int64_t n, double* out,
                                            cudaStream_t stream);

/* Vector steps of Fig. 2's iteration (Sec. 4.1) on caller-owned float device
 * vectors of length n, for callers that drive CG themselves - the
 * slab-partitioned solve, where each rank owns a contiguous run of mode-1
 * planes, applies K to its slab with its own plan (factor 1 restricted to the
 * slab's columns) and combines inner products across ranks.
 *   tca_vec_axpby: y = a x + b y (C += alpha P, R -= alpha Q, P = R + beta P);
 *   tca_vec_dot:   *out = sum_i a[i] b[i], FP32 products summed in FP64; out is
 *                  one device double, zeroed and then accumulated on the stream
 *                  (block sums combined by FP64 atomics: the last bits of the
 *                  sum may vary from run to run).
 * Asynchronous on the stream; host pointers give TCA_ERR_UNSUPPORTED. */
TCA_API tca_status tca_vec_axpby(float* y, const float* x, double a, double b, int64_t n, cudaStream_t stream);
TCA_API tca_status tca_vec_dot(const float* a, const float* b, int64_t n, double* out, cudaStream_t stream);

/* Synchronise the stream, then report whether any bounded device wait (TMA
 * and tensor-core pipelines) gave up since the last check: TCA_ERR_TIMEOUT,
 * clearing the flag, or TCA_OK.  The flag is per process, not per plan. */
TCA_API tca_status tca_check_timeout(cudaStream_t stream);

/* Diagnostic of the wait machinery: one block waits on an mbarrier that
 * nothing arrives at, at most `polls` polls (>= 0), then gives up exactly as
 * a real wait would.  Returns the tca_check_timeout verdict: TCA_ERR_TIMEOUT
 * for any polls count (the wait cannot succeed), TCA_ERR_INVALID_ARG for
 * polls < 0.  The context stays usable.  Synchronises the stream. */
TCA_API tca_status tca_wait_selftest(int64_t polls, cudaStream_t stream);

/* Free a plan and its device memory (NULL is ignored).  Synchronises the
 * device first, so no work of the plan may still be queued on another stream
 * that the caller keeps using. */
TCA_API void tca_destroy(tca_plan_t plan);

/* Static text for a status code. */
TCA_API const char* tca_status_string(tca_status status);

/* Text of the last CUDA error seen by this thread ("" if none). */
TCA_API const char* tca_last_error_string(void);

/* Number of the library's own kernels launched by this thread since the last
 * reset (counts every launch, including those replayed from CUDA graphs). */
TCA_API uint64_t tca_kernel_launches(int reset);

/* ABI version, (major << 16) | minor. */
TCA_API int tca_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TCA_H */
