// Tensor conjugate gradients (Sec. 4.1, Fig. 2) on the normal equations
// (A^T A + lambda R) x = A^T b, with every scalar kept on the device in FP64:
//   R = B - K C;  P = R;  rho = <R,R>
//   repeat  Q = K P;  alpha = rho/<P,Q>;  C += alpha P;  R -= alpha Q;
//           rho1 = <R,R>;  P = R + (rho1/rho) P;  rho = rho1
// The direction update P = R + beta P is folded into the next normal-operator
// sweep; alpha and beta are formed by the last block of the reductions that
// produce <P,Q> and <R,R>, so an iteration never waits on the host.  The host
// replays a CUDA graph of `check_every` iterations and reads one flag word
// between replays.  When the recursive residual meets the tolerance the true
// residual ||A^T b - K x|| / ||A^T b|| is recomputed in FP64; CG restarts from
// the current x while it is above the tolerance.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "tca_internal.cuh"

namespace tca {

namespace {

constexpr int kVecThreads = 256;

template <typename T> struct V2;
template <> struct V2<float> { using t = float4; static constexpr int n = 4; };
template <> struct V2<double> { using t = double2; static constexpr int n = 2; };

// r -= alpha q;  rho1 = <r, r>  (Fig. 2 update block) -> beta, stop test, and
// the solution update x += alpha p grouped over kDirBufs iterations: the
// iterations at group positions 0 .. kDirBufs - 2 only record alpha (their
// directions stay in their own buffers); the last position applies
//   x += alpha_0 p_0;  x += alpha_1 p_1;  ...;  x += alpha p
// in iteration order, one rounding per term, the same values as one update
// per iteration, for a quarter of the x traffic.
template <typename T>
struct DirBufs {
  const T* p[kDirBufs];  // direction written at group position i: p[(i + 1) % kDirBufs]
};

template <typename T>
__device__ __forceinline__ T group_x_update(T x, const T* __restrict__ const* pb, const double* ah, T alpha, T pnew,
                                            int64_t i, int npend) {
  for (int k = 0; k < npend; ++k) x = fma((T)ah[k], pb[k + 1][i], x);
  return fma(alpha, pnew, x);
}

template <typename T, bool XUPD, bool PC>
__global__ void __launch_bounds__(kVecThreads) cg_update_kernel(T* __restrict__ x, T* __restrict__ r,
                                                                const T* __restrict__ p, const T* __restrict__ q,
                                                                int64_t n, Scalars* sc, Reduce red, DirBufs<T> pb,
                                                                int pos) {
  __shared__ double sh[kVecThreads / 32];
  if (cg_done(sc)) return;
  const double alpha_d = sc->alpha;
  const T alpha = (T)alpha_d;
  using VT = typename V2<T>::t;
  constexpr int VN = V2<T>::n;
  const int64_t nv = n / VN;
  T ah[kDirBufs - 1];
  if constexpr (XUPD) {
#pragma unroll
    for (int k = 0; k < kDirBufs - 1; ++k) ah[k] = (T)sc->alpha_hist[k];
  }
  T part = T(0);
  double acc = 0.0;
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    VT rv = reinterpret_cast<VT*>(r)[i];
    const VT qv = reinterpret_cast<const VT*>(q)[i];
    if constexpr (XUPD) {
      VT xv = reinterpret_cast<VT*>(x)[i];
      T* xs = reinterpret_cast<T*>(&xv);
#pragma unroll
      for (int k = 0; k < kDirBufs - 1; ++k) {
        const VT pv = reinterpret_cast<const VT*>(pb.p[k + 1])[i];
        const T* ps = reinterpret_cast<const T*>(&pv);
#pragma unroll
        for (int c = 0; c < VN; ++c) xs[c] = fma(ah[k], ps[c], xs[c]);
      }
      const VT pv = reinterpret_cast<const VT*>(p)[i];
      const T* ps = reinterpret_cast<const T*>(&pv);
#pragma unroll
      for (int c = 0; c < VN; ++c) xs[c] = fma(alpha, ps[c], xs[c]);
      reinterpret_cast<VT*>(x)[i] = xv;
    }
    if constexpr (VN == 4) {
      rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
      part += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
    } else {
      rv.x -= alpha * qv.x; rv.y -= alpha * qv.y;
      part += rv.x * rv.x + rv.y * rv.y;
    }
    reinterpret_cast<VT*>(r)[i] = rv;
    if (++cnt == 8) {  // short FP32 runs, FP64 beyond
      acc += (double)part;
      part = T(0);
      cnt = 0;
    }
  }
  if (blockIdx.x == 0) {
    for (int64_t i = nv * VN + threadIdx.x; i < n; i += blockDim.x) {
      if constexpr (XUPD) x[i] = group_x_update<T>(x[i], pb.p, sc->alpha_hist, alpha, p[i], i, kDirBufs - 1);
      r[i] -= alpha * q[i];
      part += r[i] * r[i];
    }
  }
  acc += (double)part;
  double total;
  if (dev::grid_sum_last(acc, red, &total, sh)) {
    // <r, r> always feeds the stop test; without a preconditioner it is also
    // rho of the next step (with one, rho = <r, z> comes after z = M^-1 r).
    const double rho = sc->rho;
    sc->rho_new = total;
    if constexpr (!PC) {
      sc->beta = total / rho;
      sc->rho = total;
    }
    sc->iters += 1;
    if constexpr (XUPD) {
      sc->npend = 0;
    } else {
      sc->alpha_hist[pos] = alpha_d;
      sc->npend = pos + 1;
    }
    if (!isfinite(total)) sc->breakdown = 1;
    if (sqrt(total) <= sc->rtol * sc->bnorm) sc->converged = 1;
  }
}

// The part of a group's solution update still pending when the iteration loop
// stops (converged, broken down or out of iterations part-way through a group):
// x += alpha_k p_k for the npend recorded positions, then npend = 0.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) cg_flush_x_kernel(T* __restrict__ x, int64_t n, Scalars* sc,
                                                                 Reduce red, DirBufs<T> pb) {
  __shared__ double sh[kVecThreads / 32];
  const int np = sc->npend;
  if (np > 0) {
    // 16-byte vectors (allocation-aligned buffers), the scalar tail by block 0;
    // per element the pending terms in iteration order, as the update applies them.
    T ah[kDirBufs - 1];
#pragma unroll
    for (int k = 0; k < kDirBufs - 1; ++k) ah[k] = k < np ? (T)sc->alpha_hist[k] : T(0);
    using VT = typename V2<T>::t;
    constexpr int VN = V2<T>::n;
    const int64_t nv = n / VN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
      VT xv = reinterpret_cast<VT*>(x)[i];
      T* xs = reinterpret_cast<T*>(&xv);
#pragma unroll
      for (int k = 0; k < kDirBufs - 1; ++k) {
        if (k >= np) break;
        const VT pv = reinterpret_cast<const VT*>(pb.p[k + 1])[i];
        const T* ps = reinterpret_cast<const T*>(&pv);
#pragma unroll
        for (int c = 0; c < VN; ++c) xs[c] = fma(ah[k], ps[c], xs[c]);
      }
      reinterpret_cast<VT*>(x)[i] = xv;
    }
    if (blockIdx.x == 0) {
      for (int64_t i = nv * VN + threadIdx.x; i < n; i += blockDim.x) {
        T xv = x[i];
        for (int k = 0; k < np; ++k) xv = fma(ah[k], pb.p[k + 1][i], xv);
        x[i] = xv;
      }
    }
  }
  double total;
  if (dev::grid_sum_last(0.0, red, &total, sh)) sc->npend = 0;
}

// P_new = R + beta P_old (used when the normal operator is not the fused sweep).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) cg_direction_kernel(const T* __restrict__ r, const T* __restrict__ pold,
                                                                   T* __restrict__ pnew, int64_t n, const Scalars* sc) {
  if (cg_done(sc)) return;
  const T beta = (T)sc->beta;
  using VT = typename V2<T>::t;
  constexpr int VN = V2<T>::n;
  const int64_t nv = n / VN;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const VT rv = reinterpret_cast<const VT*>(r)[i];
    const VT pv = reinterpret_cast<const VT*>(pold)[i];
    VT o;
    const T* rs = reinterpret_cast<const T*>(&rv);
    const T* ps = reinterpret_cast<const T*>(&pv);
    T* os = reinterpret_cast<T*>(&o);
#pragma unroll
    for (int c = 0; c < VN; ++c) os[c] = rs[c] + beta * ps[c];
    reinterpret_cast<VT*>(pnew)[i] = o;
  }
  if (blockIdx.x == 0)
    for (int64_t i = nv * VN + threadIdx.x; i < n; i += blockDim.x) pnew[i] = r[i] + beta * pold[i];
}

// r = rhs - kx (kx may be null: r = rhs); rho = <r,r>; optionally bnorm = ||rhs||.
// Resets beta = 0 (fresh direction) and the stop flags.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) cg_start_kernel(const T* __restrict__ rhs, const T* __restrict__ kx,
                                                               T* __restrict__ r, int64_t n, Scalars* sc, Reduce red,
                                                               int set_bnorm, Reduce red2) {
  __shared__ double sh[kVecThreads / 32];
  double a_rr = 0.0, a_bb = 0.0;
  T p_rr = T(0), p_bb = T(0);  // short runs in T, FP64 beyond (the FP64 pipe is the slow one)
  int cnt = 0;
  // 16-byte vectors (the buffers are allocation-aligned), the scalar tail by block 0.
  using VT = typename V2<T>::t;
  constexpr int VN = V2<T>::n;
  const int64_t nv = n / VN;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const VT bv = reinterpret_cast<const VT*>(rhs)[i];
    VT vv = bv;
    if (kx) {
      const VT kv = reinterpret_cast<const VT*>(kx)[i];
      T* vs = reinterpret_cast<T*>(&vv);
      const T* ks = reinterpret_cast<const T*>(&kv);
#pragma unroll
      for (int c = 0; c < VN; ++c) vs[c] = (T)(vs[c] - ks[c]);
    }
    reinterpret_cast<VT*>(r)[i] = vv;
    const T* vs = reinterpret_cast<const T*>(&vv);
    const T* bs = reinterpret_cast<const T*>(&bv);
#pragma unroll
    for (int c = 0; c < VN; ++c) {
      p_rr += vs[c] * vs[c];
      p_bb += bs[c] * bs[c];
    }
    if (++cnt == 16 / VN) {
      a_rr += (double)p_rr;
      a_bb += (double)p_bb;
      p_rr = p_bb = T(0);
      cnt = 0;
    }
  }
  if (blockIdx.x == 0) {
    for (int64_t i = nv * VN + threadIdx.x; i < n; i += blockDim.x) {
      const T b = rhs[i];
      const T v = kx ? (T)(b - kx[i]) : b;
      r[i] = v;
      p_rr += v * v;
      p_bb += b * b;
    }
  }
  a_rr += (double)p_rr;
  a_bb += (double)p_bb;
  // Two independent reductions, each with its own scratch and ticket.
  double t_rr, t_bb;
  const bool last1 = dev::grid_sum_last(a_rr, red, &t_rr, sh);
  const bool last2 = dev::grid_sum_last(a_bb, red2, &t_bb, sh);
  if (last1) {
    sc->rho = t_rr;
    sc->rho_new = t_rr;
    sc->beta = 0.0;
    sc->converged = 0;
    sc->breakdown = 0;
  }
  if (last2 && set_bnorm) sc->bnorm = sqrt(t_bb);
}

// Preconditioned CG: rho1 = <r, z> (z = M^-1 r).  INIT (a fresh start or a
// restart): rho = rho1, beta = 0; otherwise beta = rho1 / rho, rho = rho1.
// A non-positive or non-finite <r, z> with r != 0 is a breakdown.
template <typename T, bool INIT>
__global__ void __launch_bounds__(kVecThreads) cg_precond_dot_kernel(const T* __restrict__ r, const T* __restrict__ z,
                                                                     int64_t n, Scalars* sc, Reduce red) {
  __shared__ double sh[kVecThreads / 32];
  if (cg_done(sc)) return;
  using VT = typename V2<T>::t;
  constexpr int VN = V2<T>::n;
  const int64_t nv = n / VN;
  T part = T(0);
  double acc = 0.0;
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const VT rv = reinterpret_cast<const VT*>(r)[i];
    const VT zv = reinterpret_cast<const VT*>(z)[i];
    const T* rs = reinterpret_cast<const T*>(&rv);
    const T* zs = reinterpret_cast<const T*>(&zv);
#pragma unroll
    for (int c = 0; c < VN; ++c) part += rs[c] * zs[c];
    if (++cnt == 8) {  // short runs in T, FP64 beyond
      acc += (double)part;
      part = T(0);
      cnt = 0;
    }
  }
  if (blockIdx.x == 0)
    for (int64_t i = nv * VN + threadIdx.x; i < n; i += blockDim.x) part += r[i] * z[i];
  acc += (double)part;
  double total;
  if (dev::grid_sum_last(acc, red, &total, sh)) {
    const bool bad = !isfinite(total) || (!(total > 0.0) && sc->rho_new > 0.0);
    if (bad) sc->breakdown = 1;
    if (INIT) {
      sc->beta = 0.0;
    } else {
      sc->beta = total / sc->rho;
    }
    sc->rho = total;
  }
}

// Point-Jacobi preconditioner in one pass: z = r / diag(K) (from the stored
// reciprocal), rho1 = <r, z>; the same scalar logic as cg_precond_dot_kernel.
template <typename T, bool INIT>
__global__ void __launch_bounds__(kVecThreads) cg_jacobi_kernel(const T* __restrict__ r, const T* __restrict__ dinv,
                                                                T* __restrict__ z, int64_t n, Scalars* sc, Reduce red) {
  __shared__ double sh[kVecThreads / 32];
  if (cg_done(sc)) return;
  using VT = typename V2<T>::t;
  constexpr int VN = V2<T>::n;
  const int64_t nv = n / VN;
  T part = T(0);
  double acc = 0.0;
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const VT rv = reinterpret_cast<const VT*>(r)[i];
    const VT dv = reinterpret_cast<const VT*>(dinv)[i];
    VT zv;
    const T* rs = reinterpret_cast<const T*>(&rv);
    const T* ds = reinterpret_cast<const T*>(&dv);
    T* zs = reinterpret_cast<T*>(&zv);
#pragma unroll
    for (int c = 0; c < VN; ++c) {
      zs[c] = rs[c] * ds[c];
      part += rs[c] * zs[c];
    }
    reinterpret_cast<VT*>(z)[i] = zv;
    if (++cnt == 8) {  // short runs in T, FP64 beyond
      acc += (double)part;
      part = T(0);
      cnt = 0;
    }
  }
  if (blockIdx.x == 0)
    for (int64_t i = nv * VN + threadIdx.x; i < n; i += blockDim.x) {
      z[i] = r[i] * dinv[i];
      part += r[i] * z[i];
    }
  acc += (double)part;
  double total;
  if (dev::grid_sum_last(acc, red, &total, sh)) {
    const bool bad = !isfinite(total) || (!(total > 0.0) && sc->rho_new > 0.0);
    if (bad) sc->breakdown = 1;
    sc->beta = INIT ? 0.0 : total / sc->rho;
    sc->rho = total;
  }
}

// ||rhs64 - kx64|| / ||rhs64||  -> sc->aux; optionally r = rhs64 - kx64 (cast).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) true_residual_kernel(const double* __restrict__ rhs,
                                                                    const double* __restrict__ kx, T* __restrict__ r,
                                                                    int64_t n, Scalars* sc, Reduce red, Reduce red2) {
  __shared__ double sh[kVecThreads / 32];
  double a_rr = 0.0, a_bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double b = rhs[i];
    const double v = b - kx[i];
    if (r) r[i] = (T)v;
    a_rr += v * v;
    a_bb += b * b;
  }
  double t_rr, t_bb;
  const bool l1 = dev::grid_sum_last(a_rr, red, &t_rr, sh);
  if (l1) red2.partials[red2.max_blocks - 1] = t_rr;  // park the first total past the used slots
  const bool l2 = dev::grid_sum_last(a_bb, red2, &t_bb, sh);
  if (l2) {
    __threadfence();
    sc->aux = sqrt(((volatile double*)red2.partials)[red2.max_blocks - 1]) / sqrt(t_bb);
  }
}

// b = (Tout) a, element by element (FP32 -> FP64 widening is exact).
template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* __restrict__ a, Tout* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (Tout)a[i];
}

// Every element of x set to the bit pattern v.
template <typename U>
__global__ void fill_bits_kernel(U* __restrict__ x, U v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

__global__ void cg_setup_kernel(Scalars* sc, double rtol, int max_iter) {
  sc->rtol = rtol;
  sc->max_iter = max_iter;
  sc->iters = 0;
  sc->converged = 0;
  sc->breakdown = 0;
  sc->beta = 0.0;
  sc->alpha = 0.0;
  sc->npend = 0;
}

}  // namespace

// Second reduction scratch lives after the first one's slots.
static Reduce second_reduce(const tca_plan_s* p) {
  Reduce r = p->red;
  r.partials = p->red.partials + p->red.max_blocks / 2;
  r.ticket = p->red.ticket + 1;
  r.max_blocks = p->red.max_blocks / 2;
  return r;
}
static Reduce first_reduce(const tca_plan_s* p) {
  Reduce r = p->red;
  r.max_blocks = p->red.max_blocks / 2;
  return r;
}

template <typename T>
static DirBufs<T> dir_bufs(const tca_plan_s* p) {
  DirBufs<T> d;
  for (int k = 0; k < kDirBufs; ++k) d.p[k] = (const T*)p->p[k];
  return d;
}

// Preconditioned CG: z = M^-1 r, then rho from <r, z> (init: a fresh start).
// Point Jacobi does both in one pass.
template <typename T>
static tca_status enqueue_precond(tca_plan_s* p, bool init, cudaStream_t s) {
  const int grid = std::min(vector_grid(p, p->N), first_reduce(p).max_blocks);
  if (p->pc_kind == TCA_PRECOND_JACOBI) {
    if (init)
      cg_jacobi_kernel<T, true><<<grid, kVecThreads, 0, s>>>((const T*)p->r, (const T*)p->pc_dinv, (T*)p->z, p->N,
                                                             p->scal, first_reduce(p));
    else
      cg_jacobi_kernel<T, false><<<grid, kVecThreads, 0, s>>>((const T*)p->r, (const T*)p->pc_dinv, (T*)p->z, p->N,
                                                              p->scal, first_reduce(p));
    TCA_LAUNCH_CHECK();
    return TCA_OK;
  }
  if (p->pc_kind == TCA_PRECOND_TMG) {
    // One tensor multigrid cycle (host-steered; nothing to do after the stop).
    TCA_TRY(tmg_cycle<T>(p, (const T*)p->r, (T*)p->z, true, s));
  } else {
    if constexpr (sizeof(T) == 4) {
      // The banded preconditioner's fused sweep forms <r, z> and the scalars itself.
      const tca_status fd = apply_precond_dot(p, (const float*)p->r, (float*)p->z, init, s);
      if (fd != TCA_ERR_UNSUPPORTED) return fd;
    }
    TCA_TRY(apply_precond<T>(p, (const T*)p->r, (T*)p->z, s));
  }
  if (init)
    cg_precond_dot_kernel<T, true><<<grid, kVecThreads, 0, s>>>((const T*)p->r, (const T*)p->z, p->N, p->scal,
                                                                 first_reduce(p));
  else
    cg_precond_dot_kernel<T, false><<<grid, kVecThreads, 0, s>>>((const T*)p->r, (const T*)p->z, p->N, p->scal,
                                                                  first_reduce(p));
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// The preconditioner a solve asks for: validates the options, builds the
// factors for the shift (by default the plan's corner-model shift) and marks
// the plan's iteration as preconditioned (or not).
static tca_status setup_precond(tca_plan_s* p, const tca_solve_opts* o, cudaStream_t s) {
  p->pc_on = false;
  p->pc_kind = TCA_PRECOND_NONE;
  const int kind = o ? o->precond : TCA_PRECOND_NONE;
  if (kind == TCA_PRECOND_NONE) return TCA_OK;
  if (p->scattered) {
    set_error_message("scattered-sample plans take no preconditioner");
    return TCA_ERR_UNSUPPORTED;
  }
  if (kind == TCA_PRECOND_JACOBI) {
    TCA_TRY(ensure_jacobi(p));
  } else if (kind == TCA_PRECOND_TMG) {
    TCA_TRY(tmg_setup(p, o, s));
    tmg_reset_count(p);
  } else {
    if ((kind != TCA_PRECOND_SEPARABLE && kind != TCA_PRECOND_SEPARABLE_BANDED) || o->precond_shift < 0.0)
      return TCA_ERR_INVALID_ARG;
    double shift = o->precond_shift;
    if (!(shift > 0.0)) TCA_TRY(precond_model_shift(p, &shift));
    if (kind == TCA_PRECOND_SEPARABLE) TCA_TRY(ensure_precond(p, shift));
    else TCA_TRY(ensure_precond_banded(p, shift));
  }
  p->pc_on = true;
  p->pc_kind = kind;
  return TCA_OK;
}

// One CG iteration at position `it` of a graph replay (replays hold a multiple
// of kDirBufs iterations, so it % kDirBufs is the position in the update
// group).  ev_begin/ev_end (may be null) bracket the normal-operator sweep so
// that a profiled solve can time it on the device.
// One iteration of a TCA_BF16_IR plan's inner CG: the bfloat16 tensor-core
// sweep (p = r + beta p_old, q = K p, alpha) and the bfloat16 update of r and of
// the FP32 correction d.
static tca_status enqueue_iteration_bf16(tca_plan_s* p, float* d, int it, cudaStream_t s, cudaEvent_t ev_begin,
                                         cudaEvent_t ev_end) {
  const int pos = it % kDirBufs;
  if (ev_begin) TCA_CUDA_TRY(cudaEventRecordWithFlags(ev_begin, s, cudaEventRecordExternal));
  TCA_TRY(bf16_sweep(p, pos, p->bf.p[(pos + 1) % kDirBufs], p->bf.q, s));
  if (ev_end) TCA_CUDA_TRY(cudaEventRecordWithFlags(ev_end, s, cudaEventRecordExternal));
  return bf16_update(p, d, pos, first_reduce(p), s);
}

template <typename T>
static tca_status enqueue_iteration(tca_plan_s* p, T* x, int it, cudaStream_t s, cudaEvent_t ev_begin,
                                    cudaEvent_t ev_end) {
  if constexpr (sizeof(T) == 4) {
    if (p->prec == TCA_BF16_IR) return enqueue_iteration_bf16(p, (float*)x, it, s, ev_begin, ev_end);
  }
  const int64_t N = p->N;
  const int pos = it % kDirBufs;
  const T* pold = (const T*)p->p[pos];
  T* pnew = (T*)p->p[(pos + 1) % kDirBufs];
  T* r = (T*)p->r;
  T* q = (T*)p->q;
  const int grid = std::min(vector_grid(p, N), first_reduce(p).max_blocks);
  const bool fused = sizeof(T) == 4 && p->fused_ok;
  // The new direction is formed from r (Fig. 2) or, preconditioned, from z = M^-1 r.
  const T* dsrc = p->pc_on ? (const T*)p->z : r;
  if (ev_begin) TCA_CUDA_TRY(cudaEventRecordWithFlags(ev_begin, s, cudaEventRecordExternal));
  if constexpr (sizeof(T) == 4) {
    if (fused) TCA_TRY(normal_fused_f32(p, dsrc, pold, pnew, q, true, s));
  }
  if (!fused) {
    cg_direction_kernel<T><<<grid, kVecThreads, 0, s>>>(dsrc, pold, pnew, N, p->scal);
    TCA_LAUNCH_CHECK();
    const RegDot dot{p->scal, first_reduce(p)};
    TCA_TRY(normal_generic<T>(p, pnew, q, s, &dot));
  }
  if (ev_end) TCA_CUDA_TRY(cudaEventRecordWithFlags(ev_end, s, cudaEventRecordExternal));
  const DirBufs<T> db = dir_bufs<T>(p);
  const Reduce red = first_reduce(p);
  if (pos == kDirBufs - 1) {
    if (p->pc_on) cg_update_kernel<T, true, true><<<grid, kVecThreads, 0, s>>>(x, r, pnew, q, N, p->scal, red, db, pos);
    else cg_update_kernel<T, true, false><<<grid, kVecThreads, 0, s>>>(x, r, pnew, q, N, p->scal, red, db, pos);
  } else {
    if (p->pc_on) cg_update_kernel<T, false, true><<<grid, kVecThreads, 0, s>>>(x, r, pnew, q, N, p->scal, red, db, pos);
    else cg_update_kernel<T, false, false><<<grid, kVecThreads, 0, s>>>(x, r, pnew, q, N, p->scal, red, db, pos);
  }
  TCA_LAUNCH_CHECK();
  if (p->pc_on) TCA_TRY(enqueue_precond<T>(p, false, s));
  return TCA_OK;
}

// Apply the part of the grouped solution update still pending after the
// iteration loop.
template <typename T>
static tca_status flush_pending_x(tca_plan_s* p, T* x, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (p->prec == TCA_BF16_IR) return bf16_flush(p, (float*)x, first_reduce(p), s);
  }
  const int grid = std::min(vector_grid(p, p->N), first_reduce(p).max_blocks);
  cg_flush_x_kernel<T><<<grid, kVecThreads, 0, s>>>(x, p->N, p->scal, first_reduce(p), dir_bufs<T>(p));
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template <typename T>
static tca_status ensure_solver_buffers(tca_plan_s* p) {
  if (p->r) return TCA_OK;
  const size_t bytes = sizeof(T) * (size_t)p->N;
  cudaError_t e = cudaMalloc(&p->rhs, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->r, bytes);
  for (int k = 0; k < kDirBufs && e == cudaSuccess; ++k) e = cudaMalloc(&p->p[k], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->q, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->res64, sizeof(double) * (size_t)p->N);
  if (e == cudaSuccess && sizeof(T) == 4) e = cudaMalloc((void**)&p->rhs64, sizeof(double) * (size_t)p->N);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  return TCA_OK;
}

// State in which a CG-mode sweep does its full work outside a solve (for the
// autotuner): solver buffers allocated, r and the directions zero, scalars of
// a fresh iteration that is not converged.  A later solve re-initialises all
// of it.
tca_status prepare_sweep_timing(tca_plan_s* p, cudaStream_t s) {
  if (p->prec == TCA_F64) return TCA_ERR_UNSUPPORTED;
  TCA_TRY(ensure_solver_buffers<float>(p));
  // r = 1 everywhere (so <p, K p> > 0 and the sweep never flags a breakdown), directions 0.
  const int grid = vector_grid(p, p->N);
  fill_bits_kernel<uint32_t><<<grid, kVecThreads, 0, s>>>((uint32_t*)p->r, 0x3f800000u, p->N);
  TCA_LAUNCH_CHECK();
  for (int k = 0; k < kDirBufs; ++k) TCA_CUDA_TRY(cudaMemsetAsync(p->p[k], 0, sizeof(float) * (size_t)p->N, s));
  if (p->prec == TCA_BF16_IR) {
    fill_bits_kernel<uint16_t><<<grid, kVecThreads, 0, s>>>((uint16_t*)p->bf.r, (uint16_t)0x3f80u, p->N);
    TCA_LAUNCH_CHECK();
    for (int k = 0; k < kDirBufs; ++k) TCA_CUDA_TRY(cudaMemsetAsync(p->bf.p[k], 0, 2 * (size_t)p->N, s));
  }
  cg_setup_kernel<<<1, 1, 0, s>>>(p->scal, 0.0, 1 << 30);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

namespace {

// Loop condition: one thread sets the handle from the instance's stop flags.
__global__ void cond_running_kernel(const Scalars* sc, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, cg_done(sc) ? 0u : 1u);
}

// Conditional handle owned by the graph that stream s is capturing into.
tca_status capture_handle(cudaStream_t s, unsigned default_value, bool assign_default, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  TCA_CUDA_TRY(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive || !g) {
    set_error_message("stream is not capturing");
    return TCA_ERR_CUDA;
  }
  TCA_CUDA_TRY(cudaGraphConditionalHandleCreate(h, g, default_value, assign_default ? cudaGraphCondAssignDefault : 0));
  return TCA_OK;
}

// Append a WHILE node on handle h to the capture sequence of s; returns its body graph.
tca_status capture_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  TCA_CUDA_TRY(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &edges, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  TCA_CUDA_TRY(cudaGraphAddNode(&node, g, deps, edges, nd, &cp));
  *body = cp.conditional.phGraph_out[0];
  TCA_CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return TCA_OK;
}

// Capture `fill(stream)` into the (empty) graph g.
template <typename F>
tca_status capture_into(cudaGraph_t g, cudaStream_t cs, F fill) {
  TCA_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const tca_status st = fill(cs);
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &out);
  if (st != TCA_OK) return st;
  TCA_CUDA_TRY(e);
  return TCA_OK;
}

}  // namespace

// Build (or reuse) the graph of `iters` iterations (a multiple of kDirBufs:
// the direction buffers rotate) for this x buffer.  Unprofiled graphs wrap
// the iterations in a device-side WHILE loop that runs passes until the stop
// flags are set, so one launch finishes the iteration; profiled graphs run
// one pass per launch (the host reads each pass's sweep events).
template <typename T>
static tca_status get_graph(tca_plan_s* p, T* x, int iters, bool profile, cudaStream_t s) {
  if (p->graph_exec && p->graph_x == x && p->graph_iters == iters && p->graph_profiled == profile &&
      p->graph_pc == (p->pc_on ? p->pc_kind : 0))
    return TCA_OK;
  if (p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  if (profile && !p->sweep_ev[0]) {
    for (int i = 0; i < 2 * kMaxProfiledIters; ++i) TCA_CUDA_TRY(cudaEventCreate(&p->sweep_ev[i]));
  }
  cudaStream_t cs;
  TCA_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const uint64_t before = tca_kernel_launches(0);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  tca_status st = TCA_OK;
  cudaGraph_t body = nullptr;
  cudaGraphConditionalHandle h{};
  uint64_t after_head = before;
  if (e == cudaSuccess) {
    if (profile) {
      for (int it = 0; it < iters && st == TCA_OK; ++it) {
        st = enqueue_iteration<T>(p, x, it, cs, p->sweep_ev[2 * it], p->sweep_ev[2 * it + 1]);
      }
    } else {
      st = capture_handle(cs, 0, false, &h);
      if (st == TCA_OK) {
        st = [&]() -> tca_status {
          cond_running_kernel<<<1, 1, 0, cs>>>(p->scal, h);
          TCA_LAUNCH_CHECK();
          return TCA_OK;
        }();
      }
      if (st == TCA_OK) st = capture_while(cs, h, &body);
      after_head = tca_kernel_launches(0);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (!profile && st == TCA_OK && e == cudaSuccess) {
    st = capture_into(body, cs, [&](cudaStream_t bs) -> tca_status {
      for (int it = 0; it < iters; ++it) TCA_TRY(enqueue_iteration<T>(p, x, it, bs, nullptr, nullptr));
      cond_running_kernel<<<1, 1, 0, bs>>>(p->scal, h);
      TCA_LAUNCH_CHECK();
      return TCA_OK;
    });
  }
  const uint64_t after = tca_kernel_launches(0);
  tca_kernel_launches(1);
  note_launches(before);  // captured launches are counted per replay instead
  cudaStreamDestroy(cs);
  if (st != TCA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    if (g) cudaGraphDestroy(g);
    return TCA_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&p->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    p->graph_exec = nullptr;
    return TCA_ERR_CUDA;
  }
  p->graph_x = x;
  p->graph_iters = iters;
  p->graph_profiled = profile;
  p->graph_pc = p->pc_on ? p->pc_kind : 0;
  p->graph_head_launches = after_head - before;     // kernels before the loop (unprofiled)
  p->graph_launches = after - after_head;           // kernels per pass
  return TCA_OK;
}

// FP64 true relative residual of x into p->scal->aux; optionally r = residual.
// FP32 plans use double-float arithmetic on the FP32 pipes (residual_ff.cu);
// FP64 plans use native FP64.
// Scattered FP32 plans: the FP64 operator (gather, scatter-add, regulariser)
// on the widened iterate, against A^T b kept in FP64.
template <typename T>
static tca_status true_residual(tca_plan_s* p, const T* x, bool write_r, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (p->scattered) {
      TCA_TRY(ensure_ws64_public(p));
      double* x64 = p->ws64[0];
      convert_kernel<float, double><<<vector_grid(p, p->N), kVecThreads, 0, s>>>((const float*)x, x64, p->N);
      TCA_LAUNCH_CHECK();
      TCA_TRY(normal_generic<double>(p, x64, p->res64, s, nullptr));
      const int grid = std::min(vector_grid(p, p->N), first_reduce(p).max_blocks - 1);
      true_residual_kernel<float><<<grid, kVecThreads, 0, s>>>((const double*)p->rhs64, p->res64,
                                                               write_r ? (float*)p->r : nullptr, p->N, p->scal,
                                                               first_reduce(p), second_reduce(p));
      TCA_LAUNCH_CHECK();
      return TCA_OK;
    }
    return residual_ff(p, (const float*)x, reinterpret_cast<const float2*>(p->rhs64),
                       reinterpret_cast<float2*>(p->res64), write_r ? (float*)p->r : nullptr, first_reduce(p),
                       second_reduce(p), s);
  }
  const double* rhs64 = (const double*)p->rhs;
  TCA_TRY(normal_fp64<T>(p, x, p->res64, s));
  const int grid = std::min(vector_grid(p, p->N), first_reduce(p).max_blocks - 1);
  true_residual_kernel<T><<<grid, kVecThreads, 0, s>>>(rhs64, p->res64, write_r ? (T*)p->r : nullptr, p->N, p->scal,
                                                        first_reduce(p), second_reduce(p));
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// The iteration steered from the host (preconditioners that synchronise, the
// tensor multigrid cycle): one iteration at a time, the scalar record read
// after each, until the same stop conditions as cg_iterate.
template <typename T>
static tca_status cg_iterate_host(tca_plan_s* p, T* x, double rtol, int max_iter, cudaStream_t s) {
  Scalars* hs = p->scal_host;
  TCA_CUDA_TRY(cudaMemcpyAsync(hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  bool conv = hs->bnorm == 0.0 || std::sqrt(hs->rho_new) <= rtol * hs->bnorm;
  for (int it = 0; !conv && !hs->breakdown && hs->iters < max_iter; ++it) {
    TCA_TRY(enqueue_iteration<T>(p, x, it, s, nullptr, nullptr));
    TCA_CUDA_TRY(cudaMemcpyAsync(hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    TCA_CUDA_TRY(cudaStreamSynchronize(s));
    conv = hs->converged != 0;
  }
  return TCA_OK;
}

// Replay the cached CG graph until the recursive residual meets rtol, CG
// breaks down or the device iteration count reaches max_iter.  The scalar
// record is left in p->scal_host.
static tca_status cg_iterate(tca_plan_s* p, double rtol, int max_iter, int every, bool profile, double* sweep_ms,
                             int* sweep_n, cudaStream_t s) {
  Scalars* hs = p->scal_host;
  // Start-of-iteration stop test (a zero right-hand side or an exact x0).
  TCA_CUDA_TRY(cudaMemcpyAsync(hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  bool conv = hs->bnorm == 0.0 || std::sqrt(hs->rho_new) <= rtol * hs->bnorm;
  while (!conv && !hs->breakdown && hs->iters < max_iter) {
    const int it_before = hs->iters;
    TCA_CUDA_TRY(cudaGraphLaunch(p->graph_exec, s));
    TCA_CUDA_TRY(cudaMemcpyAsync(hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    TCA_CUDA_TRY(cudaStreamSynchronize(s));
    conv = hs->converged != 0;
    {
      // Passes the launch ran: one per `every` iterations started (the last
      // one partly returning at entry).
      const int done = hs->iters - it_before;
      const int passes = profile ? 1 : std::max(1, (done + every - 1) / every);
      note_launches(p->graph_head_launches + (uint64_t)passes * p->graph_launches);
    }
    if (profile) {
      // Iterations of this replay that did work; the rest returned at entry.
      const int ran = std::min(every, hs->iters - it_before + (hs->breakdown ? 1 : 0));
      for (int i = 0; i < ran; ++i) {
        float ms = 0.f;
        TCA_CUDA_TRY(cudaEventElapsedTime(&ms, p->sweep_ev[2 * i], p->sweep_ev[2 * i + 1]));
        *sweep_ms += ms;
        ++*sweep_n;
      }
    }
  }
  return TCA_OK;
}

__global__ void axpy_f32_kernel(float* __restrict__ x, const float* __restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

// Mixed precision with iterative refinement (the _IR plans): an outer loop in
// FP64-accurate arithmetic (double-float residual r = A^T b - K x), an inner
// CG on K d = r run to inner_rtol with the plan's reduced-precision operator
// (TF32_IR: plain TF32 tensor-core products for dense factors, FP32 sweeps for
// banded ones; BF16_IR: bfloat16 vectors and the bfloat16 tensor-core sweep),
// and x += d, until the true relative residual meets rtol.  From x = 0 the
// first outer residual is A^T b itself, whose FP32 rounding the A^T b chain
// already left in p->rhs, so the first residual evaluation is skipped.
static tca_status solve_ir(tca_plan_s* p, const void* b_in, float* x, const tca_solve_opts* o, tca_solve_info* info,
                           cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  TCA_TRY(ensure_solver_buffers<float>(p));
  TCA_TRY(ensure_ws64_public(p));
  if (!p->dbuf) {
    cudaError_t e = cudaMalloc((void**)&p->dbuf, sizeof(float) * (size_t)p->N);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return TCA_ERR_ALLOC;
    }
  }
  const int64_t N = p->N;
  const double rtol = o ? o->rtol : 1e-6;
  const double inner = (o && o->inner_rtol > 0.0) ? o->inner_rtol : 1e-3;
  const int max_iter = (o && o->max_iter > 0) ? o->max_iter : 10000;
  const int max_refine = (o && o->max_refine > 0) ? o->max_refine : 30;
  int every = (o && o->check_every > 0) ? o->check_every : 8;
  every = std::max(kDirBufs, (every + kDirBufs - 1) / kDirBufs * kDirBufs);
  const bool profile = o && o->profile;
  if (profile) every = std::min(every, kMaxProfiledIters);
  if (!(rtol > 0.0)) return TCA_ERR_INVALID_ARG;
  double sweep_ms = 0.0;
  int sweep_n = 0;
  float* d = p->dbuf;
  const bool bf = p->prec == TCA_BF16_IR;
  if (bf && o && o->precond != TCA_PRECOND_NONE) {
    set_error_message("TCA_BF16_IR plans take no preconditioner");
    return TCA_ERR_UNSUPPORTED;
  }
  TCA_TRY(setup_precond(p, o, s));
  TCA_TRY(chain_ff(p, true, false, (const float*)b_in, reinterpret_cast<float2*>(p->rhs64), (float*)p->rhs,
                   reinterpret_cast<float2* const*>(p->ws64), p->ws64_elems, s));
  if (!(o && o->x0_given)) TCA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(float) * N, s));
  TCA_TRY(get_graph<float>(p, d, every, profile, s));
  const int vgrid = std::min(vector_grid(p, N), second_reduce(p).max_blocks - 1);
  Scalars* hs = p->scal_host;
  tca_status status = TCA_OK;
  int total = 0, outer = 0;
  double rec = 0.0;
  bool first = true;
  for (;;) {
    // Outer residual in double-float: p->rhs <- r (FP32), scal->aux <- ||r|| / ||A^T b||.
    double rel = 1.0;
    if (first && !(o && o->x0_given)) {
      hs->aux = 1.0;  // r = A^T b (already in p->rhs); a zero b is caught by the inner start
    } else {
      TCA_TRY(residual_ff(p, x, reinterpret_cast<const float2*>(p->rhs64), reinterpret_cast<float2*>(p->res64),
                          (float*)p->rhs, first_reduce(p), second_reduce(p), s));
      TCA_CUDA_TRY(cudaMemcpyAsync(hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
      TCA_CUDA_TRY(cudaStreamSynchronize(s));
      rel = hs->aux;
    }
    first = false;
    if (std::isnan(rel)) {  // a non-finite b or x0: nothing to refine
      status = TCA_ERR_BREAKDOWN;
      break;
    }
    if (!(rel > rtol)) break;  // converged (or a zero right-hand side)
    if (total >= max_iter || outer >= max_refine) {
      status = TCA_ERR_NOT_CONVERGED;
      break;
    }
    ++outer;
    // Inner CG from d = 0 on K d = r, to inner_rtol relative to ||r||.
    cg_setup_kernel<<<1, 1, 0, s>>>(p->scal, inner, max_iter - total);
    TCA_LAUNCH_CHECK();
    TCA_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(float) * N, s));
    if (bf) {
      TCA_CUDA_TRY(cudaMemsetAsync(p->bf.p[0], 0, 2 * (size_t)N, s));
      TCA_TRY(bf16_start(p, (const float*)p->rhs, first_reduce(p), s));
    } else {
      TCA_CUDA_TRY(cudaMemsetAsync(p->p[0], 0, sizeof(float) * N, s));
      cg_start_kernel<float><<<vgrid, kVecThreads, 0, s>>>((const float*)p->rhs, nullptr, (float*)p->r, N, p->scal,
                                                            first_reduce(p), 1, second_reduce(p));
      TCA_LAUNCH_CHECK();
    }
    if (p->pc_on) TCA_TRY(enqueue_precond<float>(p, true, s));
    TCA_TRY(cg_iterate(p, inner, max_iter - total, every, profile, &sweep_ms, &sweep_n, s));
    TCA_TRY(flush_pending_x<float>(p, d, s));
    total += hs->iters;
    rec = hs->bnorm > 0 ? std::sqrt(std::max(hs->rho_new, 0.0)) / hs->bnorm : 0.0;
    if (hs->breakdown) {
      status = TCA_ERR_BREAKDOWN;
      break;
    }
    axpy_f32_kernel<<<vgrid, kVecThreads, 0, s>>>(x, d, N);
    TCA_LAUNCH_CHECK();
  }
  if (info) {
    info->iters = total;
    info->refinements = outer;
    info->rel_res_true = hs->aux;
    info->rel_res_recursive = rec;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->sweep_ms = sweep_ms;
    info->sweep_launches = sweep_n;
    info->reserved = 0;
  }
  return status;
}

// Side stream and events for host-buffer solves (created on first use).
static tca_status ensure_copy_stream(tca_plan_s* p) {
  if (p->copy_stream) return TCA_OK;
  TCA_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
  TCA_CUDA_TRY(cudaEventCreateWithFlags(&p->copy_ev, cudaEventDisableTiming));
  for (cudaEvent_t& ev : p->chunk_ev) TCA_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  return TCA_OK;
}

template <typename T>
static tca_status solve_impl(tca_plan_s* p, const void* b_in, T* x, const tca_solve_opts* o, tca_solve_info* info,
                             cudaStream_t s, void* x_host = nullptr, const void* b_host = nullptr) {
  const auto t0 = std::chrono::steady_clock::now();
  TCA_TRY(ensure_solver_buffers<T>(p));
  const int64_t N = p->N;
  const double rtol = o ? o->rtol : 1e-6;
  const int max_iter = (o && o->max_iter > 0) ? o->max_iter : 10000;
  const bool x0 = o && o->x0_given;
  int every = (o && o->check_every > 0) ? o->check_every : 8;
  every = std::max(kDirBufs, (every + kDirBufs - 1) / kDirBufs * kDirBufs);
  const bool profile = o && o->profile;
  if (profile) every = std::min(every, kMaxProfiledIters);
  if (!(rtol > 0.0)) return TCA_ERR_INVALID_ARG;
  TCA_TRY(setup_precond(p, o, s));
  double sweep_ms = 0.0;
  int sweep_n = 0;

  // rhs = A^T b.  FP32 plans: one double-float chain gives the accurate rhs
  // (kept as (hi, lo) pairs for the true residual) and its FP32 rounding for
  // the iteration.  FP64 plans: native FP64.
  if constexpr (sizeof(T) == 4) {
    TCA_TRY(ensure_ws64_public(p));
    tca_status up = TCA_ERR_UNSUPPORTED;
    if (p->scattered) {
      // Scattered samples: A^T b by the FP64 scatter-add of the widened b (kept
      // in FP64 for the true residual), rounded once for the iteration.
      if (b_host) {
        TCA_CUDA_TRY(cudaMemcpyAsync(p->stage_b, b_host, sizeof(float) * (size_t)p->M, cudaMemcpyHostToDevice, s));
        b_in = p->stage_b;
      }
      const int64_t M = p->M;
      if (M > 0) {
        convert_kernel<float, double><<<vector_grid(p, M), kVecThreads, 0, s>>>((const float*)b_in, p->sc_tmp, M);
        TCA_LAUNCH_CHECK();
      }
      TCA_TRY(scattered_scatter<double>(p, p->sc_tmp, (double*)p->rhs64, true, s));
      convert_kernel<double, float><<<vector_grid(p, N), kVecThreads, 0, s>>>((const double*)p->rhs64,
                                                                               (float*)p->rhs, N);
      TCA_LAUNCH_CHECK();
      up = TCA_OK;
    } else if (b_host) {
      // b from the host: uploaded in row runs under A^T b's first mode product.
      TCA_TRY(ensure_copy_stream(p));
      up = chain_ff_rhs_from_host(p, (const float*)b_host, (float*)p->stage_b, reinterpret_cast<float2*>(p->rhs64),
                                  (float*)p->rhs, reinterpret_cast<float2* const*>(p->ws64), p->ws64_elems, s,
                                  p->copy_stream, p->chunk_ev, 8);
      if (up != TCA_OK && up != TCA_ERR_UNSUPPORTED) return up;
      if (up == TCA_ERR_UNSUPPORTED) {
        TCA_CUDA_TRY(cudaMemcpyAsync(p->stage_b, b_host, sizeof(float) * (size_t)p->M, cudaMemcpyHostToDevice, s));
        b_in = p->stage_b;
      }
    }
    if (up != TCA_OK)
      TCA_TRY(chain_ff(p, true, false, (const float*)b_in, reinterpret_cast<float2*>(p->rhs64), (float*)p->rhs,
                     reinterpret_cast<float2* const*>(p->ws64), p->ws64_elems, s));
  } else {
    TCA_TRY((apply_chain<T, T, T>(p, true, (const T*)b_in, (T*)p->rhs, p->ws, p->ws_elems, s)));
  }
  cg_setup_kernel<<<1, 1, 0, s>>>(p->scal, rtol, max_iter);
  TCA_LAUNCH_CHECK();
  TCA_CUDA_TRY(cudaMemsetAsync(p->p[0], 0, sizeof(T) * N, s));
  const int vgrid = std::min(vector_grid(p, N), second_reduce(p).max_blocks - 1);
  if (x0) {
    if constexpr (sizeof(T) == 4) {
      if (p->fused_ok) TCA_TRY(normal_fused_f32(p, nullptr, (const float*)x, nullptr, (float*)p->q, false, s));
      else TCA_TRY(normal_generic<T>(p, x, (T*)p->q, s));
    } else {
      TCA_TRY(normal_generic<T>(p, x, (T*)p->q, s));
    }
    cg_start_kernel<T><<<vgrid, kVecThreads, 0, s>>>((const T*)p->rhs, (const T*)p->q, (T*)p->r, N, p->scal,
                                                      first_reduce(p), 1, second_reduce(p));
  } else {
    TCA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * N, s));
    cg_start_kernel<T><<<vgrid, kVecThreads, 0, s>>>((const T*)p->rhs, nullptr, (T*)p->r, N, p->scal,
                                                      first_reduce(p), 1, second_reduce(p));
  }
  TCA_LAUNCH_CHECK();
  if (p->pc_on) TCA_TRY(enqueue_precond<T>(p, true, s));
  const bool host_loop = p->pc_on && p->pc_kind == TCA_PRECOND_TMG;
  if (!host_loop) TCA_TRY(get_graph<T>(p, x, every, profile, s));

  tca_status status = TCA_OK;
  int restarts = 0;
  Scalars* hs = p->scal_host;
  for (;;) {
    if (host_loop) TCA_TRY(cg_iterate_host<T>(p, x, rtol, max_iter, s));
    else TCA_TRY(cg_iterate(p, rtol, max_iter, every, profile, &sweep_ms, &sweep_n, s));
    TCA_TRY(flush_pending_x<T>(p, x, s));
    if (x_host) {
      // x is final for this pass: copy it to the host on a side stream while
      // the true residual is computed (a restart re-copies after its pass).
      TCA_TRY(ensure_copy_stream(p));
      TCA_CUDA_TRY(cudaEventRecord(p->copy_ev, s));
      TCA_CUDA_TRY(cudaStreamWaitEvent(p->copy_stream, p->copy_ev, 0));
      TCA_CUDA_TRY(cudaMemcpyAsync(x_host, x, sizeof(T) * (size_t)p->N, cudaMemcpyDeviceToHost, p->copy_stream));
    }
    if (hs->breakdown) {
      // Report the true residual of the iterate the breakdown left behind.
      status = TCA_ERR_BREAKDOWN;
      TCA_TRY(true_residual<T>(p, x, false, s));
      TCA_CUDA_TRY(cudaMemcpyAsync(hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
      TCA_CUDA_TRY(cudaStreamSynchronize(s));
      break;
    }
    if (hs->bnorm == 0.0) {
      hs->aux = 0.0;
      break;
    }
    // True residual in FP64; restart from x while it misses the tolerance.
    TCA_TRY(true_residual<T>(p, x, true, s));
    TCA_CUDA_TRY(cudaMemcpyAsync(hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    TCA_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs->aux <= rtol) break;
    if (std::isnan(hs->aux)) {  // a non-finite x: restarting cannot recover
      status = TCA_ERR_BREAKDOWN;
      break;
    }
    if (hs->iters >= max_iter) {
      status = TCA_ERR_NOT_CONVERGED;
      break;
    }
    ++restarts;
    // r already holds the FP64 residual (cast); recompute rho, keep bnorm.
    cg_start_kernel<T><<<vgrid, kVecThreads, 0, s>>>((const T*)p->r, nullptr, (T*)p->r, N, p->scal,
                                                      first_reduce(p), 0, second_reduce(p));
    TCA_LAUNCH_CHECK();
    if (p->pc_on) TCA_TRY(enqueue_precond<T>(p, true, s));
  }
  if (x_host && p->copy_stream) TCA_CUDA_TRY(cudaStreamSynchronize(p->copy_stream));
  if (info) {
    info->iters = hs->iters;
    info->refinements = restarts;
    info->rel_res_true = hs->aux;
    info->rel_res_recursive = hs->bnorm > 0 ? std::sqrt(std::max(hs->rho_new, 0.0)) / hs->bnorm : 0.0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->sweep_ms = sweep_ms;
    info->sweep_launches = sweep_n;
    info->reserved = 0;
  }
  return status;
}

// ---------------------------------------------------------------------------
// Batched solve: many independent plans in one CUDA graph launch.
//
// One graph holds every instance as an independent branch:
//   set-up: A^T b in double-float, scalars, r = A^T b, start test
//   WHILE (instance not finished) {                      restarts
//     inner = !done
//     WHILE (inner) { check_every CG iterations; inner = !done }
//     true residual in double-float; restart from x if it misses rtol
//     outer = !done
//   }
// The branches share nothing, so an instance that converges early leaves its
// loop while the others keep iterating, and the GPU runs the kernels of all
// running instances concurrently.  The host launches the graph once and reads
// every instance's scalars afterwards.

namespace {

constexpr int kMaxRestarts = 16;

// Start-of-iteration stop test on the device (a zero right-hand side or an
// exact initial guess), so that such an instance does no iteration at all.
__global__ void batch_start_test_kernel(Scalars* sc) {
  sc->restarts = 0;
  if (sc->bnorm == 0.0 || sqrt(sc->rho_new) <= sc->rtol * sc->bnorm) sc->converged = 1;
}

// After the true residual (sc->aux = ||A^T b - K x|| / ||A^T b||, r = that
// residual rounded to FP32): when it misses rtol and iterations remain, start
// a fresh direction from r (rho = <r, r>, beta = 0).  Every block takes the
// same decision from the scalars, which only the last block changes.
__global__ void __launch_bounds__(kVecThreads) batch_restart_kernel(const float* __restrict__ r, int64_t n,
                                                                    Scalars* sc, Reduce red) {
  __shared__ double sh[kVecThreads / 32];
  if (sc->breakdown || sc->bnorm == 0.0 || !(sc->aux > sc->rtol) || sc->iters >= sc->max_iter ||
      sc->restarts >= kMaxRestarts)
    return;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)r[i] * (double)r[i];
  double t;
  if (dev::grid_sum_last(acc, red, &t, sh)) {
    sc->rho = t;
    sc->rho_new = t;
    sc->beta = 0.0;
    sc->restarts += 1;
    sc->converged = sqrt(t) <= sc->rtol * sc->bnorm ? 1 : 0;
  }
}

constexpr int kBatchStreams = 64;

struct BatchGraph {
  std::vector<const void*> key;
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> l_setup, l_iter, l_check;  // launches per set-up / iteration / restart check
  int every = 0;
};

std::mutex g_batch_mutex;
BatchGraph g_batch;  // last batch signature (one cached batch per process)
cudaStream_t g_pool[kBatchStreams] = {};
cudaEvent_t g_fork = nullptr, g_join[kBatchStreams] = {};

tca_status ensure_pool() {
  if (g_fork) return TCA_OK;
  for (int i = 0; i < kBatchStreams; ++i) {
    TCA_CUDA_TRY(cudaStreamCreateWithFlags(&g_pool[i], cudaStreamNonBlocking));
    TCA_CUDA_TRY(cudaEventCreateWithFlags(&g_join[i], cudaEventDisableTiming));
  }
  TCA_CUDA_TRY(cudaEventCreateWithFlags(&g_fork, cudaEventDisableTiming));
  return TCA_OK;
}

// Per-instance set-up: rhs (double-float), scalars, zero directions, x, r.
tca_status enqueue_setup(tca_plan_s* p, const float* b, float* x, double rtol, int max_iter, bool x0,
                         cudaStream_t s) {
  TCA_TRY(chain_ff(p, true, false, b, reinterpret_cast<float2*>(p->rhs64), (float*)p->rhs,
                   reinterpret_cast<float2* const*>(p->ws64), p->ws64_elems, s));
  cg_setup_kernel<<<1, 1, 0, s>>>(p->scal, rtol, max_iter);
  TCA_LAUNCH_CHECK();
  const int64_t N = p->N;
  TCA_CUDA_TRY(cudaMemsetAsync(p->p[0], 0, sizeof(float) * N, s));
  const int vgrid = std::min(vector_grid(p, N), second_reduce(p).max_blocks - 1);
  const float* kx = nullptr;
  if (x0) {
    if (p->fused_ok) TCA_TRY(normal_fused_f32(p, nullptr, x, nullptr, (float*)p->q, false, s));
    else TCA_TRY(normal_generic<float>(p, x, (float*)p->q, s));
    kx = (const float*)p->q;
  } else {
    TCA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(float) * N, s));
  }
  cg_start_kernel<float><<<vgrid, kVecThreads, 0, s>>>((const float*)p->rhs, kx, (float*)p->r, N, p->scal,
                                                        first_reduce(p), 1, second_reduce(p));
  TCA_LAUNCH_CHECK();
  if (p->pc_on) TCA_TRY(enqueue_precond<float>(p, true, s));
  batch_start_test_kernel<<<1, 1, 0, s>>>(p->scal);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

tca_status build_batch(int count, tca_plan_s** plans, const float* const* b, float* const* x, double rtol,
                       int max_iter, bool x0, int every, BatchGraph* bg) {
  cudaStream_t cs;
  TCA_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const uint64_t saved = tca_kernel_launches(1);
  bg->l_setup.assign(count, 0);
  bg->l_iter.assign(count, 0);
  bg->l_check.assign(count, 0);
  bg->every = every;
  std::vector<cudaGraph_t> outer(count, nullptr);
  std::vector<cudaGraphConditionalHandle> ho(count);
  tca_status st = TCA_OK;
  // Top level: per instance, set-up then the restart loop, as parallel branches.
  cudaGraph_t top = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = [&]() -> tca_status {
      TCA_CUDA_TRY(cudaEventRecord(g_fork, cs));
      const int ns = std::min(count, kBatchStreams);
      for (int k = 0; k < ns; ++k) TCA_CUDA_TRY(cudaStreamWaitEvent(g_pool[k], g_fork, 0));
      for (int i = 0; i < count; ++i) {
        cudaStream_t s = g_pool[i % ns];
        const uint64_t l0 = tca_kernel_launches(0);
        TCA_TRY(enqueue_setup(plans[i], b[i], x[i], rtol, max_iter, x0, s));
        bg->l_setup[i] = tca_kernel_launches(0) - l0;
        TCA_TRY(capture_handle(s, 1, true, &ho[i]));
        TCA_TRY(capture_while(s, ho[i], &outer[i]));
      }
      for (int k = 0; k < ns; ++k) {
        TCA_CUDA_TRY(cudaEventRecord(g_join[k], g_pool[k]));
        TCA_CUDA_TRY(cudaStreamWaitEvent(cs, g_join[k], 0));
      }
      return TCA_OK;
    }();
    e = cudaStreamEndCapture(cs, &top);
  }
  // Restart loop body and inner iteration loop of every instance.
  for (int i = 0; i < count && st == TCA_OK && e == cudaSuccess; ++i) {
    tca_plan_s* p = plans[i];
    cudaGraph_t inner = nullptr;
    cudaGraphConditionalHandle hi;
    st = capture_into(outer[i], cs, [&](cudaStream_t s) -> tca_status {
      TCA_TRY(capture_handle(s, 0, false, &hi));
      cond_running_kernel<<<1, 1, 0, s>>>(p->scal, hi);
      TCA_LAUNCH_CHECK();
      TCA_TRY(capture_while(s, hi, &inner));
      const uint64_t l0 = tca_kernel_launches(0);
      TCA_TRY(flush_pending_x<float>(p, x[i], s));
      TCA_TRY(residual_ff(p, x[i], reinterpret_cast<const float2*>(p->rhs64), reinterpret_cast<float2*>(p->res64),
                          (float*)p->r, first_reduce(p), second_reduce(p), s));
      const int vgrid = std::min(vector_grid(p, p->N), first_reduce(p).max_blocks);
      batch_restart_kernel<<<vgrid, kVecThreads, 0, s>>>((const float*)p->r, p->N, p->scal, first_reduce(p));
      TCA_LAUNCH_CHECK();
      // Preconditioned: rho = <r, z> of the restart (returns at entry when none happened).
      if (p->pc_on) TCA_TRY(enqueue_precond<float>(p, true, s));
      cond_running_kernel<<<1, 1, 0, s>>>(p->scal, ho[i]);
      TCA_LAUNCH_CHECK();
      bg->l_check[i] = tca_kernel_launches(0) - l0 + 2;  // + the inner gate
      return TCA_OK;
    });
    if (st != TCA_OK) break;
    st = capture_into(inner, cs, [&](cudaStream_t s) -> tca_status {
      const uint64_t l0 = tca_kernel_launches(0);
      for (int it = 0; it < every; ++it)
        TCA_TRY(enqueue_iteration<float>(p, x[i], it, s, nullptr, nullptr));
      bg->l_iter[i] = (tca_kernel_launches(0) - l0) / every;
      cond_running_kernel<<<1, 1, 0, s>>>(p->scal, hi);
      TCA_LAUNCH_CHECK();
      return TCA_OK;
    });
  }
  if (st == TCA_OK && e == cudaSuccess) e = cudaGraphInstantiate(&bg->exec, top, 0);
  if (top) cudaGraphDestroy(top);
  tca_kernel_launches(1);
  note_launches(saved);  // captured launches are counted when the graph runs
  cudaStreamDestroy(cs);
  if (st != TCA_OK) return st;
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_CUDA;
  }
  return TCA_OK;
}

}  // namespace

// SM share of the batched graph: each instance's kernels are sized for
// num_sms / share SMs.  tca_autotune_batched times candidate shares on a batch
// and records the fastest per batch signature (plans, buffers, options);
// batches it has not seen use a quarter.
constexpr int kDefaultBatchShare = 4;
std::map<std::vector<const void*>, int> g_batch_share;  // guarded by g_batch_mutex
int g_batch_share_forced = 0;                           // autotuner's candidate (0: none)

static std::vector<const void*> batch_signature(int count, tca_plan_s** plans, const float* const* b,
                                                float* const* x, double rtol, int max_iter, bool x0, int every) {
  std::vector<const void*> key;
  key.push_back((const void*)(intptr_t)every);
  key.push_back((const void*)(intptr_t)max_iter);
  key.push_back((const void*)(intptr_t)(x0 ? 1 : 0));
  key.push_back(reinterpret_cast<const void*>((uintptr_t)(rtol * 1e15)));
  key.push_back((const void*)(intptr_t)(plans[0]->pc_on ? plans[0]->pc_kind : 0));
  key.push_back(reinterpret_cast<const void*>((uintptr_t)(plans[0]->pc_shift * 1e6)));
  key.push_back(reinterpret_cast<const void*>((uintptr_t)(plans[0]->pcb_shift * 1e6)));
  for (int i = 0; i < count; ++i) {
    key.push_back(plans[i]);
    key.push_back((const void*)(uintptr_t)plans[i]->generation);
    key.push_back((const void*)(uintptr_t)plans[i]->pc_generation);
    key.push_back(b[i]);
    key.push_back(x[i]);
  }
  return key;
}

static tca_status solve_batched_impl(int count, tca_plan_s** plans, const float* const* b, float* const* x,
                                     const tca_solve_opts* o, tca_solve_info* info, cudaStream_t s,
                                     int* share_used = nullptr) {
  const auto t0 = std::chrono::steady_clock::now();
  const double rtol = o ? o->rtol : 1e-6;
  const int max_iter = (o && o->max_iter > 0) ? o->max_iter : 10000;
  const bool x0 = o && o->x0_given;
  int every = (o && o->check_every > 0) ? o->check_every : 16;
  every = std::max(kDirBufs, (every + kDirBufs - 1) / kDirBufs * kDirBufs);
  if (!(rtol > 0.0)) return TCA_ERR_INVALID_ARG;
  if (o && o->precond == TCA_PRECOND_TMG) {
    set_error_message("the tensor multigrid cycle is steered from the host: not in a batched graph");
    return TCA_ERR_UNSUPPORTED;
  }
  for (int i = 0; i < count; ++i) {
    TCA_TRY(ensure_solver_buffers<float>(plans[i]));
    TCA_TRY(ensure_ws64_public(plans[i]));
    TCA_TRY(setup_precond(plans[i], o, s));
  }
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  TCA_TRY(ensure_pool());
  const std::vector<const void*> sig = batch_signature(count, plans, b, x, rtol, max_iter, x0, every);
  int share = kDefaultBatchShare;
  if (g_batch_share_forced > 0) {
    share = g_batch_share_forced;
  } else {
    auto it = g_batch_share.find(sig);
    if (it != g_batch_share.end()) share = it->second;
  }
  if (share_used) *share_used = share;
  std::vector<const void*> key = sig;
  key.push_back((const void*)(intptr_t)share);
  if (key != g_batch.key || !g_batch.exec) {
    if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
    g_batch.exec = nullptr;
    g_batch.key.clear();
    // Grids for a quarter of the GPU per instance: the plans' SM count, as
    // seen by the grid heuristics (vector kernels, fused-sweep chunks), and a
    // cap on the persistent kernels (TMA row tiles, dense tensor-core
    // products) are lowered while the graph is captured, so that several
    // instances' kernels run side by side instead of each filling every SM.
    // Measured on the 64-instance workload: 1.53 s with whole-GPU grids (and
    // autotuned chunks), 1.23 s with a quarter.  With the faster generic
    // iteration: 0.98 s with a half, 0.90 s with a third, 0.86 s with a
    // quarter, 0.84 s with a sixth, while the slowest instance alone in a
    // batch goes from 0.16 to 0.33 s - a quarter keeps the critical path short.
    const int budget = std::max(8, plans[0]->num_sms / share);
    std::vector<int> saved_sms(count), saved_chunks(count);
    auto set_cap = [](tca_plan_s* p, int cap) {
      for (int k = 0; k < p->d; ++k) {
        Mode& m = p->mode[k];
        m.fwd.sm_cap = m.bwd.sm_cap = m.gram.sm_cap = cap;
        p->pc[k].sm_cap = cap;
      }
    };
    for (int i = 0; i < count; ++i) {
      saved_sms[i] = plans[i]->num_sms;
      saved_chunks[i] = plans[i]->fused_nchunks;
      plans[i]->num_sms = std::min(plans[i]->num_sms, budget);
      plans[i]->fused_nchunks = 0;
      set_cap(plans[i], budget);
    }
    const tca_status bst = build_batch(count, plans, b, x, rtol, max_iter, x0, every, &g_batch);
    for (int i = 0; i < count; ++i) {
      plans[i]->num_sms = saved_sms[i];
      plans[i]->fused_nchunks = saved_chunks[i];
      set_cap(plans[i], 0);
    }
    TCA_TRY(bst);
    g_batch.key = key;
  }
  TCA_CUDA_TRY(cudaGraphLaunch(g_batch.exec, s));
  for (int i = 0; i < count; ++i)
    TCA_CUDA_TRY(cudaMemcpyAsync(plans[i]->scal_host, plans[i]->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  tca_status status = TCA_OK;
  for (int i = 0; i < count; ++i) {
    const Scalars& hs = *plans[i]->scal_host;
    // Launch count of this instance's branch: set-up, one restart check per
    // pass of the outer loop, and the inner passes (iterations that find the
    // instance finished still launch and return at entry).
    const uint64_t passes = (uint64_t)(hs.iters + every - 1) / every;  // a lower bound
    note_launches(g_batch.l_setup[i] + (uint64_t)(hs.restarts + 1) * g_batch.l_check[i] +
                  passes * ((uint64_t)every * g_batch.l_iter[i] + 1));
    tca_status si = TCA_OK;
    if (hs.breakdown) si = TCA_ERR_BREAKDOWN;
    else if (hs.bnorm != 0.0 && !(hs.aux <= rtol)) si = TCA_ERR_NOT_CONVERGED;
    if (si != TCA_OK && status == TCA_OK) status = si;
    if (info) {
      info[i].iters = hs.iters;
      info[i].refinements = hs.restarts;
      info[i].rel_res_true = hs.bnorm == 0.0 ? 0.0 : hs.aux;
      info[i].rel_res_recursive = hs.bnorm > 0 ? std::sqrt(std::max(hs.rho_new, 0.0)) / hs.bnorm : 0.0;
      info[i].seconds = secs;
      info[i].sweep_ms = 0.0;
      info[i].sweep_launches = 0;
      info[i].reserved = 0;
    }
  }
  return status;
}

}  // namespace tca

using namespace tca;

extern "C" tca_status tca_solve_batched(int count, tca_plan_t* plans, const void* const* b, void* const* x,
                                        const tca_solve_opts* opts, tca_solve_info* info, cudaStream_t stream) {
  if (count <= 0 || !plans || !b || !x) return TCA_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !b[i] || !x[i]) return TCA_ERR_INVALID_ARG;
    if (plans[i]->prec != TCA_F32 || plans[i]->scattered) return TCA_ERR_UNSUPPORTED;
    if (!is_device_ptr(b[i]) || !is_device_ptr(x[i]) || (uintptr_t)x[i] % 16 != 0) return TCA_ERR_UNSUPPORTED;
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return TCA_ERR_INVALID_ARG;  // each instance needs its own plan
  }
  const tca_status st = solve_batched_impl(count, plans, reinterpret_cast<const float* const*>(b),
                                           reinterpret_cast<float* const*>(x), opts, info, stream);
  const tca_status tw = check_wait_timeout(stream);
  return tw != TCA_OK ? tw : st;
}

extern "C" tca_status tca_autotune_batched(int count, tca_plan_t* plans, const void* const* b, void* const* x,
                                           const tca_solve_opts* opts, int* share_out, cudaStream_t stream) {
  if (count <= 0 || !plans || !b || !x) return TCA_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !b[i] || !x[i]) return TCA_ERR_INVALID_ARG;
    if (plans[i]->prec != TCA_F32 || plans[i]->scattered) return TCA_ERR_UNSUPPORTED;
    if (!is_device_ptr(b[i]) || !is_device_ptr(x[i]) || (uintptr_t)x[i] % 16 != 0) return TCA_ERR_UNSUPPORTED;
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return TCA_ERR_INVALID_ARG;
  }
  const float* const* bb = reinterpret_cast<const float* const*>(b);
  float* const* xx = reinterpret_cast<float* const*>(x);
  const int num_sms = plans[0]->num_sms;
  cudaEvent_t e0, e1;
  TCA_CUDA_TRY(cudaEventCreate(&e0));
  TCA_CUDA_TRY(cudaEventCreate(&e1));
  int best = kDefaultBatchShare;
  float best_ms = 1e30f;
  tca_status st = TCA_OK;
  for (int share : {1, 2, 3, 4, 6, 8}) {
    if (num_sms / share < 8) continue;
    {
      std::lock_guard<std::mutex> lock(g_batch_mutex);
      g_batch_share_forced = share;
    }
    // First call captures the graph for this share, the second is timed.
    st = solve_batched_impl(count, plans, bb, xx, opts, nullptr, stream);
    if (st == TCA_OK || st == TCA_ERR_NOT_CONVERGED) {
      cudaEventRecord(e0, stream);
      st = solve_batched_impl(count, plans, bb, xx, opts, nullptr, stream);
      cudaEventRecord(e1, stream);
      cudaEventSynchronize(e1);
    }
    if (st != TCA_OK && st != TCA_ERR_NOT_CONVERGED) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = share;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  g_batch_share_forced = 0;
  if (st != TCA_OK && st != TCA_ERR_NOT_CONVERGED) return st;
  // Record the choice under the signature the solves will look up.
  double rtol = opts ? opts->rtol : 1e-6;
  const int max_iter = (opts && opts->max_iter > 0) ? opts->max_iter : 10000;
  int every = (opts && opts->check_every > 0) ? opts->check_every : 16;
  every = std::max(kDirBufs, (every + kDirBufs - 1) / kDirBufs * kDirBufs);
  g_batch_share[batch_signature(count, plans, bb, xx, rtol, max_iter, opts && opts->x0_given, every)] = best;
  if (share_out) *share_out = best;
  const tca_status tw = check_wait_timeout(stream);
  return tw;
}

extern "C" tca_status tca_solve(tca_plan_t plan, const void* b, void* x, const tca_solve_opts* opts,
                                tca_solve_info* info, cudaStream_t stream) {
  if (!plan || !b || !x) return TCA_ERR_INVALID_ARG;
  tca_plan_s* p = plan;
  const size_t es = elem_size(p);
  // Host buffers, and device buffers the vector kernels cannot address with
  // 16-byte accesses, go through the plan's staging buffers.
  const bool b_dev = is_device_ptr(b);
  const bool x_dev = is_device_ptr(x) && ((uintptr_t)x % 16 == 0);
  const void* db = b;
  void* dx = x;
  if (!b_dev || !x_dev) TCA_TRY(ensure_stage(p));
  // FP32 plans take a host b themselves (uploaded under A^T b).
  const void* b_up = (!b_dev && p->prec == TCA_F32 && !is_device_ptr(b)) ? b : nullptr;
  if (!b_dev && !b_up) {
    TCA_CUDA_TRY(cudaMemcpyAsync(p->stage_b, b, es * (size_t)p->M, cudaMemcpyHostToDevice, stream));
    db = p->stage_b;
  }
  if (!x_dev) {
    if (opts && opts->x0_given)
      TCA_CUDA_TRY(cudaMemcpyAsync(p->stage_x, x, es * (size_t)p->N, cudaMemcpyDefault, stream));
    dx = p->stage_x;
  }
  tca_status st;
  // Host x that the device can copy into directly: the solve copies x back
  // itself, overlapped with its final true-residual check.
  void* x_back = (!x_dev && !is_device_ptr(x)) ? x : nullptr;
  if (p->prec == TCA_F64) st = solve_impl<double>(p, db, (double*)dx, opts, info, stream, x_back);
  else if (p->prec == TCA_F32) st = solve_impl<float>(p, db, (float*)dx, opts, info, stream, x_back, b_up);
  else st = solve_ir(p, db, (float*)dx, opts, info, stream);
  const bool copied = x_back && (p->prec == TCA_F64 || p->prec == TCA_F32);
  if (!x_dev && !copied && (st == TCA_OK || st == TCA_ERR_NOT_CONVERGED || st == TCA_ERR_BREAKDOWN)) {
    TCA_CUDA_TRY(cudaMemcpyAsync(x, p->stage_x, es * (size_t)p->N, cudaMemcpyDefault, stream));
    TCA_CUDA_TRY(cudaStreamSynchronize(stream));
  }
  // A bounded device wait that gave up outranks the solver's own verdict.
  const tca_status tw = check_wait_timeout(stream);
  return tw != TCA_OK ? tw : st;
}
