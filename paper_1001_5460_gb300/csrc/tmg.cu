// Tensor multigrid preconditioner (Sec. 4.2, Fig. 3): a two-grid V-cycle
// z = V r used as M^-1 inside the preconditioned CG.
//
//   pre-smoothing      z = S(0)                      (nu Chebyshev steps on D^-1 K)
//   restriction        r_c = P^T (r - K z)           (separable: one mode product per coarsened mode)
//   coarse solve       z_c = K_c^-1 r_c,  K_c = P^T K P  (CG to a relative tolerance)
//   prolongation       z += P z_c
//   post-smoothing     z = S(z)                      (the same polynomial)
//
// P = P_1 kron .. kron P_d with P_k linear interpolation from the even points
// of mode k (Table 1's up-sampling) or the identity on modes that are kept;
// restriction is its transpose.  Fig. 3 leaves the coarse-scale operator to
// GetScale: here it is the Galerkin product P^T K P, applied without being
// formed (prolong, the fine normal operator, restrict), and the direct solve
// at the last scale is reached by CG.  The smoother is Chebyshev iteration
// for K z = r with the point-Jacobi scaling D = diag(K) over
// [lambda_max / 30, 1.05 lambda_max] of D^-1 K (point Jacobi alone cannot be
// damped stably for this operator); lambda_max is given or estimated by power
// steps.  Every step is a kernel of this library: the transfers are the
// ELL-4 band mode products of a transfer plan (factor k = P_k), the fine
// operator is the plan's own (fused sweep or generic chain), and the vector
// updates and inner products are the kernels below (FP64 reductions).
#include <algorithm>
#include <cmath>
#include <vector>

#include "tca_internal.cuh"

namespace tca {

constexpr int kTmgThreads = 256;
constexpr int kPowerSteps = 60;         // power steps of the lambda_max estimate
constexpr int kMaxCoarseIters = 2000;   // cap on the coarse CG of one cycle
constexpr int kMaxNu = 64;
constexpr double kDefaultCoarseRtol = 0.3;
constexpr int kDefaultNu = 3;
constexpr int64_t kCoarsenMin = 16;     // default mask: modes at least this long

struct TmgState {
  int mask = 0;                 // modes coarsened
  int nu = kDefaultNu;          // smoothing steps before and after
  double coarse_rtol = kDefaultCoarseRtol;
  double lam_max = 0.0;         // in use
  double lam_est = 0.0;         // power-step estimate (0: not formed)
  int64_t n[kMaxModes] = {};    // fine sizes
  int64_t nc[kMaxModes] = {};   // coarse sizes
  int64_t Nc = 0;
  tca_plan_s* tp = nullptr;     // transfer plan: factor k = P_k (n_k x nc_k), ELL-4
  void* d = nullptr;            // fine: Chebyshev direction
  void* t = nullptr;            // fine: K z, residual, K P v
  void* u = nullptr;            // fine: P v
  void* xc = nullptr;           // coarse CG: solution, residual, direction, K_c p
  void* rc = nullptr;
  void* pc = nullptr;
  void* qc = nullptr;
  Scalars* sc = nullptr;        // coarse CG scalars and power-step norms (device)
  Scalars* sc_host = nullptr;   // pinned mirror
  int64_t coarse_iters = 0;
};

namespace {

__device__ __forceinline__ bool tmg_sum_last(double v, Reduce red, double* total) {
  __shared__ double sh[kTmgThreads / 32];
  return dev::grid_sum_last(v, red, total, sh);
}

// Counter-based pseudo-random start of the power steps: SplitMix64 of the
// index, its top 53 bits mapped to [-1, 1).
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_seed_kernel(T* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    v[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

// v = dinv * q (dinv null: v = q) and ||v||^2 -> *out.
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_scaled_norm_kernel(const T* __restrict__ q,
                                                                      const T* __restrict__ dinv, T* __restrict__ v,
                                                                      int64_t n, double* out, Reduce red) {
  double acc = 0.0;
  T part = T(0);
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T w = dinv ? q[i] * dinv[i] : q[i];
    v[i] = w;
    part += w * w;
    if (++cnt == 8) {  // short runs in T, FP64 beyond
      acc += (double)part;
      part = T(0);
      cnt = 0;
    }
  }
  acc += (double)part;
  double total;
  if (tmg_sum_last(acc, red, &total)) *out = total;
}

// v *= 1 / sqrt(*nrm2) (left unscaled when the norm is zero or not finite).
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_normalise_kernel(T* __restrict__ v, int64_t n,
                                                                    const double* nrm2) {
  const double s2 = *nrm2;
  if (!(s2 > 0.0) || !isfinite(s2)) return;
  const T f = (T)(1.0 / sqrt(s2));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= f;
}

// 16-byte vectors of the fine-size passes (float4 / double2).
template <typename T> struct Vec16;
template <> struct Vec16<float> { using t = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using t = double2; static constexpr int n = 2; };

// One Chebyshev step: d = cd d + cr D^-1 (r - t), then z = d (z_add 0) or
// z += d.  t null: K z = 0 (z is zero).  cd = 0: d is not read.  VEC: the
// pointers are 16-byte aligned; 16-byte vectors, the scalar tail by block 0.
template <typename T>
__device__ __forceinline__ void cheb_one(const T* __restrict__ r, const T* __restrict__ t,
                                         const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ z,
                                         int64_t i, T cd, T cr, bool keep_d, int z_add) {
  const T res = t ? r[i] - t[i] : r[i];
  T dn = cr * (res * dinv[i]);
  if (keep_d) dn += cd * d[i];
  d[i] = dn;
  z[i] = z_add ? z[i] + dn : dn;
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kTmgThreads) tmg_cheb_kernel(const T* __restrict__ r, const T* __restrict__ t,
                                                               const T* __restrict__ dinv, T* __restrict__ d,
                                                               T* __restrict__ z, int64_t n, T cd, T cr, int z_add) {
  const bool keep_d = cd != T(0);
  int64_t done = 0;
  if constexpr (VEC) {
    using VT = typename Vec16<T>::t;
    constexpr int VN = Vec16<T>::n;
    const int64_t nv = n / VN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
      VT rv = reinterpret_cast<const VT*>(r)[i];
      const VT gv = reinterpret_cast<const VT*>(dinv)[i];
      T* rs = reinterpret_cast<T*>(&rv);
      const T* gs = reinterpret_cast<const T*>(&gv);
      if (t) {
        const VT tv = reinterpret_cast<const VT*>(t)[i];
        const T* ts = reinterpret_cast<const T*>(&tv);
#pragma unroll
        for (int c = 0; c < VN; ++c) rs[c] = rs[c] - ts[c];
      }
      VT dv;
      T* ds = reinterpret_cast<T*>(&dv);
      if (keep_d) dv = reinterpret_cast<const VT*>(d)[i];
#pragma unroll
      for (int c = 0; c < VN; ++c) {
        T dn = cr * (rs[c] * gs[c]);
        if (keep_d) dn += cd * ds[c];
        ds[c] = dn;
      }
      reinterpret_cast<VT*>(d)[i] = dv;
      VT zv;
      T* zs = reinterpret_cast<T*>(&zv);
      if (z_add) zv = reinterpret_cast<const VT*>(z)[i];
#pragma unroll
      for (int c = 0; c < VN; ++c) zs[c] = z_add ? zs[c] + ds[c] : ds[c];
      reinterpret_cast<VT*>(z)[i] = zv;
    }
    done = nv * VN;
    if (blockIdx.x == 0)
      for (int64_t i = done + threadIdx.x; i < n; i += blockDim.x) cheb_one(r, t, dinv, d, z, i, cd, cr, keep_d, z_add);
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      cheb_one(r, t, dinv, d, z, i, cd, cr, keep_d, z_add);
  }
}

// t = r - t.
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_residual_kernel(const T* __restrict__ r, T* __restrict__ t,
                                                                   int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    t[i] = r[i] - t[i];
}

// z = u (z_add 0) or z += u.
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_add_kernel(T* __restrict__ z, const T* __restrict__ u, int64_t n,
                                                              int z_add) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = z_add ? z[i] + u[i] : u[i];
}

// ---- coarse CG (Fig. 2 on K_c, x_c = 0 at the start) ----------------------

// rho = <r_c, r_c>, bnorm = ||r_c||, fresh flags.
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_cstart_kernel(const T* __restrict__ rc, int64_t n, Scalars* sc,
                                                                 Reduce red) {
  double acc = 0.0;
  T part = T(0);
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    part += rc[i] * rc[i];
    if (++cnt == 8) {
      acc += (double)part;
      part = T(0);
      cnt = 0;
    }
  }
  acc += (double)part;
  double total;
  if (tmg_sum_last(acc, red, &total)) {
    sc->rho = total;
    sc->rho_new = total;
    sc->bnorm = sqrt(total);
    sc->beta = 0.0;
    sc->converged = 0;
    sc->breakdown = 0;
    sc->iters = 0;
  }
}

// p_c = r_c (first) or r_c + beta p_c.
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_cdir_kernel(const T* __restrict__ rc, T* __restrict__ pc,
                                                               int64_t n, const Scalars* sc, int first) {
  const T beta = (T)sc->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pc[i] = first ? rc[i] : rc[i] + beta * pc[i];
}

// <p_c, q_c> -> alpha = rho / <p_c, q_c>; breakdown unless it is positive and finite.
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_calpha_kernel(const T* __restrict__ pc, const T* __restrict__ qc,
                                                                 int64_t n, Scalars* sc, Reduce red) {
  double acc = 0.0;
  T part = T(0);
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    part += pc[i] * qc[i];
    if (++cnt == 8) {
      acc += (double)part;
      part = T(0);
      cnt = 0;
    }
  }
  acc += (double)part;
  double total;
  if (tmg_sum_last(acc, red, &total)) {
    sc->pq = total;
    if (!(total > 0.0) || !isfinite(total)) {
      sc->breakdown = 1;
      sc->alpha = 0.0;
    } else {
      sc->alpha = sc->rho / total;
    }
  }
}

// x_c += alpha p_c; r_c -= alpha q_c; rho1 = <r_c, r_c>; beta = rho1 / rho; rho = rho1.
template <typename T>
__global__ void __launch_bounds__(kTmgThreads) tmg_cupdate_kernel(T* __restrict__ xc, T* __restrict__ rc,
                                                                  const T* __restrict__ pc, const T* __restrict__ qc,
                                                                  int64_t n, Scalars* sc, Reduce red) {
  if (sc->breakdown) return;
  const T alpha = (T)sc->alpha;
  double acc = 0.0;
  T part = T(0);
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    xc[i] += alpha * pc[i];
    const T rv = rc[i] - alpha * qc[i];
    rc[i] = rv;
    part += rv * rv;
    if (++cnt == 8) {
      acc += (double)part;
      part = T(0);
      cnt = 0;
    }
  }
  acc += (double)part;
  double total;
  if (tmg_sum_last(acc, red, &total)) {
    sc->beta = total / sc->rho;
    sc->rho = total;
    sc->rho_new = total;
    sc->iters += 1;
  }
}

Reduce half_reduce(const tca_plan_s* p) {
  Reduce r = p->red;
  r.max_blocks = p->red.max_blocks / 2;
  return r;
}

int tmg_grid(const tca_plan_s* p, int64_t n) {
  return std::max(1, std::min(vector_grid(p, n), half_reduce(p).max_blocks));
}

// The plan's fine normal operator y = K x (its fused sweep where it has one).
template <typename T>
tca_status tmg_normal(tca_plan_s* p, const T* x, T* y, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (p->fused_ok) {
      const tca_status st = normal_fused_f32(p, nullptr, x, nullptr, y, false, s);
      if (st != TCA_ERR_UNSUPPORTED) return st;
    }
    return normal_generic<float>(p, x, y, s);
  } else {
    return normal_generic<double>(p, x, y, s);
  }
}

// Coarsened modes in the order the transfer plan's chain takes them
// (restriction: its A^T order; prolongation: its A order).
int chain_modes(const TmgState* g, bool restriction, int* ks) {
  const tca_plan_s* tp = g->tp;
  const int* order = restriction ? tp->order_bwd : tp->order_fwd;
  int nk = 0;
  for (int j = 0; j < tp->d; ++j)
    if ((g->mask >> order[j]) & 1) ks[nk++] = order[j];
  return nk;
}

// Largest intermediate of a transfer chain (elements), the final output excluded.
int64_t chain_peak_elems(const TmgState* g, bool restriction) {
  int ks[kMaxModes];
  const int nk = chain_modes(g, restriction, ks);
  const int d = g->tp->d;
  int64_t dims[kMaxModes];
  for (int k = 0; k < d; ++k) dims[k] = restriction ? g->n[k] : g->nc[k];
  int64_t peak = 0;
  for (int j = 0; j + 1 < nk; ++j) {
    dims[ks[j]] = restriction ? g->nc[ks[j]] : g->n[ks[j]];
    int64_t e = 1;
    for (int k = 0; k < d; ++k) e *= dims[k];
    peak = std::max(peak, e);
  }
  return peak;
}

// out = P^T in (restriction, fine -> coarse) or P in (prolongation, coarse ->
// fine): one band mode product per coarsened mode, intermediates in the
// transfer plan's ping-pong buffers.
template <typename T>
tca_status transfer(const TmgState* g, bool restriction, const T* in, T* out, cudaStream_t s) {
  const tca_plan_s* tp = g->tp;
  int ks[kMaxModes];
  const int nk = chain_modes(g, restriction, ks);
  const int d = tp->d;
  int64_t dims[kMaxModes];
  for (int k = 0; k < d; ++k) dims[k] = restriction ? g->n[k] : g->nc[k];
  const T* src = in;
  for (int j = 0; j < nk; ++j) {
    const int k = ks[j];
    T* dst = (j == nk - 1) ? out : (T*)tp->ws[j & 1];
    int64_t O = 1, I = 1;
    for (int a = 0; a < k; ++a) O *= dims[a];
    for (int a = k + 1; a < d; ++a) I *= dims[a];
    const ModeOp& op = restriction ? tp->mode[k].bwd : tp->mode[k].fwd;
    TCA_TRY((launch_mode_op<T, T, T>(op, src, dst, O, I, s)));
    dims[k] = restriction ? g->nc[k] : g->n[k];
    src = dst;
  }
  return TCA_OK;
}

template <typename T>
tca_status launch_cheb(const tca_plan_s* p, const T* r, const T* t, const T* dinv, T* d, T* z, int64_t n, double cd,
                       double cr, int z_add, cudaStream_t s) {
  const int grid = tmg_grid(p, n);
  const bool vec = ((uintptr_t)r | (uintptr_t)t | (uintptr_t)dinv | (uintptr_t)d | (uintptr_t)z) % 16 == 0;
  if (vec) tmg_cheb_kernel<T, true><<<grid, kTmgThreads, 0, s>>>(r, t, dinv, d, z, n, (T)cd, (T)cr, z_add);
  else tmg_cheb_kernel<T, false><<<grid, kTmgThreads, 0, s>>>(r, t, dinv, d, z, n, (T)cd, (T)cr, z_add);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// nu Chebyshev steps for K z = r, preconditioned by D (z zero: the first step
// needs no product with K).
template <typename T>
tca_status smooth(tca_plan_s* p, const T* r, T* z, bool z_zero, cudaStream_t s) {
  TmgState* g = p->tmg;
  const int64_t N = p->N;
  T* d = (T*)g->d;
  T* t = (T*)g->t;
  const T* dinv = (const T*)p->pc_dinv;
  const double lo = g->lam_max / 30.0, hi = 1.05 * g->lam_max;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  if (z_zero) {
    TCA_TRY(launch_cheb<T>(p, r, nullptr, dinv, d, z, N, 0.0, 1.0 / theta, 0, s));
  } else {
    TCA_TRY(tmg_normal<T>(p, z, t, s));
    TCA_TRY(launch_cheb<T>(p, r, t, dinv, d, z, N, 0.0, 1.0 / theta, 1, s));
  }
  double rho = 1.0 / sigma;
  for (int i = 1; i < g->nu; ++i) {
    TCA_TRY(tmg_normal<T>(p, z, t, s));
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    TCA_TRY(launch_cheb<T>(p, r, t, dinv, d, z, N, rho_new * rho, 2.0 * rho_new / delta, 1, s));
    rho = rho_new;
  }
  return TCA_OK;
}

// x_c = K_c^-1 r_c by CG (r_c is overwritten by the coarse residual).  The
// host reads the coarse scalars after every iteration for the stop test.
template <typename T>
tca_status coarse_cg(tca_plan_s* p, cudaStream_t s) {
  TmgState* g = p->tmg;
  const int64_t Nc = g->Nc;
  const int gc = tmg_grid(p, Nc);
  const Reduce red = half_reduce(p);
  T* xc = (T*)g->xc;
  T* rc = (T*)g->rc;
  T* pc = (T*)g->pc;
  T* qc = (T*)g->qc;
  TCA_CUDA_TRY(cudaMemsetAsync(xc, 0, sizeof(T) * (size_t)Nc, s));
  tmg_cstart_kernel<T><<<gc, kTmgThreads, 0, s>>>(rc, Nc, g->sc, red);
  TCA_LAUNCH_CHECK();
  for (int it = 0;; ++it) {
    TCA_CUDA_TRY(cudaMemcpyAsync(g->sc_host, g->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    TCA_CUDA_TRY(cudaStreamSynchronize(s));
    const Scalars& h = *g->sc_host;
    // Fig. 2's test sqrt(rho) / ||b|| <= tolerance (not finite: stop as well).
    if (h.bnorm == 0.0 || h.breakdown || !(std::sqrt(h.rho) > g->coarse_rtol * h.bnorm) || it >= kMaxCoarseIters)
      break;
    tmg_cdir_kernel<T><<<gc, kTmgThreads, 0, s>>>(rc, pc, Nc, g->sc, it == 0 ? 1 : 0);
    TCA_LAUNCH_CHECK();
    TCA_TRY(transfer<T>(g, false, pc, (T*)g->u, s));
    TCA_TRY(tmg_normal<T>(p, (const T*)g->u, (T*)g->t, s));
    TCA_TRY(transfer<T>(g, true, (const T*)g->t, qc, s));
    tmg_calpha_kernel<T><<<gc, kTmgThreads, 0, s>>>(pc, qc, Nc, g->sc, red);
    TCA_LAUNCH_CHECK();
    tmg_cupdate_kernel<T><<<gc, kTmgThreads, 0, s>>>(xc, rc, pc, qc, Nc, g->sc, red);
    TCA_LAUNCH_CHECK();
    ++g->coarse_iters;
  }
  return TCA_OK;
}

// lambda_max of D^-1 K by power steps from the pseudo-random start: v = D^-1 K v / ||D^-1 K v||,
// the last norm being the estimate.  One synchronisation at the end.
template <typename T>
tca_status estimate_lambda_max(tca_plan_s* p, cudaStream_t s, double* out) {
  TmgState* g = p->tmg;
  const int64_t N = p->N;
  const int grid = tmg_grid(p, N);
  const Reduce red = half_reduce(p);
  T* v = (T*)g->d;
  T* t = (T*)g->t;
  double* nrm2 = &g->sc->aux;
  tmg_seed_kernel<T><<<grid, kTmgThreads, 0, s>>>(t, N);
  TCA_LAUNCH_CHECK();
  tmg_scaled_norm_kernel<T><<<grid, kTmgThreads, 0, s>>>(t, nullptr, v, N, nrm2, red);
  TCA_LAUNCH_CHECK();
  tmg_normalise_kernel<T><<<grid, kTmgThreads, 0, s>>>(v, N, nrm2);
  TCA_LAUNCH_CHECK();
  for (int it = 0; it < kPowerSteps; ++it) {
    TCA_TRY(tmg_normal<T>(p, v, t, s));
    tmg_scaled_norm_kernel<T><<<grid, kTmgThreads, 0, s>>>(t, (const T*)p->pc_dinv, v, N, nrm2, red);
    TCA_LAUNCH_CHECK();
    tmg_normalise_kernel<T><<<grid, kTmgThreads, 0, s>>>(v, N, nrm2);
    TCA_LAUNCH_CHECK();
  }
  TCA_CUDA_TRY(cudaMemcpyAsync(g->sc_host, g->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  const double lam = std::sqrt(g->sc_host->aux);
  if (!(lam > 0.0) || !std::isfinite(lam)) {
    set_error_message("tensor multigrid: the lambda_max estimate of D^-1 K is not positive and finite");
    return TCA_ERR_BREAKDOWN;
  }
  *out = lam;
  return TCA_OK;
}

void free_state_buffers(TmgState* g) {
  if (g->tp) tca_destroy(g->tp);
  g->tp = nullptr;
  for (void** b : {&g->d, &g->t, &g->u, &g->xc, &g->rc, &g->pc, &g->qc}) {
    cudaFree(*b);
    *b = nullptr;
  }
  cudaFree(g->sc);
  g->sc = nullptr;
  if (g->sc_host) cudaFreeHost(g->sc_host);
  g->sc_host = nullptr;
  g->lam_est = 0.0;
}

// Transfer plan and vectors for coarsening `mask`.
tca_status build_state(tca_plan_s* p, TmgState* g, int mask, cudaStream_t s) {
  free_state_buffers(g);
  g->mask = mask;
  const int d = p->d;
  std::vector<std::vector<double>> vals(d);
  std::vector<std::vector<int32_t>> col0(d);
  tca_factor f[kMaxModes] = {};
  int64_t ncs[kMaxModes];
  g->Nc = 1;
  for (int k = 0; k < d; ++k) {
    const int64_t n = p->n[k];
    const bool coarse = (mask >> k) & 1;
    const int64_t nc = coarse ? (n + 1) / 2 : n;
    g->n[k] = n;
    g->nc[k] = nc;
    ncs[k] = nc;
    g->Nc *= nc;
    vals[k].assign((size_t)n * 4, 0.0);
    col0[k].assign((size_t)n, 0);
    for (int64_t i = 0; i < n; ++i) {
      if (!coarse) {
        col0[k][i] = (int32_t)i;  // identity (never applied: kept modes are skipped)
        vals[k][i * 4] = 1.0;
      } else if (i % 2 == 0) {
        col0[k][i] = (int32_t)(i / 2);  // even fine point = coarse point i / 2
        vals[k][i * 4] = 1.0;
      } else {
        const int64_t c = i / 2;  // odd fine point: halfway between coarse points c and c + 1
        col0[k][i] = (int32_t)c;
        vals[k][i * 4] = 0.5;
        if (c + 1 < nc) vals[k][i * 4 + 1] = 0.5;
      }
    }
    f[k].kind = TCA_FACTOR_ELL4;
    f[k].m = n;
    f[k].n = nc;
    f[k].values = vals[k].data();
    f[k].col0 = col0[k].data();
  }
  const tca_reg none = {0.0, 0u, 0u};
  TCA_TRY(tca_plan(&g->tp, d, ncs, f, &none, (tca_precision)p->prec, s));
  if (chain_peak_elems(g, true) > g->tp->ws_elems || chain_peak_elems(g, false) > g->tp->ws_elems) {
    set_error_message("tensor multigrid: transfer intermediates exceed the transfer plan's workspace");
    return TCA_ERR_UNSUPPORTED;
  }
  const size_t es = elem_size(p);
  cudaError_t e = cudaSuccess;
  for (void** b : {&g->d, &g->t, &g->u})
    if (e == cudaSuccess) e = cudaMalloc(b, es * (size_t)p->N);
  for (void** b : {&g->xc, &g->rc, &g->pc, &g->qc})
    if (e == cudaSuccess) e = cudaMalloc(b, es * (size_t)g->Nc);
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->sc, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&g->sc_host, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMemsetAsync(g->sc, 0, sizeof(Scalars), s);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    free_state_buffers(g);
    return TCA_ERR_ALLOC;
  }
  return TCA_OK;
}

}  // namespace

tca_status tmg_setup(tca_plan_s* p, const tca_solve_opts* o, cudaStream_t s) {
  if (p->scattered || (p->prec != TCA_F32 && p->prec != TCA_F64)) {
    set_error_message("the tensor multigrid preconditioner takes TCA_F32 and TCA_F64 Gram-form plans");
    return TCA_ERR_UNSUPPORTED;
  }
  const double crt = o ? o->tmg_coarse_rtol : 0.0;
  const double lmax = o ? o->tmg_lambda_max : 0.0;
  if (!(crt >= 0.0) || !std::isfinite(crt) || !(lmax >= 0.0) || !std::isfinite(lmax)) return TCA_ERR_INVALID_ARG;
  int mask = o ? o->tmg_coarsen_mask : 0;
  if (mask < 0 || (mask >> p->d) != 0) return TCA_ERR_INVALID_ARG;
  if (mask == 0) {
    for (int k = 0; k < p->d; ++k)
      if (p->n[k] >= kCoarsenMin) mask |= 1 << k;
    if (mask == 0) {
      set_error_message("tensor multigrid: no mode of at least 16 points to coarsen (give tmg_coarsen_mask)");
      return TCA_ERR_UNSUPPORTED;
    }
  }
  for (int k = 0; k < p->d; ++k)
    if (((mask >> k) & 1) && p->n[k] < 2) return TCA_ERR_INVALID_ARG;
  const int nu_in = o ? o->tmg_nu : 0;
  const int nu = nu_in == 0 ? kDefaultNu : (nu_in < 0 ? 0 : nu_in);
  if (nu > kMaxNu) return TCA_ERR_INVALID_ARG;
  TCA_TRY(ensure_jacobi(p));
  if (!p->tmg) p->tmg = new TmgState();
  TmgState* g = p->tmg;
  if (!g->tp || g->mask != mask) TCA_TRY(build_state(p, g, mask, s));
  g->nu = nu;
  g->coarse_rtol = crt > 0.0 ? crt : kDefaultCoarseRtol;
  if (lmax > 0.0) {
    g->lam_max = lmax;
  } else {
    if (g->lam_est == 0.0) {
      if (p->prec == TCA_F64) TCA_TRY(estimate_lambda_max<double>(p, s, &g->lam_est));
      else TCA_TRY(estimate_lambda_max<float>(p, s, &g->lam_est));
    }
    g->lam_max = g->lam_est;
  }
  return TCA_OK;
}

template <typename T>
tca_status tmg_cycle(tca_plan_s* p, const T* r, T* z, bool skip_if_done, cudaStream_t s) {
  TmgState* g = p->tmg;
  if (!g || !g->tp) return TCA_ERR_INVALID_ARG;
  if (skip_if_done) {
    TCA_CUDA_TRY(cudaMemcpyAsync(p->scal_host, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
    TCA_CUDA_TRY(cudaStreamSynchronize(s));
    if (cg_done(p->scal_host)) return TCA_OK;
  }
  const int64_t N = p->N;
  const int grid = tmg_grid(p, N);
  bool z_zero = true;
  if (g->nu > 0) {
    TCA_TRY(smooth<T>(p, r, z, true, s));
    z_zero = false;
  }
  // Restriction of the residual (of z = 0 without smoothing: r itself).
  const T* res = r;
  if (!z_zero) {
    TCA_TRY(tmg_normal<T>(p, z, (T*)g->t, s));
    tmg_residual_kernel<T><<<grid, kTmgThreads, 0, s>>>(r, (T*)g->t, N);
    TCA_LAUNCH_CHECK();
    res = (const T*)g->t;
  }
  TCA_TRY(transfer<T>(g, true, res, (T*)g->rc, s));
  TCA_TRY(coarse_cg<T>(p, s));
  // Coarse-grid correction z += P x_c.
  TCA_TRY(transfer<T>(g, false, (const T*)g->xc, (T*)g->u, s));
  tmg_add_kernel<T><<<grid, kTmgThreads, 0, s>>>(z, (const T*)g->u, N, z_zero ? 0 : 1);
  TCA_LAUNCH_CHECK();
  if (g->nu > 0) TCA_TRY(smooth<T>(p, r, z, false, s));
  return TCA_OK;
}

template tca_status tmg_cycle<float>(tca_plan_s*, const float*, float*, bool, cudaStream_t);
template tca_status tmg_cycle<double>(tca_plan_s*, const double*, double*, bool, cudaStream_t);

void tmg_reset_count(tca_plan_s* p) {
  if (p->tmg) p->tmg->coarse_iters = 0;
}

void tmg_release(tca_plan_s* p) {
  if (!p->tmg) return;
  free_state_buffers(p->tmg);
  delete p->tmg;
  p->tmg = nullptr;
}

}  // namespace tca

using namespace tca;

extern "C" tca_status tca_tmg_apply(tca_plan_t plan, const void* r, void* z, const tca_solve_opts* opts,
                                    cudaStream_t stream) {
  if (!plan || !r || !z || r == z) return TCA_ERR_INVALID_ARG;
  tca_plan_s* p = plan;
  if (!is_device_ptr(r) || !is_device_ptr(z)) {
    set_error_message("tca_tmg_apply takes device buffers");
    return TCA_ERR_INVALID_ARG;
  }
  TCA_TRY(tmg_setup(p, opts, stream));
  tmg_reset_count(p);
  tca_status st;
  if (p->prec == TCA_F64) st = tmg_cycle<double>(p, (const double*)r, (double*)z, false, stream);
  else st = tmg_cycle<float>(p, (const float*)r, (float*)z, false, stream);
  if (st != TCA_OK) return st;
  TCA_CUDA_TRY(cudaStreamSynchronize(stream));
  return TCA_OK;
}

extern "C" tca_status tca_tmg_info(tca_plan_t plan, double* lambda_max, int64_t* coarse_iters) {
  if (!plan) return TCA_ERR_INVALID_ARG;
  const TmgState* g = plan->tmg;
  if (lambda_max) *lambda_max = g ? g->lam_max : 0.0;
  if (coarse_iters) *coarse_iters = g ? g->coarse_iters : 0;
  return TCA_OK;
}
