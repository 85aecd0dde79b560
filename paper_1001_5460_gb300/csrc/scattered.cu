// Scattered (off-grid) samples: the system tensor whose rows are Kronecker
// products of per-mode rows (the row-wise, face-splitting product of d
// ELL-4 matrices A_k, each with one row per sample).
//
// This is the structure of the paper's real 4D problem (Sec. 5: B-spline
// reconstruction from about 9M scattered measurements) and of a tensor
// multiplication with a repeated index (Sec. 2.2): sample s weights unknown
// (i_1..i_d) by prod_k A_k[s, i_k], so
//   (A x)_s   = sum over the 4^d window of s of prod_k w_k[s, a_k] x[c_1 + a_1, ..]
//   (A^T y)_i = sum over the samples whose window holds i of the same weight y_s
// and A^T A is a sum over samples of rank-1 tensor products - not separable,
// so there is no Gram shortcut: the normal operator goes through sample space
// (gather, then scatter-add) plus the separable regulariser.
//
// The samples are reordered at plan time by the first grid cell of their
// window (lexicographic, mode 1 slowest) so that neighbouring threads gather
// and scatter around the same unknowns; the caller's order is kept for the
// sample tensor at the boundary (apply, apply_T, b) through a permutation.
// FP64 data and arithmetic; the scatter adds with FP64 atomics (the order of
// the additions to one unknown varies from run to run in its last bits).
#include <algorithm>
#include <numeric>
#include <vector>

#include "tca_internal.cuh"

namespace tca {

namespace {

constexpr int kThreads = 256;

struct ScatView {
  int64_t m;
  int64_t n[4];
  const int32_t* col0;  // [k][s], window start per mode (4 taps)
  const double* w;      // [k][s][4]
  const int32_t* perm;  // sorted position -> caller's sample index (null: internal order)
};

// Flat index of tap (a0..a3) of sample s and whether it lies on the grid.
template <int D>
__device__ __forceinline__ bool tap_index(const ScatView& v, const int32_t* c, int a0, int a1, int a2, int a3,
                                          int64_t* flat) {
  const int64_t i0 = c[0] + a0, i1 = c[1] + a1, i2 = c[2] + a2, i3 = D == 4 ? c[3] + a3 : 0;
  if (i0 < 0 || i0 >= v.n[0] || i1 < 0 || i1 >= v.n[1] || i2 < 0 || i2 >= v.n[2]) return false;
  if (D == 4 && (i3 < 0 || i3 >= v.n[3])) return false;
  *flat = ((i0 * v.n[1] + i1) * v.n[2] + i2) * (D == 4 ? v.n[3] : 1) + i3;
  return true;
}

template <int D>
__global__ void __launch_bounds__(kThreads) gather_kernel(ScatView v, const double* __restrict__ x,
                                                          double* __restrict__ y) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < v.m; s += (int64_t)gridDim.x * blockDim.x) {
    int32_t c[4];
    double w[4][4];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      c[k] = v.col0[k * v.m + s];
#pragma unroll
      for (int a = 0; a < 4; ++a) w[k][a] = v.w[(k * v.m + s) * 4 + a];
    }
    double acc = 0.0;
#pragma unroll
    for (int a0 = 0; a0 < 4; ++a0)
#pragma unroll
      for (int a1 = 0; a1 < 4; ++a1)
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) {
          const double w012 = w[0][a0] * w[1][a1] * w[2][a2];
#pragma unroll
          for (int a3 = 0; a3 < (D == 4 ? 4 : 1); ++a3) {
            int64_t f;
            if (tap_index<D>(v, c, a0, a1, a2, a3, &f)) acc = fma(D == 4 ? w012 * w[3][a3] : w012, x[f], acc);
          }
        }
    y[v.perm ? v.perm[s] : s] = acc;
  }
}

template <int D>
__global__ void __launch_bounds__(kThreads) scatter_kernel(ScatView v, const double* __restrict__ y,
                                                           double* __restrict__ x) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < v.m; s += (int64_t)gridDim.x * blockDim.x) {
    const double ys = y[v.perm ? v.perm[s] : s];
    int32_t c[4];
    double w[4][4];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      c[k] = v.col0[k * v.m + s];
#pragma unroll
      for (int a = 0; a < 4; ++a) w[k][a] = v.w[(k * v.m + s) * 4 + a];
    }
#pragma unroll
    for (int a0 = 0; a0 < 4; ++a0)
#pragma unroll
      for (int a1 = 0; a1 < 4; ++a1)
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) {
          const double w012 = w[0][a0] * w[1][a1] * w[2][a2] * ys;
#pragma unroll
          for (int a3 = 0; a3 < (D == 4 ? 4 : 1); ++a3) {
            int64_t f;
            const double wt = D == 4 ? w012 * w[3][a3] : w012;
            if (wt != 0.0 && tap_index<D>(v, c, a0, a1, a2, a3, &f)) atomicAdd(x + f, wt);
          }
        }
  }
}

ScatView view_of(const tca_plan_s* p, bool perm) {
  ScatView v;
  v.m = p->sc_m;
  for (int k = 0; k < 4; ++k) v.n[k] = k < p->d ? p->n[k] : 1;
  v.col0 = p->sc_col0;
  v.w = p->sc_w;
  v.perm = perm ? p->sc_perm : nullptr;
  return v;
}

int grid_of(const tca_plan_s* p) {
  const int64_t want = (p->sc_m + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)p->num_sms * 16));
}

}  // namespace

tca_status scattered_gather(const tca_plan_s* p, const double* x, double* y, bool perm, cudaStream_t s) {
  if (p->sc_m == 0) return TCA_OK;
  const ScatView v = view_of(p, perm);
  if (p->d == 4) gather_kernel<4><<<grid_of(p), kThreads, 0, s>>>(v, x, y);
  else gather_kernel<3><<<grid_of(p), kThreads, 0, s>>>(v, x, y);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

tca_status scattered_scatter(const tca_plan_s* p, const double* y, double* x, bool perm, cudaStream_t s) {
  TCA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)p->N, s));
  if (p->sc_m == 0) return TCA_OK;
  const ScatView v = view_of(p, perm);
  if (p->d == 4) scatter_kernel<4><<<grid_of(p), kThreads, 0, s>>>(v, y, x);
  else scatter_kernel<3><<<grid_of(p), kThreads, 0, s>>>(v, y, x);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// Attach the scattered rows to a plan built over the grid (with identity
// per-mode factors, which give it the regulariser bands and workspace):
// validate, sort the samples by the first cell of their window, upload.
tca_status scattered_attach(tca_plan_s* p, int64_t m, const tca_factor* rows) {
  const int d = p->d;
  for (int k = 0; k < d; ++k) {
    if (rows[k].kind != TCA_FACTOR_ELL4 || !rows[k].col0 || !rows[k].values || rows[k].reserved != 0)
      return TCA_ERR_INVALID_ARG;
    if (rows[k].m != m || rows[k].n != p->n[k]) return TCA_ERR_SHAPE;
  }
  if (m > INT32_MAX) return TCA_ERR_UNSUPPORTED;
  std::vector<int64_t> order((size_t)m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    for (int k = 0; k < d; ++k) {
      const int32_t ca = rows[k].col0[a], cb = rows[k].col0[b];
      if (ca != cb) return ca < cb;
    }
    return false;
  });
  std::vector<int32_t> c0((size_t)d * m), perm((size_t)m);
  std::vector<double> w((size_t)d * m * 4);
  for (int64_t s = 0; s < m; ++s) {
    const int64_t src = order[(size_t)s];
    perm[(size_t)s] = (int32_t)src;
    for (int k = 0; k < d; ++k) {
      c0[(size_t)(k * m + s)] = rows[k].col0[src];
      for (int a = 0; a < 4; ++a) w[(size_t)((k * m + s) * 4 + a)] = rows[k].values[src * 4 + a];
    }
  }
  p->sc_m = m;
  cudaError_t e = cudaSuccess;
  if (m > 0) {
    e = cudaMalloc((void**)&p->sc_col0, sizeof(int32_t) * c0.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->sc_w, sizeof(double) * w.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->sc_perm, sizeof(int32_t) * perm.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->sc_tmp, sizeof(double) * (size_t)m);
    if (e == cudaSuccess) e = cudaMemcpy(p->sc_col0, c0.data(), sizeof(int32_t) * c0.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->sc_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->sc_perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  p->scattered = true;
  p->M = m;
  return TCA_OK;
}

void scattered_release(tca_plan_s* p) {
  cudaFree(p->sc_col0);
  cudaFree(p->sc_w);
  cudaFree(p->sc_perm);
  cudaFree(p->sc_tmp);
  p->sc_col0 = nullptr;
  p->sc_w = nullptr;
  p->sc_perm = nullptr;
  p->sc_tmp = nullptr;
}

}  // namespace tca

using namespace tca;

extern "C" tca_status tca_plan_scattered(tca_plan_t* out, int order, const int64_t* n, int64_t m,
                                         const tca_factor* rows, const tca_reg* reg, tca_precision prec,
                                         cudaStream_t stream) {
  if (!out || !n || !rows || m < 0) return TCA_ERR_INVALID_ARG;
  *out = nullptr;
  if (order != 3 && order != 4) return TCA_ERR_INVALID_ARG;
  if (prec != TCA_F64) {
    set_error_message("scattered plans compute in FP64 (TCA_F64)");
    return TCA_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < order; ++k)
    if (n[k] <= 0 || n[k] > (1 << 24)) return TCA_ERR_INVALID_ARG;
  // The grid plan: identity ELL-4 factors give it the regulariser bands and
  // the workspace; its Gram factors are never used.
  std::vector<std::vector<double>> vals(order);
  std::vector<std::vector<int32_t>> cols(order);
  std::vector<tca_factor> ident(order);
  for (int k = 0; k < order; ++k) {
    vals[k].assign((size_t)n[k] * 4, 0.0);
    cols[k].resize((size_t)n[k]);
    for (int64_t i = 0; i < n[k]; ++i) {
      vals[k][(size_t)i * 4] = 1.0;
      cols[k][(size_t)i] = (int32_t)i;
    }
    ident[k] = tca_factor{TCA_FACTOR_ELL4, 0, n[k], n[k], vals[k].data(), cols[k].data()};
  }
  tca_plan_t p = nullptr;
  TCA_TRY(tca_plan(&p, order, n, ident.data(), reg, prec, stream));
  const tca_status st = scattered_attach(p, m, rows);
  if (st != TCA_OK) {
    tca_destroy(p);
    return st;
  }
  *out = p;
  return TCA_OK;
}
