// Plan construction and lifetime: factor ingest, Gram and regulariser bands,
// mode ordering, workspace.  Implements tca_plan / tca_destroy and the small
// status helpers of tca.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tca_internal.cuh"

namespace tca {

static thread_local char g_last_error[256] = "";
static thread_local uint64_t g_launches = 0;

void set_cuda_error(cudaError_t e) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}
void set_error_message(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
void note_launches(uint64_t count) { g_launches += count; }

int vector_grid(const tca_plan_s* p, int64_t n) {
  const int64_t want = (n + 1023) / 1024;  // ~4 float4 per thread at 256 threads
  const int64_t cap = (int64_t)p->num_sms * 8;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

// ---- Gram formation G = A^T A in FP64 (plan step; App. "Tensor transposition")

// Banded Gram of an ELL4 factor.  One thread per (column i, offset e): entry
// G[i][i-3+e] = sum over rows r touching both columns of A[r][i] A[r][i-3+e],
// rows taken in ascending order so that G[i][c] and G[c][i] are bit-identical.
__global__ void gram_ell4_kernel(const int32_t* __restrict__ col0, const double* __restrict__ w,
                                 const int32_t* __restrict__ tstart, const int32_t* __restrict__ tcount,
                                 int64_t n, double* __restrict__ g64, float* __restrict__ g32) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 7) return;
  const int64_t i = t / 7;
  const int e = (int)(t % 7);
  const int64_t c = i - kGramHalf + e;
  double s = 0.0;
  if (c >= 0 && c < n) {
    const int64_t r0 = tstart[i], r1 = r0 + tcount[i];
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t oi = i - col0[r], oc = c - col0[r];
      if (oc >= 0 && oc < 4) s += w[r * 4 + oi] * w[r * 4 + oc];
    }
  }
  g64[t] = s;
  g32[t] = (float)s;
}

// Dense Gram G[i][c] = sum_r A[r][i] A[r][c] (ascending r; exactly symmetric).
__global__ void gram_dense_kernel(const double* __restrict__ a, int64_t m, int64_t n,
                                  double* __restrict__ g64, float* __restrict__ g32) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int64_t i = t / n, c = t % n;
  double s = 0.0;
  for (int64_t r = 0; r < m; ++r) s += a[r * n + i] * a[r * n + c];
  g64[t] = s;
  g32[t] = (float)s;
}

// lambda * (D2^T D2) as a 5-band: entry [i][e] couples i with c = i-2+e;
// (D2^T D2)[i][c] = sum_r D2[r][i] D2[r][c], D2[r][r..r+2] = (1, -2, 1).
__global__ void lap_band_kernel(int64_t n, double lam, double* __restrict__ l64, float* __restrict__ l32,
                                int32_t* __restrict__ start) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 5) return;
  const int64_t i = t / 5;
  const int e = (int)(t % 5);
  const int64_t c = i - kLapHalf + e;
  double s = 0.0;
  if (c >= 0 && c < n) {
    for (int64_t r = 0; r + 2 < n; ++r) {
      const int64_t di = i - r, dc = c - r;
      if (di < 0 || di > 2 || dc < 0 || dc > 2) continue;
      const double vi = di == 1 ? -2.0 : 1.0, vc = dc == 1 ? -2.0 : 1.0;
      s += vi * vc;
    }
  }
  l64[t] = lam * s;
  l32[t] = (float)(lam * s);
  if (e == 0) start[i] = (int32_t)(i - kLapHalf);
}

__global__ void cast_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

__global__ void transpose_kernel(const double* __restrict__ a, int64_t rows, int64_t cols,
                                 double* __restrict__ at64, float* __restrict__ at32) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const int64_t r = t / cols, c = t % cols;
  at64[c * rows + r] = a[t];
  at32[c * rows + r] = (float)a[t];
}

__global__ void iota_kernel(int32_t* __restrict__ s, int64_t n, int shift) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) s[t] = (int32_t)(t - shift);
}

static int nblk(int64_t n, int b = 256) { return (int)((n + b - 1) / b); }

template <typename T>
static tca_status dmalloc(T** ptr, int64_t count) {
  *ptr = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void**)ptr, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  return TCA_OK;
}

static void free_band(Band& b) {
  cudaFree(b.start);
  cudaFree(b.w32);
  cudaFree(b.w64);
  cudaFree(b.wff);
  b = Band();
}
static void free_dense(Dense& d) {
  cudaFree(d.a32);
  cudaFree(d.a64);
  cudaFree(d.aff);
  cudaFree(d.zero_start);
  d = Dense();
}

// Double-float copies of the FP64 coefficients (used by the FP64-accurate residual).
static tca_status add_ff_band(Band& b, cudaStream_t s) {
  const int64_t n = b.n_out * b.W;
  TCA_TRY(dmalloc(&b.wff, n));
  return split_ff(b.w64, b.wff, n, s);
}
static tca_status add_ff_op(ModeOp& op, cudaStream_t s) {
  if (op.kind == OP_BAND) return add_ff_band(op.band, s);
  Dense& d = op.dense;
  TCA_TRY(dmalloc(&d.aff, d.n_out * d.n_in));
  TCA_TRY(dmalloc(&d.zero_start, d.n_out));
  TCA_CUDA_TRY(cudaMemsetAsync(d.zero_start, 0, sizeof(int32_t) * d.n_out, s));
  return split_ff(d.a64, d.aff, d.n_out * d.n_in, s);
}
static void free_op(ModeOp& o) {
  free_band(o.band);
  free_dense(o.dense);
}

static tca_status ingest_mode(tca_plan_s* p, int k, const tca_factor& f, bool reg, cudaStream_t s) {
  Mode& md = p->mode[k];
  md.n = f.n;
  md.m = f.m;
  md.factor_kind = f.kind;
  const int64_t m = f.m, n = f.n;
  if (f.kind == TCA_FACTOR_ELL4) {
    // Forward band: row r reads columns col0[r] .. col0[r]+3.
    std::vector<double> w((size_t)m * 4);
    std::vector<int32_t> c0(f.col0, f.col0 + m);
    for (int64_t r = 0; r < m; ++r) {
      if (r > 0 && c0[r] < c0[r - 1]) return TCA_ERR_INVALID_ARG;  // must be non-decreasing
    }
    for (int64_t r = 0; r < m; ++r) {
      // A row whose window starts at or below -4, or at or past n, has no column in
      // the grid: clamping its start to [-4, n] keeps the order and every index
      // the kernels form from it small.
      c0[r] = (int32_t)std::min<int64_t>(std::max<int64_t>(c0[r], -4), n);
      for (int c = 0; c < 4; ++c) {
        const int64_t col = (int64_t)c0[r] + c;
        w[r * 4 + c] = (col >= 0 && col < n) ? f.values[r * 4 + c] : 0.0;
      }
    }
    Band& fb = md.fwd.band;
    md.fwd.kind = OP_BAND;
    fb.n_out = m;
    fb.n_in = n;
    fb.W = 4;
    fb.rows32 = rows_per_chunk(c0.data(), m, 4);
    TCA_TRY(dmalloc(&fb.start, m));
    TCA_TRY(dmalloc(&fb.w64, m * 4));
    TCA_TRY(dmalloc(&fb.w32, m * 4));
    TCA_CUDA_TRY(cudaMemcpyAsync(fb.start, c0.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    TCA_CUDA_TRY(cudaMemcpyAsync(fb.w64, w.data(), sizeof(double) * m * 4, cudaMemcpyHostToDevice, s));
    cast_kernel<<<nblk(m * 4), 256, 0, s>>>(fb.w64, fb.w32, m * 4);
    TCA_LAUNCH_CHECK();

    // Transposed band: column i is touched by the contiguous rows jlo..jhi
    // (col0 non-decreasing), so A^T is again a band in gather form.
    std::vector<int32_t> ts((size_t)n), tc((size_t)n);
    int W = 1;
    {
      int64_t lo = 0;
      for (int64_t i = 0; i < n; ++i) {
        while (lo < m && (int64_t)c0[lo] + 3 < i) ++lo;
        int64_t hi = lo;
        while (hi < m && (int64_t)c0[hi] <= i) ++hi;
        ts[i] = (int32_t)lo;
        tc[i] = (int32_t)std::max<int64_t>(0, hi - lo);
        W = std::max<int>(W, tc[i]);
      }
    }
    if (W > kMaxBandW) return TCA_ERR_UNSUPPORTED;
    std::vector<double> wt((size_t)n * W, 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int e = 0; e < tc[i]; ++e) {
        const int64_t r = ts[i] + e;
        const int64_t off = i - c0[r];
        if (off >= 0 && off < 4) wt[i * W + e] = w[r * 4 + off];
      }
    Band& bb = md.bwd.band;
    md.bwd.kind = OP_BAND;
    bb.n_out = n;
    bb.n_in = m;
    bb.W = W;
    bb.rows32 = rows_per_chunk(ts.data(), n, W);
    TCA_TRY(dmalloc(&bb.start, n));
    TCA_TRY(dmalloc(&bb.w64, n * W));
    TCA_TRY(dmalloc(&bb.w32, n * W));
    TCA_CUDA_TRY(cudaMemcpyAsync(bb.start, ts.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    bb.start_host.assign(ts.begin(), ts.end());
    TCA_CUDA_TRY(cudaMemcpyAsync(bb.w64, wt.data(), sizeof(double) * n * W, cudaMemcpyHostToDevice, s));
    cast_kernel<<<nblk(n * W), 256, 0, s>>>(bb.w64, bb.w32, n * W);
    TCA_LAUNCH_CHECK();

    // Gram band on the device (FP64).
    int32_t* dcount = nullptr;
    TCA_TRY(dmalloc(&dcount, n));
    TCA_CUDA_TRY(cudaMemcpyAsync(dcount, tc.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    Band& gb = md.gram.band;
    md.gram.kind = OP_BAND;
    gb.n_out = n;
    gb.n_in = n;
    gb.W = 2 * kGramHalf + 1;
    gb.rows32 = (int)std::min<int64_t>(n, 32) - 1 + gb.W;
    gb.unit = true;
    TCA_TRY(dmalloc(&gb.start, n));
    TCA_TRY(dmalloc(&gb.w64, n * 7));
    TCA_TRY(dmalloc(&gb.w32, n * 7));
    iota_kernel<<<nblk(n), 256, 0, s>>>(gb.start, n, kGramHalf);
    TCA_LAUNCH_CHECK();
    gram_ell4_kernel<<<nblk(n * 7), 256, 0, s>>>(fb.start, fb.w64, bb.start, dcount, n, gb.w64, gb.w32);
    TCA_LAUNCH_CHECK();
    TCA_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(dcount);
  } else if (f.kind == TCA_FACTOR_DENSE) {
    Dense& fd = md.fwd.dense;
    md.fwd.kind = OP_DENSE;
    fd.n_out = m;
    fd.n_in = n;
    TCA_TRY(dmalloc(&fd.a64, m * n));
    TCA_TRY(dmalloc(&fd.a32, m * n));
    TCA_CUDA_TRY(cudaMemcpyAsync(fd.a64, f.values, sizeof(double) * m * n, cudaMemcpyHostToDevice, s));
    cast_kernel<<<nblk(m * n), 256, 0, s>>>(fd.a64, fd.a32, m * n);
    TCA_LAUNCH_CHECK();
    Dense& bd = md.bwd.dense;
    md.bwd.kind = OP_DENSE;
    bd.n_out = n;
    bd.n_in = m;
    TCA_TRY(dmalloc(&bd.a64, m * n));
    TCA_TRY(dmalloc(&bd.a32, m * n));
    transpose_kernel<<<nblk(m * n), 256, 0, s>>>(fd.a64, m, n, bd.a64, bd.a32);
    TCA_LAUNCH_CHECK();
    Dense& gd = md.gram.dense;
    md.gram.kind = OP_DENSE;
    gd.n_out = n;
    gd.n_in = n;
    TCA_TRY(dmalloc(&gd.a64, n * n));
    TCA_TRY(dmalloc(&gd.a32, n * n));
    gram_dense_kernel<<<nblk(n * n), 256, 0, s>>>(fd.a64, m, n, gd.a64, gd.a32);
    TCA_LAUNCH_CHECK();
    // FP32 plans run dense products on the tensor cores with the 3xTF32 split
    // (about FP32 accuracy); reduced-precision plans use plain TF32.
    const int split = p->prec == TCA_F32 ? 2 : (p->prec == TCA_F64 ? 0 : 1);
    md.fwd.tc_split = md.bwd.tc_split = md.gram.tc_split = split;
  } else {
    return TCA_ERR_INVALID_ARG;
  }
  // Regulariser band (zeros when the mode is not regularised).
  md.reg = reg && n >= 3;
  Band& lb = md.lap;
  lb.n_out = n;
  lb.n_in = n;
  lb.W = 2 * kLapHalf + 1;
  lb.rows32 = (int)std::min<int64_t>(n, 32) - 1 + lb.W;
  lb.unit = true;
  TCA_TRY(dmalloc(&lb.start, n));
  TCA_TRY(dmalloc(&lb.w64, n * 5));
  TCA_TRY(dmalloc(&lb.w32, n * 5));
  lap_band_kernel<<<nblk(n * 5), 256, 0, s>>>(n, md.reg ? p->lambda : 0.0, lb.w64, lb.w32, lb.start);
  TCA_LAUNCH_CHECK();
  TCA_TRY(add_ff_op(md.fwd, s));
  TCA_TRY(add_ff_op(md.bwd, s));
  TCA_TRY(add_ff_op(md.gram, s));
  TCA_TRY(add_ff_band(lb, s));
  return TCA_OK;
}

// ---- Separable-inverse preconditioner (a tensor inverse, Sec. 3, Eq. TensorEq)
//
// M_k = G_k + s (lambda L_k) in FP64 on the host from the plan's FP64 Gram and
// regulariser bands, inverted through its Cholesky factor C (M_k^-1 =
// C^-T C^-1), stored as a dense factor.

// In-place inverse of the SPD n x n matrix a (row-major); false if a pivot is
// not positive.
static bool spd_inverse(std::vector<double>& a, int64_t n) {
  std::vector<double> c((size_t)(n * n), 0.0);
  for (int64_t j = 0; j < n; ++j) {
    double d = a[j * n + j];
    for (int64_t t = 0; t < j; ++t) d -= c[j * n + t] * c[j * n + t];
    if (!(d > 0.0)) return false;
    const double cjj = std::sqrt(d);
    c[j * n + j] = cjj;
    for (int64_t i = j + 1; i < n; ++i) {
      double v = a[i * n + j];
      for (int64_t t = 0; t < j; ++t) v -= c[i * n + t] * c[j * n + t];
      c[i * n + j] = v / cjj;
    }
  }
  // w = C^-1 (lower triangular), by forward substitution column by column.
  std::vector<double> w((size_t)(n * n), 0.0);
  for (int64_t col = 0; col < n; ++col) {
    for (int64_t i = col; i < n; ++i) {
      double v = i == col ? 1.0 : 0.0;
      for (int64_t t = col; t < i; ++t) v -= c[i * n + t] * w[t * n + col];
      w[i * n + col] = v / c[i * n + i];
    }
  }
  // a = W^T W.
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j <= i; ++j) {
      double v = 0.0;
      for (int64_t t = i; t < n; ++t) v += w[t * n + i] * w[t * n + j];
      a[i * n + j] = v;
      a[j * n + i] = v;
    }
  return true;
}

// G_k and lambda L_k of mode k as dense n x n FP64 matrices on the host, from
// the plan's FP64 Gram and regulariser bands.
static tca_status mode_dense_host(const tca_plan_s* p, int k, std::vector<double>& a, std::vector<double>& lap) {
  const Mode& md = p->mode[k];
  const int64_t n = md.n;
  a.assign((size_t)(n * n), 0.0);
  lap.assign((size_t)(n * n), 0.0);
  if (md.gram.kind == OP_DENSE) {
    TCA_CUDA_TRY(cudaMemcpy(a.data(), md.gram.dense.a64, sizeof(double) * n * n, cudaMemcpyDeviceToHost));
  } else {
    const Band& gb = md.gram.band;
    std::vector<double> g((size_t)(n * gb.W));
    std::vector<int32_t> st((size_t)n);
    TCA_CUDA_TRY(cudaMemcpy(g.data(), gb.w64, sizeof(double) * n * gb.W, cudaMemcpyDeviceToHost));
    TCA_CUDA_TRY(cudaMemcpy(st.data(), gb.start, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i)
      for (int e = 0; e < gb.W; ++e) {
        const int64_t c = (int64_t)st[i] + e;
        if (c >= 0 && c < n) a[i * n + c] += g[i * gb.W + e];
      }
  }
  const Band& lb = md.lap;
  std::vector<double> l((size_t)(n * lb.W));
  TCA_CUDA_TRY(cudaMemcpy(l.data(), lb.w64, sizeof(double) * n * lb.W, cudaMemcpyDeviceToHost));
  const int half = lb.W / 2;
  for (int64_t i = 0; i < n; ++i)
    for (int e = 0; e < lb.W; ++e) {
      const int64_t c = i - half + e;
      if (c >= 0 && c < n) lap[i * n + c] += l[i * lb.W + e];
    }
  return TCA_OK;
}

// Smallest and largest eigenvalue of the symmetric n x n matrix a (destroyed):
// cyclic Jacobi rotations until the off-diagonal mass is below 1e-24 of the
// total (or 60 sweeps).
static void sym_eig_extremes(std::vector<double>& a, int64_t n, double* lo, double* hi) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        const double v = a[i * n + j] * a[i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (!(off > 1e-24 * tot)) break;
    for (int64_t pp = 0; pp < n; ++pp)
      for (int64_t q = pp + 1; q < n; ++q) {
        const double apq = a[pp * n + q];
        if (apq == 0.0) continue;
        const double theta = (a[q * n + q] - a[pp * n + pp]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int64_t k = 0; k < n; ++k) {  // columns pp, q
          const double akp = a[k * n + pp], akq = a[k * n + q];
          a[k * n + pp] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; ++k) {  // rows pp, q
          const double apk = a[pp * n + k], aqk = a[q * n + k];
          a[pp * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  *lo = *hi = a[0];
  for (int64_t i = 1; i < n; ++i) {
    *lo = std::min(*lo, a[i * n + i]);
    *hi = std::max(*hi, a[i * n + i]);
  }
}

// Corner model of the spectrum of M^-1 K for M = (x)_k (G_k + s lambda L_k):
// mode k at its smooth corner (g_max, 0) or its rough corner
// (g_min, lambda l_max); at a corner K is modelled by prod g + sum l and M by
// prod (g + s l); s on the grid 2^(j/2), j = 0 .. 16, minimises the spread
// max / min of K / M over the 2^d corners (the first grid point of the
// minimum).  Modes longer than 512 are not modelled: the default shift 16.
constexpr double kFallbackShift = 16.0;
tca_status precond_model_shift(tca_plan_s* p, double* shift) {
  if (p->pc_model_shift > 0.0) {
    *shift = p->pc_model_shift;
    return TCA_OK;
  }
  const int d = p->d;
  double gs[kMaxModes][2], ls[kMaxModes][2];
  bool ok = true;
  for (int k = 0; k < d && ok; ++k) {
    const int64_t n = p->mode[k].n;
    if (n > 512) {
      ok = false;
      break;
    }
    std::vector<double> a, lap;
    TCA_TRY(mode_dense_host(p, k, a, lap));
    double gmin, gmax, lmin, lmax;
    sym_eig_extremes(a, n, &gmin, &gmax);
    sym_eig_extremes(lap, n, &lmin, &lmax);
    gs[k][0] = gmax;
    ls[k][0] = 0.0;
    gs[k][1] = std::max(gmin, 0.0);
    ls[k][1] = std::max(lmax, 0.0);
  }
  double best = kFallbackShift;
  if (ok) {
    double best_spread = -1.0;
    for (int j = 0; j <= 16; ++j) {
      const double s = std::pow(2.0, j / 2.0);
      double rmin = 0.0, rmax = 0.0;
      bool any = false;
      for (int c = 0; c < (1 << d); ++c) {
        double prod_g = 1.0, sum_l = 0.0, m = 1.0;
        for (int k = 0; k < d; ++k) {
          const int side = (c >> k) & 1;
          prod_g *= gs[k][side];
          sum_l += ls[k][side];
          m *= gs[k][side] + s * ls[k][side];
        }
        if (!(m > 0.0)) continue;
        const double r = (prod_g + sum_l) / m;
        if (!any || r < rmin) rmin = r;
        if (!any || r > rmax) rmax = r;
        any = true;
      }
      if (!any || !(rmin > 0.0)) continue;
      const double spread = rmax / rmin;
      if (best_spread < 0.0 || spread < best_spread) {
        best_spread = spread;
        best = s;
      }
    }
  }
  p->pc_model_shift = best;
  *shift = best;
  return TCA_OK;
}

// M_k = G_k + s (lambda L_k), dense n x n in FP64 on the host, inverted in place.
static tca_status precond_inverse_host(const tca_plan_s* p, int k, double shift, std::vector<double>& a) {
  {
    const Mode& md = p->mode[k];
    const int64_t n = md.n;
    a.assign((size_t)(n * n), 0.0);
    if (md.gram.kind == OP_DENSE) {
      TCA_CUDA_TRY(cudaMemcpy(a.data(), md.gram.dense.a64, sizeof(double) * n * n, cudaMemcpyDeviceToHost));
    } else {
      const Band& gb = md.gram.band;
      std::vector<double> g((size_t)(n * gb.W));
      std::vector<int32_t> st((size_t)n);
      TCA_CUDA_TRY(cudaMemcpy(g.data(), gb.w64, sizeof(double) * n * gb.W, cudaMemcpyDeviceToHost));
      TCA_CUDA_TRY(cudaMemcpy(st.data(), gb.start, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < n; ++i)
        for (int e = 0; e < gb.W; ++e) {
          const int64_t c = (int64_t)st[i] + e;
          if (c >= 0 && c < n) a[i * n + c] += g[i * gb.W + e];
        }
    }
    {
      const Band& lb = md.lap;
      std::vector<double> l((size_t)(n * lb.W));
      TCA_CUDA_TRY(cudaMemcpy(l.data(), lb.w64, sizeof(double) * n * lb.W, cudaMemcpyDeviceToHost));
      const int half = lb.W / 2;
      for (int64_t i = 0; i < n; ++i)
        for (int e = 0; e < lb.W; ++e) {
          const int64_t c = i - half + e;
          if (c >= 0 && c < n) a[i * n + c] += shift * l[i * lb.W + e];
        }
    }
    if (!spd_inverse(a, n)) {
      set_error_message("separable preconditioner: G_k + s lambda L_k is not positive definite");
      return TCA_ERR_UNSUPPORTED;
    }
  }
  return TCA_OK;
}

// Drop a cached iteration graph (it holds the old preconditioner's addresses).
static tca_status drop_graph(tca_plan_s* p) {
  TCA_CUDA_TRY(cudaDeviceSynchronize());
  if (p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  ++p->pc_generation;
  return TCA_OK;
}

static tca_status ensure_z(tca_plan_s* p) {
  if (p->z) return TCA_OK;
  cudaError_t e = cudaMalloc(&p->z, elem_size(p) * (size_t)p->N);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  return TCA_OK;
}

tca_status ensure_precond(tca_plan_s* p, double shift) {
  if (!(shift >= 0.0) || !std::isfinite(shift)) return TCA_ERR_INVALID_ARG;
  if (p->pc_shift == shift && p->z) return TCA_OK;
  TCA_TRY(drop_graph(p));
  for (int k = 0; k < kMaxModes; ++k) free_op(p->pc[k]);
  p->pc_shift = 0.0;
  for (int k = 0; k < p->d; ++k) {
    const int64_t n = p->mode[k].n;
    std::vector<double> a;
    TCA_TRY(precond_inverse_host(p, k, shift, a));
    ModeOp& op = p->pc[k];
    op.kind = OP_DENSE;
    op.dense.n_out = n;
    op.dense.n_in = n;
    TCA_TRY(dmalloc(&op.dense.a64, n * n));
    TCA_TRY(dmalloc(&op.dense.a32, n * n));
    TCA_CUDA_TRY(cudaMemcpy(op.dense.a64, a.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice));
    cast_kernel<<<nblk(n * n), 256>>>(op.dense.a64, op.dense.a32, n * n);
    TCA_LAUNCH_CHECK();
    // FP32 plans: 3xTF32 where the tiles fit, plain TF32 otherwise (a
    // preconditioner needs no more); reduced-precision plans TF32; FP64 native.
    const int split = dense_tc_max_split(n, n);
    op.tc_split = p->prec == TCA_F64 ? 0 : (p->prec == TCA_F32 ? split : std::min(split, 1));
    op.stop = p->scal;  // products after the stop flags are set skip their work
  }
  TCA_TRY(ensure_z(p));
  TCA_CUDA_TRY(cudaDeviceSynchronize());
  p->pc_shift = shift;
  return TCA_OK;
}

// Banded separable preconditioner: each (G_k + s lambda L_k)^-1 keeps its
// entries with |i - j| <= 3 (the inverses of these banded SPD matrices decay
// away from the diagonal), checked positive definite, stored as a 7-band in
// the Gram band's layout.  M^-1 = B_1 kron .. kron B_d then has exactly the
// structure of the fused sweep with zero regulariser bands.
tca_status ensure_precond_banded(tca_plan_s* p, double shift) {
  if (!(shift >= 0.0) || !std::isfinite(shift)) return TCA_ERR_INVALID_ARG;
  if (p->pcb_shift == shift && p->z) return TCA_OK;
  TCA_TRY(drop_graph(p));
  for (int k = 0; k < kMaxModes; ++k) free_op(p->pcb[k]);
  cudaFree(p->pcb_zero);
  p->pcb_zero = nullptr;
  p->pcb_fused = FusedBands();
  p->pcb_shift = 0.0;
  int64_t nmax = 1;
  for (int k = 0; k < p->d; ++k) nmax = std::max(nmax, p->n[k]);
  TCA_TRY(dmalloc(&p->pcb_zero, nmax * 5));
  TCA_CUDA_TRY(cudaMemset(p->pcb_zero, 0, sizeof(float) * (size_t)(nmax * 5)));
  for (int k = 0; k < p->d; ++k) {
    const int64_t n = p->n[k];
    std::vector<double> a;
    TCA_TRY(precond_inverse_host(p, k, shift, a));
    std::vector<double> band((size_t)(n * 7), 0.0), trunc((size_t)(n * n), 0.0);
    std::vector<float> band32((size_t)(n * 7));
    std::vector<int32_t> start((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      start[(size_t)i] = (int32_t)(i - kGramHalf);
      for (int e = 0; e < 7; ++e) {
        const int64_t j = i - kGramHalf + e;
        if (j < 0 || j >= n) continue;
        const double v = 0.5 * (a[i * n + j] + a[j * n + i]);  // symmetric by construction
        band[(size_t)(i * 7 + e)] = v;
        trunc[(size_t)(i * n + j)] = v;
      }
    }
    for (size_t t = 0; t < band.size(); ++t) band32[t] = (float)band[t];
    if (!spd_inverse(trunc, n)) {
      set_error_message("banded separable preconditioner: a truncated inverse is not positive definite");
      return TCA_ERR_UNSUPPORTED;
    }
    ModeOp& op = p->pcb[k];
    op.kind = OP_BAND;
    Band& b = op.band;
    b.n_out = n;
    b.n_in = n;
    b.W = 7;
    b.rows32 = (int)std::min<int64_t>(n, 32) - 1 + b.W;
    b.unit = true;
    TCA_TRY(dmalloc(&b.start, n));
    TCA_TRY(dmalloc(&b.w64, n * 7));
    TCA_TRY(dmalloc(&b.w32, n * 7));
    TCA_CUDA_TRY(cudaMemcpy(b.start, start.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    TCA_CUDA_TRY(cudaMemcpy(b.w64, band.data(), sizeof(double) * n * 7, cudaMemcpyHostToDevice));
    TCA_CUDA_TRY(cudaMemcpy(b.w32, band32.data(), sizeof(float) * n * 7, cudaMemcpyHostToDevice));
    p->pcb_fused.g[k] = b.w32;
    p->pcb_fused.l[k] = p->pcb_zero;
    if (k == 3 && n == 8)
      for (int t = 0; t < 8 * 7; ++t) p->pcb_fused.g4[t] = band32[(size_t)t];
  }
  TCA_TRY(ensure_z(p));
  TCA_CUDA_TRY(cudaDeviceSynchronize());
  p->pcb_shift = shift;
  return TCA_OK;
}

// ---- Point-Jacobi preconditioner (Fig. 1 solver family): M = diag(K) ----
//
// diag(K)[i_1..i_d] = prod_k G_k[i_k][i_k] + sum_k lambda L_k[i_k][i_k]: the
// diagonal of a Kronecker product is the product of the factors' diagonals,
// and each regulariser term adds its own mode's diagonal.  The per-mode
// diagonals come from the plan's FP64 bands; one kernel writes 1 / diag(K).

__global__ void jacobi_dinv_kernel(const double* __restrict__ gd, const double* __restrict__ ld, int d, int64_t n0,
                                   int64_t n1, int64_t n2, int64_t n3, float* __restrict__ out32,
                                   double* __restrict__ out64, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n[4] = {n0, n1, n2, n3};
    int64_t idx[4] = {0, 0, 0, 0};
    int64_t rem = i;
    for (int k = d - 1; k >= 0; --k) {
      idx[k] = rem % n[k];
      rem /= n[k];
    }
    double g = 1.0, l = 0.0;
    int64_t off = 0;
    for (int k = 0; k < d; ++k) {
      g *= gd[off + idx[k]];
      l += ld[off + idx[k]];
      off += n[k];
    }
    const double v = 1.0 / (g + l);
    if (out32) out32[i] = (float)v;
    if (out64) out64[i] = v;
  }
}

tca_status ensure_jacobi(tca_plan_s* p) {
  if (p->pc_dinv && p->z) return TCA_OK;
  int64_t tot = 0;
  for (int k = 0; k < p->d; ++k) tot += p->n[k];
  std::vector<double> gd((size_t)tot), ld((size_t)tot);
  int64_t off = 0;
  for (int k = 0; k < p->d; ++k) {
    const Mode& md = p->mode[k];
    const int64_t n = md.n;
    if (md.gram.kind == OP_DENSE) {
      std::vector<double> a((size_t)(n * n));
      TCA_CUDA_TRY(cudaMemcpy(a.data(), md.gram.dense.a64, sizeof(double) * n * n, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < n; ++i) gd[off + i] = a[i * n + i];
    } else {
      const Band& gb = md.gram.band;
      std::vector<double> g((size_t)(n * gb.W));
      std::vector<int32_t> st((size_t)n);
      TCA_CUDA_TRY(cudaMemcpy(g.data(), gb.w64, sizeof(double) * n * gb.W, cudaMemcpyDeviceToHost));
      TCA_CUDA_TRY(cudaMemcpy(st.data(), gb.start, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < n; ++i) {
        const int64_t e = i - st[i];  // tap that couples i with itself
        gd[off + i] = (e >= 0 && e < gb.W) ? g[i * gb.W + e] : 0.0;
      }
    }
    const Band& lb = md.lap;
    std::vector<double> l((size_t)(n * lb.W));
    TCA_CUDA_TRY(cudaMemcpy(l.data(), lb.w64, sizeof(double) * n * lb.W, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) ld[off + i] = l[i * lb.W + lb.W / 2];
    off += n;
  }
  for (int64_t i = 0; i < tot; ++i) {
    if (!(gd[i] >= 0.0)) {
      set_error_message("Jacobi preconditioner: a Gram diagonal entry is negative or not finite");
      return TCA_ERR_UNSUPPORTED;
    }
  }
  double *dg = nullptr, *dl = nullptr;
  tca_status st = dmalloc(&dg, tot);
  if (st == TCA_OK) st = dmalloc(&dl, tot);
  if (st != TCA_OK) {
    cudaFree(dg);
    return st;
  }
  cudaError_t e = cudaMemcpy(dg, gd.data(), sizeof(double) * tot, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dl, ld.data(), sizeof(double) * tot, cudaMemcpyHostToDevice);
  const size_t es = elem_size(p);
  if (e == cudaSuccess && !p->pc_dinv) e = cudaMalloc(&p->pc_dinv, es * (size_t)p->N);
  if (e == cudaSuccess && !p->z) e = cudaMalloc(&p->z, es * (size_t)p->N);
  if (e == cudaSuccess) {
    jacobi_dinv_kernel<<<std::min(nblk(p->N), 4096), 256>>>(dg, dl, p->d, p->n[0], p->n[1], p->n[2], p->n[3],
                                            es == 4 ? (float*)p->pc_dinv : nullptr,
                                            es == 8 ? (double*)p->pc_dinv : nullptr, p->N);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    st = TCA_ERR_CUDA;
  }
  cudaFree(dg);
  cudaFree(dl);
  return st;
}

// Largest intermediate of a chain of mode products applied in `order`.
static int64_t chain_peak(const int64_t* start, const int64_t* end, const int* order, int d) {
  int64_t cur[kMaxModes];
  for (int k = 0; k < d; ++k) cur[k] = start[k];
  int64_t peak = 0;
  for (int s = 0; s < d; ++s) {
    cur[order[s]] = end[order[s]];
    int64_t sz = 1;
    for (int k = 0; k < d; ++k) sz *= cur[k];
    if (s + 1 < d) peak = std::max(peak, sz);
  }
  return peak;
}

static void destroy_plan(tca_plan_s* p) {
  if (!p) return;
  for (int k = 0; k < kMaxModes; ++k) free_op(p->pc[k]);
  for (int k = 0; k < kMaxModes; ++k) free_op(p->pcb[k]);
  cudaFree(p->pcb_zero);
  cudaFree(p->z);
  cudaFree(p->pc_dinv);
  for (int k = 0; k < kMaxModes; ++k) {
    free_op(p->mode[k].fwd);
    free_op(p->mode[k].bwd);
    free_op(p->mode[k].gram);
    free_band(p->mode[k].lap);
  }
  cudaFree(p->ws[0]);
  cudaFree(p->ws[1]);
  cudaFree(p->ws64[0]);
  cudaFree(p->ws64[1]);
  cudaFree(p->rhs);
  cudaFree(p->r);
  for (int k = 0; k < kDirBufs; ++k) cudaFree(p->p[k]);
  cudaFree(p->q);
  cudaFree(p->rhs64);
  cudaFree(p->res64);
  cudaFree(p->dbuf);
  cudaFree(p->stage_x);
  cudaFree(p->stage_b);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  if (p->copy_ev) cudaEventDestroy(p->copy_ev);
  for (cudaEvent_t& ev : p->chunk_ev)
    if (ev) cudaEventDestroy(ev);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  for (cudaEvent_t& ev : p->sweep_ev)
    if (ev) cudaEventDestroy(ev);
  bf16_release(p);
  tmg_release(p);
  scattered_release(p);
  cudaFree(p->scal);
  if (p->scal_host) cudaFreeHost(p->scal_host);
  cudaFree(p->red.partials);
  cudaFree(p->red.ticket);
  delete p;
}

}  // namespace tca

using namespace tca;

extern "C" tca_status tca_plan(tca_plan_t* out, int order, const int64_t* n, const tca_factor* factors,
                               const tca_reg* reg, tca_precision prec, cudaStream_t stream) {
  if (!out || !n || !factors) return TCA_ERR_INVALID_ARG;
  *out = nullptr;
  if (order != 3 && order != 4) return TCA_ERR_INVALID_ARG;
  if (prec != TCA_F64 && prec != TCA_F32 && prec != TCA_BF16_IR && prec != TCA_TF32_IR)
    return TCA_ERR_INVALID_ARG;
  for (int k = 0; k < order; ++k) {
    const tca_factor& f = factors[k];
    if (n[k] <= 0 || f.m <= 0 || f.n <= 0 || !f.values) return TCA_ERR_INVALID_ARG;
    if (f.kind == TCA_FACTOR_ELL4 && !f.col0) return TCA_ERR_INVALID_ARG;
    if (f.kind != TCA_FACTOR_ELL4 && f.kind != TCA_FACTOR_DENSE) return TCA_ERR_INVALID_ARG;
    if (f.reserved != 0) return TCA_ERR_INVALID_ARG;
    if (f.n != n[k]) return TCA_ERR_SHAPE;
    if (f.n > (1 << 24) || f.m > (1 << 24)) return TCA_ERR_UNSUPPORTED;
  }
  const double lam = reg ? reg->lambda : 0.0;
  if (!(lam >= 0.0) || !std::isfinite(lam)) return TCA_ERR_INVALID_ARG;
  const uint32_t mask = reg ? reg->reg_mode_mask : 0u;

  static std::atomic<uint64_t> generations{0};
  (void)wait_timeout_flag();  // resolve the flag's device address outside any stream capture
  tca_plan_s* p = new tca_plan_s();
  p->generation = ++generations;
  p->d = order;
  p->prec = prec;
  p->lambda = lam;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (p->num_sms <= 0) p->num_sms = 1;
  p->N = 1;
  p->M = 1;
  for (int k = 0; k < order; ++k) {
    p->n[k] = n[k];
    p->m[k] = factors[k].m;
    p->N *= n[k];
    p->M *= factors[k].m;
  }
  tca_status st = TCA_OK;
  for (int k = 0; k < order && st == TCA_OK; ++k) {
    st = ingest_mode(p, k, factors[k], (mask >> k) & 1u, stream);
    if (factors[k].kind != TCA_FACTOR_ELL4) p->all_band = false;
  }
  if (st != TCA_OK) {
    destroy_plan(p);
    return st;
  }
  // Mode order by cost (Sec. 2.1): shrinking factors first, expanding ones last,
  // which keeps every intermediate as small as the chain allows.
  for (int k = 0; k < order; ++k) p->order_fwd[k] = p->order_bwd[k] = k;
  std::stable_sort(p->order_fwd, p->order_fwd + order, [&](int a, int b) {
    return (double)p->m[a] / p->n[a] < (double)p->m[b] / p->n[b];
  });
  std::stable_sort(p->order_bwd, p->order_bwd + order, [&](int a, int b) {
    return (double)p->n[a] / p->m[a] < (double)p->n[b] / p->m[b];
  });
  const int64_t peak_f = chain_peak(p->n, p->m, p->order_fwd, order);
  const int64_t peak_b = chain_peak(p->m, p->n, p->order_bwd, order);
  p->ws_elems = std::max<int64_t>({peak_f, peak_b, p->N, 1});
  // The fused FP32 sweep covers banded operators whose fastest mode fits the tile.
  // Order 3 runs as a 4D sweep with a unit fastest mode (no G_4, no L_4); an
  // order-4 plan needs its own fastest mode to fill the tile (n4 = 4 or 8).
  if (p->all_band && prec != TCA_F64) {
    p->fused_ok = order == 3 || p->n[3] == 4 || p->n[3] == 8;
  }
  const size_t es = elem_size(p);
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&p->ws[0], es * (size_t)p->ws_elems);
  if (e == cudaSuccess) e = cudaMalloc(&p->ws[1], es * (size_t)p->ws_elems);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->scal, sizeof(Scalars));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->scal_host, sizeof(Scalars));
  p->red.max_blocks = std::max(4096, p->num_sms * 16);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->red.partials, sizeof(double) * p->red.max_blocks);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->red.ticket, 2 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(p->red.ticket, 0, 2 * sizeof(unsigned int), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->scal, 0, sizeof(Scalars), stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  // Mode-4 bands of the warp-specialised sweep travel as kernel parameters.
  if (e == cudaSuccess && p->fused_ok && order == 4 && p->n[3] == 8) {
    e = cudaMemcpy(p->ws_g4, p->mode[3].gram.band.w32, sizeof(p->ws_g4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(p->ws_l4, p->mode[3].lap.w32, sizeof(p->ws_l4), cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    destroy_plan(p);
    return TCA_ERR_ALLOC;
  }
  // bfloat16 plans: the tensor-core sweep's operand tiles and vectors.
  if (prec == TCA_BF16_IR) {
    const tca_status bs = bf16_prepare(p);
    if (bs != TCA_OK) {
      if (bs == TCA_ERR_UNSUPPORTED)
        set_error_message("TCA_BF16_IR needs banded (ELL4) factors, n4 <= 8 and n3*n4 a multiple of 8");
      destroy_plan(p);
      return bs;
    }
  }
  *out = p;
  return TCA_OK;
}

extern "C" void tca_destroy(tca_plan_t plan) {
  if (plan) cudaDeviceSynchronize();
  destroy_plan(plan);
}

extern "C" const char* tca_status_string(tca_status s) {
  switch (s) {
    case TCA_OK: return "ok";
    case TCA_ERR_INVALID_ARG: return "invalid argument";
    case TCA_ERR_SHAPE: return "shape mismatch";
    case TCA_ERR_UNSUPPORTED: return "unsupported";
    case TCA_ERR_ALLOC: return "device allocation failed";
    case TCA_ERR_CUDA: return "CUDA error";
    case TCA_ERR_NOT_CONVERGED: return "not converged";
    case TCA_ERR_BREAKDOWN: return "CG breakdown";
    case TCA_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

extern "C" tca_status tca_precond_default_shift(tca_plan_t plan, double* shift) {
  if (!plan || !shift) return TCA_ERR_INVALID_ARG;
  if (plan->scattered) return TCA_ERR_UNSUPPORTED;
  return tca::precond_model_shift(plan, shift);
}

extern "C" const char* tca_last_error_string(void) { return tca::g_last_error; }

extern "C" uint64_t tca_kernel_launches(int reset) {
  const uint64_t v = tca::g_launches;
  if (reset) tca::g_launches = 0;
  return v;
}

extern "C" int tca_version(void) { return (1 << 16) | 0; }
