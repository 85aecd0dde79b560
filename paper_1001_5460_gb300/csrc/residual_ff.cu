// FP64-accurate operator products on the FP32 pipes, for the true residual.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the true
// residual ||A^T b - K x|| / ||A^T b|| of an FP32 solve (and the right-hand
// side A^T b it is measured against) is computed in double-float arithmetic:
// a value is an unevaluated pair (hi, lo) of floats, products are made exact
// with the FMA-based TwoProduct, sums with Knuth's TwoSum, and every mode
// product is a compensated dot product (the Dot2 scheme of Ogita, Rump and
// Oishi), which returns the result as accurately as if it had been computed
// in twice the working precision and then rounded (~2^-44 relative).
//
// Operators are the plan's bands (7-band Gram factors, transposed ELL-4
// factors, 5-band regulariser) with FP64 coefficients split into float pairs;
// dense factors are run as bands of full width.
#include <algorithm>
#include <cstdio>

#include "tca_internal.cuh"

namespace tca {

namespace {

// Dot2 accumulator: s + c approximates the exact sum.
struct Acc2 {
  float s = 0.f, c = 0.f;
  // += (wh + wl) * (xh + xl), dropping only wl * xl.
  __device__ __forceinline__ void add(float wh, float wl, float xh, float xl) {
    const float ph = wh * xh;
    float pe = fmaf(wh, xh, -ph);  // exact error of the product
    pe = fmaf(wh, xl, pe);
    pe = fmaf(wl, xh, pe);
    const float t = s + ph;        // TwoSum(s, ph)
    const float bb = t - s;
    const float err = (s - (t - bb)) + (ph - bb);
    s = t;
    c += err + pe;
  }
  __device__ __forceinline__ float2 result() const {  // FastTwoSum(s, c)
    const float h = s + c;
    return make_float2(h, c - (h - s));
  }
};

template <typename T> __device__ __forceinline__ float2 as_ff(T v);
template <> __device__ __forceinline__ float2 as_ff<float>(float v) { return make_float2(v, 0.f); }
template <> __device__ __forceinline__ float2 as_ff<float2>(float2 v) { return v; }

// Mode product on the inner layout (I >= 32): lanes along the contiguous inner
// index, 8 outputs along the mode per thread.
template <typename Tin>
__global__ void __launch_bounds__(256) band_ff_inner_kernel(const Tin* __restrict__ x, float2* __restrict__ y,
                                                            float* __restrict__ y32, int64_t O, int n_in, int n_out,
                                                            int64_t I, const int32_t* __restrict__ start,
                                                            const float2* __restrict__ w, int W, int64_t i_chunks,
                                                            int j_chunks) {
  constexpr int JT = 8;
  const int64_t b = blockIdx.x;
  const int jc = (int)(b % j_chunks);
  const int64_t rest = b / j_chunks;
  const int64_t ic = rest % i_chunks;
  const int64_t o = rest / i_chunks;
  const int64_t i = ic * 64 + threadIdx.x;
  if (i >= I) return;
  const Tin* xo = x + o * (int64_t)n_in * I + i;
#pragma unroll 1
  for (int t = 0; t < JT; ++t) {
    const int j = jc * (4 * JT) + threadIdx.y + 4 * t;
    if (j >= n_out) break;
    Acc2 acc;
    const int s0 = start[j];
    for (int e = 0; e < W; ++e) {
      const int l = s0 + e;
      if (l < 0 || l >= n_in) continue;
      const float2 c = w[(int64_t)j * W + e];
      const float2 v = as_ff(xo[(int64_t)l * I]);
      acc.add(c.x, c.y, v.x, v.y);
    }
    const float2 r = acc.result();
    const int64_t oi = (o * (int64_t)n_out + j) * I + i;
    y[oi] = r;
    if (y32) y32[oi] = r.x;
  }
}

// Mode product on the outer layout (I < 32): whole (n_in x I) slabs staged in
// shared memory.
template <typename Tin>
__global__ void __launch_bounds__(256) band_ff_outer_kernel(const Tin* __restrict__ x, float2* __restrict__ y,
                                                            float* __restrict__ y32, int64_t O, int n_in, int n_out,
                                                            int I, const int32_t* __restrict__ start,
                                                            const float2* __restrict__ w, int W, int To) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  const int64_t o0 = (int64_t)blockIdx.x * To;
  const int to = (int)((O - o0) < (int64_t)To ? (O - o0) : (int64_t)To);
  const int sin = n_in * I, sout = n_out * I;
  const Tin* xsrc = x + o0 * sin;
  for (int t = threadIdx.x; t < to * sin; t += blockDim.x) xs[t] = as_ff(xsrc[t]);
  __syncthreads();
  const int lanes = to * I;
  for (int t = threadIdx.x; t < lanes * n_out; t += blockDim.x) {
    const int j = t / lanes;
    const int lane = t - j * lanes;
    const int oo = lane / I;
    const int ii = lane - oo * I;
    const float2* xf = xs + oo * sin + ii;
    Acc2 acc;
    const int s0 = start[j];
    for (int e = 0; e < W; ++e) {
      const int l = s0 + e;
      if (l < 0 || l >= n_in) continue;
      const float2 c = w[(int64_t)j * W + e];
      const float2 v = xf[l * I];
      acc.add(c.x, c.y, v.x, v.y);
    }
    const float2 r = acc.result();
    const int64_t oi = (o0 + oo) * (int64_t)sout + j * I + ii;
    y[oi] = r;
    if (y32) y32[oi] = r.x;
  }
}

struct RegFF {
  const float2* w[kMaxModes];  // lambda L_k split bands (n_k x 5), null if unregularised
  int64_t n[kMaxModes];
  int64_t stride[kMaxModes];
};

// r = rhs - (kx + lambda sum_k L_k x) in double-float; reduces ||r||^2 and
// ||rhs||^2 (FP64 accumulation of the rounded pair sums); optionally writes r
// rounded to FP32 for a CG restart.
__global__ void __launch_bounds__(256) residual_ff_kernel(const float2* __restrict__ rhs, const float2* __restrict__ kx,
                                                          const float* __restrict__ x, float* __restrict__ r_out,
                                                          int64_t total, RegFF reg, Scalars* sc, Reduce red,
                                                          Reduce red2) {
  __shared__ double sh[8];
  double a_rr = 0.0, a_bb = 0.0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    // Accumulate rhs - kx - lambda sum L x as one compensated sum.
    Acc2 acc;
    const float2 b = rhs[idx], k = kx[idx];
    acc.add(1.f, 0.f, b.x, b.y);
    acc.add(-1.f, 0.f, k.x, k.y);
    unsigned rem = (unsigned)idx;  // the host keeps total below 2^32
#pragma unroll
    for (int m = kMaxModes - 1; m >= 0; --m) {
      const int64_t im = rem % (unsigned)reg.n[m];
      rem /= (unsigned)reg.n[m];
      if (!reg.w[m]) continue;
      const float2* wm = reg.w[m] + im * 5;
#pragma unroll
      for (int e = 0; e < 5; ++e) {
        const int64_t c = im - 2 + e;
        if (c >= 0 && c < reg.n[m]) {
          const float2 cf = wm[e];
          acc.add(-cf.x, -cf.y, __ldg(x + idx + (c - im) * reg.stride[m]), 0.f);
        }
      }
    }
    const float2 rv = acc.result();
    const double rd = (double)rv.x + (double)rv.y;
    if (r_out) r_out[idx] = rv.x;
    a_rr += rd * rd;
    const double bd = (double)b.x + (double)b.y;
    a_bb += bd * bd;
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

// Split FP64 values into (hi, lo) float pairs.
__global__ void split_ff_kernel(const double* __restrict__ a, float2* __restrict__ b, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const float hi = (float)a[t];
    b[t] = make_float2(hi, (float)(a[t] - (double)hi));
  }
}

}  // namespace

tca_status split_ff(const double* a, float2* b, int64_t n, cudaStream_t s) {
  if (n <= 0) return TCA_OK;
  split_ff_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// y = x x_k op in double-float (op given as a band: start, split weights, width).
template <typename Tin>
static tca_status launch_ff(const int32_t* start, const float2* w, int W, int n_in, int n_out, const Tin* x, float2* y,
                            float* y32, int64_t O, int64_t I, cudaStream_t s) {
  if (O <= 0 || I <= 0) return TCA_OK;
  if (I >= 32) {
    const int64_t ich = (I + 63) / 64;
    const int jch = (n_out + 31) / 32;
    band_ff_inner_kernel<Tin><<<(unsigned)(O * ich * jch), dim3(64, 4), 0, s>>>(x, y, y32, O, n_in, n_out, I, start,
                                                                                w, W, ich, jch);
  } else {
    const size_t per = sizeof(float2) * (size_t)n_in * (size_t)I;
    int To = (int)std::max<size_t>(1, std::min<size_t>(256, (64 * 1024) / per));
    if ((int64_t)To > O) To = (int)O;
    const size_t sm = per * To;
    if (sm > 200 * 1024) return TCA_ERR_UNSUPPORTED;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(band_ff_outer_kernel<Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    band_ff_outer_kernel<Tin><<<(unsigned)((O + To - 1) / To), 256, sm, s>>>(x, y, y32, O, n_in, n_out, (int)I,
                                                                             start, w, W, To);
  }
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

static void op_band_ff(const ModeOp& op, const int32_t** start, const float2** w, int* W) {
  if (op.kind == OP_BAND) {
    *start = op.band.start;
    *w = op.band.wff;
    *W = op.band.W;
  } else {
    *start = op.dense.zero_start;
    *w = op.dense.aff;
    *W = (int)op.dense.n_in;
  }
}

// Chained product through the plan's ordering; x float, result float2 in y,
// optionally its hi part in y32.  Intermediates in ws[0], ws[1] (float2).
tca_status chain_ff(tca_plan_s* p, bool transpose, bool gram, const float* x, float2* y, float* y32,
                    float2* const* ws, int64_t ws_elems, cudaStream_t s) {
  const int d = p->d;
  int64_t cur[kMaxModes];
  for (int k = 0; k < d; ++k) cur[k] = (transpose && !gram) ? p->m[k] : p->n[k];
  int order_g[kMaxModes];
  for (int k = 0; k < d; ++k) order_g[k] = d - 1 - k;  // innermost first: small-I slabs, then rows
  const int* order = gram ? order_g : (transpose ? p->order_bwd : p->order_fwd);
  const void* src = x;
  for (int st = 0; st < d; ++st) {
    const int k = order[st];
    const ModeOp& op = gram ? p->mode[k].gram : (transpose ? p->mode[k].bwd : p->mode[k].fwd);
    int64_t O = 1, I = 1;
    for (int a = 0; a < k; ++a) O *= cur[a];
    for (int a = k + 1; a < d; ++a) I *= cur[a];
    const int n_in = (int)op.n_in(), n_out = (int)op.n_out();
    cur[k] = n_out;
    const bool last = st == d - 1;
    if (!last && O * I * n_out > ws_elems) return TCA_ERR_SHAPE;
    float2* dst = last ? y : ws[st % 2];
    const int32_t* start;
    const float2* w;
    int W;
    op_band_ff(op, &start, &w, &W);
    if (st == 0)
      TCA_TRY(launch_ff<float>(start, w, W, n_in, n_out, (const float*)src, dst, last ? y32 : nullptr, O, I, s));
    else
      TCA_TRY(launch_ff<float2>(start, w, W, n_in, n_out, (const float2*)src, dst, last ? y32 : nullptr, O, I, s));
    src = dst;
  }
  return TCA_OK;
}

// True residual of x (FP32) against rhs_ff: scal->aux = ||r|| / ||rhs||; r_out (may be null) gets r in FP32.
tca_status residual_ff(tca_plan_s* p, const float* x, const float2* rhs_ff, float2* kx_ff, float* r_out,
                       Reduce red, Reduce red2, cudaStream_t s) {
  TCA_TRY(chain_ff(p, false, true, x, kx_ff, nullptr, (float2* const*)p->ws64, p->ws64_elems, s));
  RegFF reg;
  int64_t stride = 1;
  for (int k = kMaxModes - 1; k >= 0; --k) {
    reg.n[k] = k < p->d ? p->n[k] : 1;
    reg.stride[k] = stride;
    stride *= reg.n[k];
    reg.w[k] = (k < p->d && p->mode[k].reg) ? p->mode[k].lap.wff : nullptr;
  }
  if (p->N >= (int64_t)1 << 32) return TCA_ERR_UNSUPPORTED;
  const int grid = std::min(vector_grid(p, p->N), red.max_blocks - 1);
  residual_ff_kernel<<<grid, 256, 0, s>>>(rhs_ff, kx_ff, x, r_out, p->N, reg, p->scal, red, red2);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace tca
