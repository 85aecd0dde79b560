// Single-mode products (one one-dimensional transformation of Eq.
// separable_transf), the separable regulariser, the chained apply / apply_T
// and the generic normal operator.  Entry points tca_apply, tca_apply_T,
// tca_apply_mode and tca_apply_normal live at the end of this file.
//
// A tensor is viewed, for a product on mode k, as (O, n_in, I): O is the
// product of the modes before k, I of the modes after it (C order).  Two
// kernel shapes cover every mode:
//   * "inner" (I >= 32): lanes run along the contiguous inner index, so every
//     warp access is a coalesced row segment; the band/dense reduction runs
//     along the strided mode index through L1.
//   * "outer" (I < 32): a block stages a run of whole (n_in x I) slabs in
//     shared memory with one contiguous load, computes from shared memory and
//     writes the (n_out x I) slabs back with one contiguous store.
#include <algorithm>
#include <cstdio>

#include "tca_internal.cuh"

namespace tca {

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec4<double> { using type = double2; static constexpr int n = 2; };

template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Banded mode product, inner layout.  Block: 64 lanes along i (VEC elements
// each) x 4 lanes along j; each thread produces JT outputs along j.
template <typename Tin, typename Tout, typename Tc, int VEC>
__global__ void __launch_bounds__(256) band_inner_kernel(
    const Tin* __restrict__ x, Tout* __restrict__ y, int64_t O, int n_in, int n_out, int64_t I,
    const int32_t* __restrict__ start, const Tc* __restrict__ w, int W, int64_t i_chunks, int j_chunks) {
  constexpr int JT = 8;
  const int64_t b = blockIdx.x;
  const int jc = (int)(b % j_chunks);
  const int64_t rest = b / j_chunks;
  const int64_t ic = rest % i_chunks;
  const int64_t o = rest / i_chunks;
  const int64_t i = (ic * 64 + threadIdx.x) * VEC;
  if (i >= I) return;
  const Tin* xo = x + o * (int64_t)n_in * I + i;
  Tout* yo = y + o * (int64_t)n_out * I + i;
  const int jb = jc * (4 * JT) + threadIdx.y;
#pragma unroll
  for (int t = 0; t < JT; ++t) {
    const int j = jb + 4 * t;
    if (j >= n_out) break;
    Tc acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = Tc(0);
    const int s0 = start[j];
    for (int e = 0; e < W; ++e) {
      const int l = s0 + e;
      if (l < 0 || l >= n_in) continue;
      const Tc c = w[(int64_t)j * W + e];
      const Tin* src = xo + (int64_t)l * I;
      if constexpr (VEC == 4 && sizeof(Tin) == 4) {
        const float4 v4 = __ldg(reinterpret_cast<const float4*>(src));
        acc[0] += c * (Tc)v4.x; acc[1] += c * (Tc)v4.y; acc[2] += c * (Tc)v4.z; acc[3] += c * (Tc)v4.w;
      } else if constexpr (VEC == 2 && sizeof(Tin) == 8) {
        const double2 v2 = __ldg(reinterpret_cast<const double2*>(src));
        acc[0] += c * (Tc)v2.x; acc[1] += c * (Tc)v2.y;
      } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v)
          if (i + v < I) acc[v] += c * (Tc)ld(src + v);
      }
    }
    Tout* dst = yo + (int64_t)j * I;
    if constexpr (VEC == 4 && sizeof(Tout) == 4) {
      *reinterpret_cast<float4*>(dst) = make_float4((float)acc[0], (float)acc[1], (float)acc[2], (float)acc[3]);
    } else if constexpr (VEC == 2 && sizeof(Tout) == 8) {
      *reinterpret_cast<double2*>(dst) = make_double2((double)acc[0], (double)acc[1]);
    } else {
#pragma unroll
      for (int v = 0; v < VEC; ++v)
        if (i + v < I) dst[v] = (Tout)acc[v];
    }
  }
}

// Dense mode product, inner layout: A (n_out x n_in) staged in shared memory,
// each thread keeps JT accumulators along j and streams x along l.
template <typename Tin, typename Tout, typename Tc>
__global__ void __launch_bounds__(256) dense_inner_kernel(
    const Tin* __restrict__ x, Tout* __restrict__ y, int64_t O, int n_in, int n_out, int64_t I,
    const Tc* __restrict__ a, int64_t i_chunks, int j_chunks) {
  constexpr int JT = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tc* as = reinterpret_cast<Tc*>(smem_raw);
  const int64_t b = blockIdx.x;
  const int jc = (int)(b % j_chunks);
  const int64_t rest = b / j_chunks;
  const int64_t ic = rest % i_chunks;
  const int64_t o = rest / i_chunks;
  const int j0 = jc * (4 * JT);
  const int jn = min(4 * JT, n_out - j0);
  const int tid = threadIdx.y * 64 + threadIdx.x;
  for (int t = tid; t < jn * n_in; t += 256) as[t] = a[(int64_t)j0 * n_in + t];
  __syncthreads();
  const int64_t i = ic * 64 + threadIdx.x;
  if (i >= I) return;
  const Tin* xo = x + o * (int64_t)n_in * I + i;
  Tc acc[JT];
#pragma unroll
  for (int t = 0; t < JT; ++t) acc[t] = Tc(0);
  for (int l = 0; l < n_in; ++l) {
    const Tc xv = (Tc)ld(xo + (int64_t)l * I);
#pragma unroll
    for (int t = 0; t < JT; ++t) {
      const int jj = threadIdx.y + 4 * t;
      if (jj < jn) acc[t] += as[jj * n_in + l] * xv;
    }
  }
  Tout* yo = y + o * (int64_t)n_out * I + i;
#pragma unroll
  for (int t = 0; t < JT; ++t) {
    const int jj = threadIdx.y + 4 * t;
    if (jj < jn) yo[(int64_t)(j0 + jj) * I] = (Tout)acc[t];
  }
}

// Outer layout for small I (banded or dense).  The block owns `to` slabs
// o0 .. o0+to-1; x slabs are contiguous (to * n_in * I elements) and so are
// the y slabs (to * n_out * I).
template <typename Tin, typename Tout, typename Tc, bool DENSE>
__global__ void __launch_bounds__(256) outer_kernel(
    const Tin* __restrict__ x, Tout* __restrict__ y, int64_t O, int n_in, int n_out, int I,
    const int32_t* __restrict__ start, const Tc* __restrict__ w, int W, int To) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t o0 = (int64_t)blockIdx.x * To;
  const int to = (int)((O - o0) < (int64_t)To ? (O - o0) : (int64_t)To);
  const int sin = n_in * I, sout = n_out * I;
  Tc* xs = reinterpret_cast<Tc*>(smem_raw);
  Tc* ys = xs + (int64_t)To * sin;
  const Tin* xsrc = x + o0 * sin;
  for (int t = threadIdx.x; t < to * sin; t += blockDim.x) xs[t] = (Tc)ld(xsrc + t);
  __syncthreads();
  const int lanes = to * I;
  for (int t = threadIdx.x; t < lanes * n_out; t += blockDim.x) {
    const int j = t / lanes;
    const int lane = t - j * lanes;
    const int oo = lane / I;
    const int ii = lane - oo * I;
    const Tc* xf = xs + oo * sin + ii;
    Tc acc = Tc(0);
    if constexpr (DENSE) {
      const Tc* arow = w + (int64_t)j * n_in;
      for (int l = 0; l < n_in; ++l) acc += ld(arow + l) * xf[l * I];
    } else {
      const int s0 = start[j];
      for (int e = 0; e < W; ++e) {
        const int l = s0 + e;
        if (l >= 0 && l < n_in) acc += w[(int64_t)j * W + e] * xf[l * I];
      }
    }
    ys[oo * sout + j * I + ii] = acc;
  }
  __syncthreads();
  Tout* ydst = y + o0 * sout;
  for (int t = threadIdx.x; t < to * sout; t += blockDim.x) ydst[t] = (Tout)ys[t];
}

// y (+)= sum_k x x_k (lambda L_k) over a 4D view; L_k 5-banded with lambda folded in.
// The view is right-aligned: mode 3 is the innermost mode of the tensor (stride 1),
// leading unit modes pad the front.
struct LapArgs {
  const void* w[kMaxModes];  // Tc-typed band weights (n_k x 5), or null if mode unregularised
  int64_t n[kMaxModes];
  int64_t stride[kMaxModes];
};

template <typename T, int VN>
struct alignas(sizeof(T) * VN) VecN {
  T v[VN];
};

// One thread per run of VN consecutive elements along mode 3 (VN divides n_3,
// so a run never crosses a row): the index is decoded once per run, the taps of
// modes 0-2 are VN-wide loads with one coefficient each, mode 3 reads a
// VN + 4 window.  Per element the terms are summed in the order mode 3, 2, 1, 0,
// taps 0-4, then added to y.  DOT (CG sweep): also <x, y_new> (FP32 runs,
// FP64 beyond) and, in the last block, alpha = rho / <x, y> (Fig. 2
// `alpha := rho/(P+*Q)`), with the same breakdown test as the sweep.
template <typename Tin, typename Tout, typename Tc, int VN, typename IDX, bool DOT>
__global__ void __launch_bounds__(256) reg_run_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, IDX runs,
                                                      LapArgs la, int accumulate, Scalars* sc, Reduce red) {
  __shared__ double sh[256 / 32];
  if constexpr (DOT) {
    if (cg_done(sc)) return;
  }
  const IDX n3 = (IDX)la.n[3], n2 = (IDX)la.n[2], n1 = (IDX)la.n[1];
  Tc part = Tc(0);
  double acc = 0.0;
  int cnt = 0;
  for (IDX ri = (IDX)blockIdx.x * blockDim.x + threadIdx.x; ri < runs; ri += (IDX)gridDim.x * blockDim.x) {
    const IDX idx = ri * VN;
    IDX rem = idx / n3;
    const int i3 = (int)(idx - rem * n3);
    int ik[3];
    ik[2] = (int)(rem % n2);
    rem /= n2;
    ik[1] = (int)(rem % n1);
    ik[0] = (int)(rem / n1);
    Tc a[VN];
#pragma unroll
    for (int j = 0; j < VN; ++j) a[j] = Tc(0);
    if (la.w[3]) {
      const Tc* w = reinterpret_cast<const Tc*>(la.w[3]) + (int64_t)i3 * 5;
      Tc xw[VN + 4];
#pragma unroll
      for (int t = 0; t < VN + 4; ++t) {
        const int c = i3 - 2 + t;
        xw[t] = (c >= 0 && c < (int)n3) ? (Tc)ld(x + idx - 2 + t) : Tc(0);
      }
#pragma unroll
      for (int j = 0; j < VN; ++j) {
#pragma unroll
        for (int e = 0; e < 5; ++e) {
          const int c = i3 + j - 2 + e;
          if (c >= 0 && c < (int)n3) a[j] += ld(w + j * 5 + e) * xw[j + e];
        }
      }
    }
#pragma unroll
    for (int k = 2; k >= 0; --k) {
      if (!la.w[k]) continue;
      const int nk = (int)la.n[k];
      const Tc* w = reinterpret_cast<const Tc*>(la.w[k]) + (int64_t)ik[k] * 5;
#pragma unroll
      for (int e = 0; e < 5; ++e) {
        const int c = ik[k] - 2 + e;
        if (c >= 0 && c < nk) {
          const Tc we = ld(w + e);
          const VecN<Tin, VN> xv =
              *reinterpret_cast<const VecN<Tin, VN>*>(x + idx + (int64_t)(c - ik[k]) * la.stride[k]);
#pragma unroll
          for (int j = 0; j < VN; ++j) a[j] += we * (Tc)xv.v[j];
        }
      }
    }
    VecN<Tout, VN> yv;
    if (accumulate) {
      yv = *reinterpret_cast<const VecN<Tout, VN>*>(y + idx);
#pragma unroll
      for (int j = 0; j < VN; ++j) yv.v[j] = (Tout)((Tc)yv.v[j] + a[j]);
    } else {
#pragma unroll
      for (int j = 0; j < VN; ++j) yv.v[j] = (Tout)a[j];
    }
    *reinterpret_cast<VecN<Tout, VN>*>(y + idx) = yv;
    if constexpr (DOT) {
      const VecN<Tin, VN> xv = *reinterpret_cast<const VecN<Tin, VN>*>(x + idx);
#pragma unroll
      for (int j = 0; j < VN; ++j) part += (Tc)xv.v[j] * (Tc)yv.v[j];
      if (++cnt == 8) {  // short runs in Tc, FP64 beyond
        acc += (double)part;
        part = Tc(0);
        cnt = 0;
      }
    }
  }
  if constexpr (DOT) {
    acc += (double)part;
    double total;
    if (dev::grid_sum_last(acc, red, &total, sh)) {
      sc->pq = total;
      const double alpha = sc->rho / total;
      if (!(total > 0.0) || !isfinite(alpha)) {
        sc->breakdown = 1;
        sc->alpha = 0.0;
      } else {
        sc->alpha = alpha;
      }
    }
  }
}

template <typename T> const T* wsel(const Band& b);
template <> const float* wsel<float>(const Band& b) { return b.w32; }
template <> const double* wsel<double>(const Band& b) { return b.w64; }
template <typename T> const T* asel(const Dense& d);
template <> const float* asel<float>(const Dense& d) { return d.a32; }
template <> const double* asel<double>(const Dense& d) { return d.a64; }

}  // namespace

template <typename Tin, typename Tout, typename Tc>
tca_status launch_mode_op(const ModeOp& op, const Tin* x, Tout* y, int64_t O, int64_t I, cudaStream_t s) {
  const int n_in = (int)op.n_in(), n_out = (int)op.n_out();
  if (O <= 0 || I <= 0) return TCA_OK;
  const bool dense = op.kind == OP_DENSE;
  if constexpr (sizeof(Tin) == 4 && sizeof(Tout) == 4 && sizeof(Tc) == 4) {
    // FP32 bands: TMA-staged row tiles or register fibres when the shape allows.
    if (!dense) {
      const tca_status st = launch_band_fast(op.band, (const float*)x, (float*)y, O, I, s, op.sm_cap);
      if (st != TCA_ERR_UNSUPPORTED) return st;
    } else if (op.tc_split > 0) {
      const tca_status st =
          launch_dense_tc(op.dense, (const float*)x, (float*)y, O, I, op.tc_split, s, op.sm_cap, op.stop);
      if (st != TCA_ERR_UNSUPPORTED) return st;
    }
  }
  const Tc* w = dense ? asel<Tc>(op.dense) : wsel<Tc>(op.band);
  if (I >= 32) {
    const int64_t i_chunks_v = (I + 255) / 256;
    const int64_t i_chunks_s = (I + 63) / 64;
    const int j_chunks = (n_out + 31) / 32;
    dim3 block(64, 4);
    if (!dense) {
      constexpr int V = Vec4<Tin>::n;
      const bool vec_ok = (I % V == 0) && sizeof(Tin) == sizeof(Tout) &&
                          ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0);
      if (vec_ok) {
        const int64_t ich = (I + 64 * V - 1) / (64 * V);
        band_inner_kernel<Tin, Tout, Tc, V><<<(unsigned)(O * ich * j_chunks), block, 0, s>>>(
            x, y, O, n_in, n_out, I, op.band.start, w, op.band.W, ich, j_chunks);
      } else {
        band_inner_kernel<Tin, Tout, Tc, 1><<<(unsigned)(O * i_chunks_s * j_chunks), block, 0, s>>>(
            x, y, O, n_in, n_out, I, op.band.start, w, op.band.W, i_chunks_s, j_chunks);
      }
      (void)i_chunks_v;
    } else {
      const size_t sm = sizeof(Tc) * 32 * (size_t)n_in;
      if (sm > 200 * 1024) return TCA_ERR_UNSUPPORTED;
      if (sm > 48 * 1024)
        cudaFuncSetAttribute(dense_inner_kernel<Tin, Tout, Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      dense_inner_kernel<Tin, Tout, Tc><<<(unsigned)(O * i_chunks_s * j_chunks), block, sm, s>>>(
          x, y, O, n_in, n_out, I, w, i_chunks_s, j_chunks);
    }
    TCA_LAUNCH_CHECK();
    return TCA_OK;
  }
  // Outer layout.
  const size_t per = sizeof(Tc) * (size_t)(n_in + n_out) * (size_t)I;
  const size_t budget = 96 * 1024;
  int To = (int)std::max<size_t>(1, std::min<size_t>(256, budget / per));
  if ((int64_t)To > O) To = (int)O;
  const size_t sm = per * To;
  if (sm > 200 * 1024) return TCA_ERR_UNSUPPORTED;
  const unsigned grid = (unsigned)((O + To - 1) / To);
  if (dense) {
    auto kfn = outer_kernel<Tin, Tout, Tc, true>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kfn<<<grid, 256, sm, s>>>(x, y, O, n_in, n_out, (int)I, nullptr, w, 0, To);
  } else {
    auto kfn = outer_kernel<Tin, Tout, Tc, false>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kfn<<<grid, 256, sm, s>>>(x, y, O, n_in, n_out, (int)I, op.band.start, w, op.band.W, To);
  }
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template <typename Tin, typename Tout, typename Tc, int VN, bool DOT>
static void launch_reg_run(const tca_plan_s* p, const Tin* x, Tout* y, int64_t total, const LapArgs& la,
                           int accumulate, const RegDot* dot, cudaStream_t s) {
  const int64_t runs = total / VN;
  int64_t grid = std::min<int64_t>((runs + 255) / 256, (int64_t)p->num_sms * 8);
  if (dot) grid = std::min<int64_t>(grid, dot->red.max_blocks);
  grid = std::max<int64_t>(grid, 1);
  Scalars* sc = dot ? dot->sc : nullptr;
  const Reduce red = dot ? dot->red : Reduce{};
  if (total + 4 * (int64_t)VN < ((int64_t)1 << 31))
    reg_run_kernel<Tin, Tout, Tc, VN, uint32_t, DOT><<<(unsigned)grid, 256, 0, s>>>(x, y, (uint32_t)runs, la,
                                                                                    accumulate, sc, red);
  else
    reg_run_kernel<Tin, Tout, Tc, VN, int64_t, DOT><<<(unsigned)grid, 256, 0, s>>>(x, y, runs, la, accumulate, sc,
                                                                                   red);
}

template <typename Tin, typename Tout>
tca_status launch_reg_add_impl(const tca_plan_s* p, const Tin* x, Tout* y, const int64_t* dims4,
                               int accumulate, const RegDot* dot, cudaStream_t s) {
  using Tc = Tout;
  // Right-align the view: the last mode with more than one element becomes mode 3.
  int last = 0;
  for (int k = 0; k < kMaxModes; ++k)
    if (dims4[k] > 1) last = k;
  const int shift = kMaxModes - 1 - last;
  LapArgs la;
  int64_t stride = 1;
  for (int k = kMaxModes - 1; k >= 0; --k) {
    const int src = k - shift;
    la.n[k] = src >= 0 ? dims4[src] : 1;
    la.stride[k] = stride;
    stride *= la.n[k];
    const bool on = src >= 0 && src < p->d && p->mode[src].reg;
    la.w[k] = on ? (const void*)wsel<Tc>(p->mode[src].lap) : nullptr;
  }
  const int64_t total = stride;
  if (total <= 0) return TCA_OK;
  constexpr int VN = 16 / (sizeof(Tin) > sizeof(Tout) ? sizeof(Tin) : sizeof(Tout));
  const bool vec = la.n[3] % VN == 0 && (uintptr_t)x % (VN * sizeof(Tin)) == 0 &&
                   (uintptr_t)y % (VN * sizeof(Tout)) == 0;
  if (dot) {
    if (vec) launch_reg_run<Tin, Tout, Tc, VN, true>(p, x, y, total, la, accumulate, dot, s);
    else launch_reg_run<Tin, Tout, Tc, 1, true>(p, x, y, total, la, accumulate, dot, s);
  } else {
    if (vec) launch_reg_run<Tin, Tout, Tc, VN, false>(p, x, y, total, la, accumulate, nullptr, s);
    else launch_reg_run<Tin, Tout, Tc, 1, false>(p, x, y, total, la, accumulate, nullptr, s);
  }
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template <typename Tin, typename Tout>
tca_status launch_reg_add(const tca_plan_s* p, const Tin* x, Tout* y, const int64_t* dims4, cudaStream_t s) {
  return launch_reg_add_impl<Tin, Tout>(p, x, y, dims4, 1, nullptr, s);
}

static void dims4_of(const tca_plan_s* p, int64_t* d4) {
  for (int k = 0; k < kMaxModes; ++k) d4[k] = k < p->d ? p->n[k] : 1;
}

template <typename Tin, typename Tout, typename Tc>
tca_status apply_chain(tca_plan_s* p, bool transpose, const Tin* x, Tout* y, void* const* ws,
                       int64_t ws_elems, cudaStream_t s) {
  if (p->scattered) {
    // Scattered samples: one gather (A x) or one scatter-add (A^T y) in the plan's type.
    if constexpr (sizeof(Tin) == sizeof(Tout)) {
      using T = Tout;
      return transpose ? scattered_scatter<T>(p, (const T*)x, (T*)y, true, s)
                       : scattered_gather<T>(p, (const T*)x, (T*)y, true, s);
    }
    return TCA_ERR_UNSUPPORTED;
  }
  const int d = p->d;
  int64_t cur[kMaxModes];
  for (int k = 0; k < d; ++k) cur[k] = transpose ? p->m[k] : p->n[k];
  const int* order = transpose ? p->order_bwd : p->order_fwd;
  const void* src = x;
  for (int st = 0; st < d; ++st) {
    const int k = order[st];
    const ModeOp& op = transpose ? p->mode[k].bwd : p->mode[k].fwd;
    int64_t O = 1, I = 1;
    for (int a = 0; a < k; ++a) O *= cur[a];
    for (int a = k + 1; a < d; ++a) I *= cur[a];
    cur[k] = op.n_out();
    int64_t out_elems = O * I * cur[k];
    const bool last = st == d - 1;
    if (!last && out_elems > ws_elems) return TCA_ERR_SHAPE;
    void* dst = last ? (void*)y : ws[st % 2];
    tca_status r;
    if (st == 0 && last) r = launch_mode_op<Tin, Tout, Tc>(op, (const Tin*)src, (Tout*)dst, O, I, s);
    else if (st == 0) r = launch_mode_op<Tin, Tc, Tc>(op, (const Tin*)src, (Tc*)dst, O, I, s);
    else if (last) r = launch_mode_op<Tc, Tout, Tc>(op, (const Tc*)src, (Tout*)dst, O, I, s);
    else r = launch_mode_op<Tc, Tc, Tc>(op, (const Tc*)src, (Tc*)dst, O, I, s);
    if (r != TCA_OK) return r;
    src = dst;
  }
  return TCA_OK;
}

// (G_1 kron .. kron G_d) x + lambda R x through single-mode sweeps; element type T.
// With dot, the regulariser pass also forms <x, y> and alpha (CG sweep).
template <typename T>
tca_status normal_generic(tca_plan_s* p, const T* x, T* y, cudaStream_t s, const RegDot* dot) {
  int64_t d4[kMaxModes];
  dims4_of(p, d4);
  if (p->scattered) {
    // A^T (A x) through sample space (grouped sample order), then lambda R x
    // (and <x, y>) as for separable plans.
    T* tmp = reinterpret_cast<T*>(p->sc_tmp);
    TCA_TRY(scattered_gather<T>(p, x, tmp, false, s));
    TCA_TRY(scattered_scatter<T>(p, tmp, y, false, s));
    return launch_reg_add_impl<T, T>(p, x, y, d4, 1, dot, s);
  }
  const int d = p->d;
  const void* src = x;
  for (int k = 0; k < d; ++k) {
    int64_t O = 1, I = 1;
    for (int a = 0; a < k; ++a) O *= p->n[a];
    for (int a = k + 1; a < d; ++a) I *= p->n[a];
    void* dst = (k == d - 1) ? (void*)y : p->ws[k % 2];
    TCA_TRY((launch_mode_op<T, T, T>(p->mode[k].gram, (const T*)src, (T*)dst, O, I, s)));
    src = dst;
  }
  return launch_reg_add_impl<T, T>(p, x, y, d4, 1, dot, s);
}

// z = M^-1 r for the separable-inverse preconditioner: one dense mode product
// per mode with the factors (G_k + s lambda L_k)^-1, through the ping-pong
// workspace.
// The banded form applies B_1 kron .. kron B_d (7-band truncated inverses): one
// plain fused sweep with zero regulariser bands where the plan has the fused
// sweep (it returns at entry once the CG stop flags are set), band mode
// products otherwise.
template <typename T>
tca_status apply_precond(tca_plan_s* p, const T* r, T* z, cudaStream_t s) {
  const bool banded = p->pc_kind == TCA_PRECOND_SEPARABLE_BANDED;
  if constexpr (sizeof(T) == 4) {
    if (banded && p->fused_ok && (uintptr_t)r % 16 == 0)
      return normal_fused_f32(p, nullptr, (const float*)r, nullptr, (float*)z, false, s, &p->pcb_fused, p->scal);
  }
  const int d = p->d;
  const void* src = r;
  for (int k = 0; k < d; ++k) {
    int64_t O = 1, I = 1;
    for (int a = 0; a < k; ++a) O *= p->n[a];
    for (int a = k + 1; a < d; ++a) I *= p->n[a];
    void* dst = (k == d - 1) ? (void*)z : p->ws[k % 2];
    TCA_TRY((launch_mode_op<T, T, T>(banded ? p->pcb[k] : p->pc[k], (const T*)src, (T*)dst, O, I, s)));
    src = dst;
  }
  return TCA_OK;
}
tca_status apply_precond_dot(tca_plan_s* p, const float* r, float* z, bool init, cudaStream_t s) {
  if (p->pc_kind != TCA_PRECOND_SEPARABLE_BANDED || !p->fused_ok || (uintptr_t)r % 16 != 0)
    return TCA_ERR_UNSUPPORTED;
  return normal_fused_f32(p, nullptr, r, nullptr, z, false, s, &p->pcb_fused, p->scal, init ? 1 : 2);
}

template tca_status apply_precond<float>(tca_plan_s*, const float*, float*, cudaStream_t);
template tca_status apply_precond<double>(tca_plan_s*, const double*, double*, cudaStream_t);

static tca_status ensure_ws64(tca_plan_s* p) {
  if (p->ws64[0]) return TCA_OK;
  const int64_t need = std::max(p->ws_elems, p->N);
  cudaError_t e = cudaMalloc((void**)&p->ws64[0], sizeof(double) * need);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->ws64[1], sizeof(double) * need);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  p->ws64_elems = need;
  return TCA_OK;
}

template <typename Tin>
tca_status normal_fp64(tca_plan_s* p, const Tin* x, double* y, cudaStream_t s) {
  TCA_TRY(ensure_ws64(p));
  if (p->scattered) {
    if constexpr (sizeof(Tin) == 8) return normal_generic<double>(p, (const double*)x, y, s, nullptr);
    return TCA_ERR_UNSUPPORTED;
  }
  const int d = p->d;
  const void* src = x;
  for (int k = 0; k < d; ++k) {
    int64_t O = 1, I = 1;
    for (int a = 0; a < k; ++a) O *= p->n[a];
    for (int a = k + 1; a < d; ++a) I *= p->n[a];
    double* dst = (k == d - 1) ? y : p->ws64[k % 2];
    if (k == 0) TCA_TRY((launch_mode_op<Tin, double, double>(p->mode[k].gram, (const Tin*)src, dst, O, I, s)));
    else TCA_TRY((launch_mode_op<double, double, double>(p->mode[k].gram, (const double*)src, dst, O, I, s)));
    src = dst;
  }
  int64_t d4[kMaxModes];
  dims4_of(p, d4);
  return launch_reg_add<Tin, double>(p, x, y, d4, s);
}

tca_status ensure_ws64_public(tca_plan_s* p) { return ensure_ws64(p); }

template tca_status normal_generic<float>(tca_plan_s*, const float*, float*, cudaStream_t, const RegDot*);
template tca_status normal_generic<double>(tca_plan_s*, const double*, double*, cudaStream_t, const RegDot*);
template tca_status normal_fp64<float>(tca_plan_s*, const float*, double*, cudaStream_t);
template tca_status normal_fp64<double>(tca_plan_s*, const double*, double*, cudaStream_t);
template tca_status apply_chain<float, float, float>(tca_plan_s*, bool, const float*, float*, void* const*, int64_t, cudaStream_t);
template tca_status apply_chain<double, double, double>(tca_plan_s*, bool, const double*, double*, void* const*, int64_t, cudaStream_t);
template tca_status apply_chain<float, double, double>(tca_plan_s*, bool, const float*, double*, void* const*, int64_t, cudaStream_t);
template tca_status launch_mode_op<float, float, float>(const ModeOp&, const float*, float*, int64_t, int64_t, cudaStream_t);
template tca_status launch_mode_op<double, double, double>(const ModeOp&, const double*, double*, int64_t, int64_t, cudaStream_t);
template tca_status launch_reg_add<float, float>(const tca_plan_s*, const float*, float*, const int64_t*, cudaStream_t);
template tca_status launch_reg_add<double, double>(const tca_plan_s*, const double*, double*, const int64_t*, cudaStream_t);

// ---- pointer staging for host buffers ---------------------------------------

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

tca_status ensure_stage(tca_plan_s* p) {
  if (p->stage_x) return TCA_OK;
  const size_t es = elem_size(p);
  const int64_t big = std::max(p->N, p->M);
  cudaError_t e = cudaMalloc(&p->stage_x, es * (size_t)big);
  if (e == cudaSuccess) e = cudaMalloc(&p->stage_b, es * (size_t)big);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  return TCA_OK;
}

}  // namespace tca

using namespace tca;

namespace {

// Run `body(in_dev, out_dev)` with host buffers staged through the plan.
template <typename F>
tca_status with_staging(tca_plan_s* p, const void* in, int64_t in_elems, void* out, int64_t out_elems,
                        cudaStream_t s, F body) {
  const bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
  if (in_dev && out_dev) return body(in, out);
  TCA_TRY(ensure_stage(p));
  const size_t es = elem_size(p);
  const void* din = in;
  void* dout = out;
  if (!in_dev) {
    TCA_CUDA_TRY(cudaMemcpyAsync(p->stage_x, in, es * in_elems, cudaMemcpyHostToDevice, s));
    din = p->stage_x;
  }
  if (!out_dev) dout = p->stage_b;
  TCA_TRY(body(din, dout));
  if (!out_dev) TCA_CUDA_TRY(cudaMemcpyAsync(out, p->stage_b, es * out_elems, cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  return TCA_OK;
}

tca_status apply_dispatch(tca_plan_s* p, bool transpose, const void* in, void* out, cudaStream_t s) {
  const int64_t in_e = transpose ? p->M : p->N, out_e = transpose ? p->N : p->M;
  return with_staging(p, in, in_e, out, out_e, s, [&](const void* a, void* b) -> tca_status {
    if (p->prec == TCA_F64)
      return apply_chain<double, double, double>(p, transpose, (const double*)a, (double*)b, p->ws, p->ws_elems, s);
    return apply_chain<float, float, float>(p, transpose, (const float*)a, (float*)b, p->ws, p->ws_elems, s);
  });
}

}  // namespace

extern "C" tca_status tca_apply(tca_plan_t plan, const void* x, void* y, cudaStream_t stream) {
  if (!plan || !x || !y) return TCA_ERR_INVALID_ARG;
  return apply_dispatch(plan, false, x, y, stream);
}

extern "C" tca_status tca_apply_T(tca_plan_t plan, const void* y, void* x, cudaStream_t stream) {
  if (!plan || !x || !y) return TCA_ERR_INVALID_ARG;
  return apply_dispatch(plan, true, y, x, stream);
}

extern "C" tca_status tca_apply_normal(tca_plan_t plan, const void* x, void* y, cudaStream_t stream) {
  if (!plan || !x || !y) return TCA_ERR_INVALID_ARG;
  if (x == y) return TCA_ERR_INVALID_ARG;
  tca_plan_s* p = plan;
  return with_staging(p, x, p->N, y, p->N, stream, [&](const void* a, void* b) -> tca_status {
    if (p->prec == TCA_F64) return normal_generic<double>(p, (const double*)a, (double*)b, stream);
    if (p->prec == TCA_BF16_IR) return normal_bf16(p, (const float*)a, (float*)b, stream);
    if (p->fused_ok && (uintptr_t)a % 16 == 0)
      return normal_fused_f32(p, nullptr, (const float*)a, nullptr, (float*)b, false, stream);
    return normal_generic<float>(p, (const float*)a, (float*)b, stream);
  });
}

extern "C" tca_status tca_apply_mode(tca_plan_t plan, int mode, int op, const int64_t* dims, const void* x,
                                     void* y, cudaStream_t stream) {
  if (!plan || !dims || !x || !y || x == y) return TCA_ERR_INVALID_ARG;
  tca_plan_s* p = plan;
  if (p->scattered) return TCA_ERR_UNSUPPORTED;  // no per-mode factors
  if (mode < 0 || mode >= p->d) return TCA_ERR_INVALID_ARG;
  const Mode& md = p->mode[mode];
  const ModeOp* mop = op == TCA_OP_FACTOR ? &md.fwd : op == TCA_OP_FACTOR_T ? &md.bwd : op == TCA_OP_GRAM ? &md.gram : nullptr;
  if (!mop) return TCA_ERR_INVALID_ARG;
  if (dims[mode] != mop->n_in()) return TCA_ERR_SHAPE;
  int64_t O = 1, I = 1;
  for (int a = 0; a < mode; ++a) {
    if (dims[a] <= 0) return TCA_ERR_SHAPE;
    O *= dims[a];
  }
  for (int a = mode + 1; a < p->d; ++a) {
    if (dims[a] <= 0) return TCA_ERR_SHAPE;
    I *= dims[a];
  }
  if (!is_device_ptr(x) || !is_device_ptr(y)) return TCA_ERR_UNSUPPORTED;
  if (p->prec == TCA_F64) return launch_mode_op<double, double, double>(*mop, (const double*)x, (double*)y, O, I, stream);
  return launch_mode_op<float, float, float>(*mop, (const float*)x, (float*)y, O, I, stream);
}
