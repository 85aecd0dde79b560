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
  // += (wh + wl) * x for an FP32 (exact, single-float) x: the same sum without
  // the product with x's zero low part.
  __device__ __forceinline__ void add_x(float wh, float wl, float x) {
    const float ph = wh * x;
    float pe = fmaf(wh, x, -ph);
    pe = fmaf(wl, x, pe);
    const float t = s + ph;
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

// acc += c * v, v an FP32 value (low part zero) or a double-float pair.
__device__ __forceinline__ void acc_add(Acc2& acc, float2 c, float v) { acc.add_x(c.x, c.y, v); }
__device__ __forceinline__ void acc_add(Acc2& acc, float2 c, float2 v) { acc.add(c.x, c.y, v.x, v.y); }

template <typename T> __device__ __forceinline__ float2 as_ff(T v);
template <> __device__ __forceinline__ float2 as_ff<float>(float v) { return make_float2(v, 0.f); }
template <> __device__ __forceinline__ float2 as_ff<float2>(float2 v) { return v; }

// Mode product on the inner layout (I >= 32): lanes along the contiguous inner
// index, JT outputs along the mode per thread, their accumulators advanced
// together so that each tap step has JT independent loads in flight.
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
  int s0[JT];
  bool jv[JT];
#pragma unroll
  for (int t = 0; t < JT; ++t) {
    const int j = jc * (4 * JT) + threadIdx.y + 4 * t;
    jv[t] = j < n_out;
    s0[t] = jv[t] ? start[j] : 0;
  }
  Acc2 acc[JT];
#pragma unroll 1
  for (int e = 0; e < W; ++e) {
#pragma unroll
    for (int t = 0; t < JT; ++t) {
      const int j = jc * (4 * JT) + threadIdx.y + 4 * t;
      const int l = s0[t] + e;
      const bool ok = jv[t] && l >= 0 && l < n_in;
      // A zero coefficient leaves the accumulator exactly unchanged.
      const float2 c = ok ? w[(int64_t)j * W + e] : make_float2(0.f, 0.f);
      const float2 v = ok ? as_ff(xo[(int64_t)l * I]) : make_float2(0.f, 0.f);
      acc[t].add(c.x, c.y, v.x, v.y);
    }
  }
#pragma unroll
  for (int t = 0; t < JT; ++t) {
    if (!jv[t]) continue;
    const int j = jc * (4 * JT) + threadIdx.y + 4 * t;
    const float2 r = acc[t].result();
    const int64_t oi = (o * (int64_t)n_out + j) * I + i;
    y[oi] = r;
    if (y32) y32[oi] = r.x;
  }
}

// Four consecutive elements (16-byte aligned): FP32 values or double-float pairs.
__device__ __forceinline__ void load4_ff(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void load4_ff(const float2* p, float2 (&v)[4]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0];
  const float4 b = reinterpret_cast<const float4*>(p)[1];
  v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
}

// One output row j over four lanes: acc[q] += sum_e w[j][e] x[start[j] + e][q],
// x given by a row pointer and a row pitch.  Rows outside [0, n_in) are
// skipped; a window wholly inside (the common case) runs unpredicated.
template <typename Tin>
__device__ __forceinline__ void taps4(Acc2 (&acc)[4], const Tin* x0, int64_t pitch, int s0, int W, int n_in,
                                      const float2* __restrict__ wj) {
  if (s0 >= 0 && s0 + W <= n_in) {
    const Tin* xr = x0 + (int64_t)s0 * pitch;
#pragma unroll 2
    for (int e = 0; e < W; ++e) {
      const float2 c = wj[e];
      Tin v[4];
      load4_ff(xr + (int64_t)e * pitch, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc_add(acc[q], c, v[q]);
    }
  } else {
    for (int e = 0; e < W; ++e) {
      const int l = s0 + e;
      if (l < 0 || l >= n_in) continue;
      const float2 c = wj[e];
      Tin v[4];
      load4_ff(x0 + (int64_t)l * pitch, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc_add(acc[q], c, v[q]);
    }
  }
}

__device__ __forceinline__ void store4_ff(float2* y, float* y32, int64_t oi, const Acc2 (&acc)[4]) {
  float2 r[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) r[q] = acc[q].result();
  reinterpret_cast<float4*>(y + oi)[0] = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
  reinterpret_cast<float4*>(y + oi)[1] = make_float4(r[2].x, r[2].y, r[3].x, r[3].y);
  if (y32) *reinterpret_cast<float4*>(y32 + oi) = make_float4(r[0].x, r[1].x, r[2].x, r[3].x);
}

// Mode product on the inner layout with I a multiple of 4 (16-byte aligned
// buffers): a thread owns four consecutive inner lanes and JT outputs along
// the mode, so each coefficient load, bounds test and address step serves four
// Dot2 accumulations and each input row arrives in one or two 16-byte loads.
template <typename Tin>
__global__ void __launch_bounds__(256) band_ff_inner4_kernel(const Tin* __restrict__ x, float2* __restrict__ y,
                                                             float* __restrict__ y32, int n_in, int n_out, int64_t I,
                                                             const int32_t* __restrict__ start,
                                                             const float2* __restrict__ w, int W, int64_t i_chunks,
                                                             int j_chunks, int j_begin, int j_end) {
  constexpr int JT = 4;
  const int64_t b = blockIdx.x;
  const int jc = (int)(b % j_chunks);
  const int64_t rest = b / j_chunks;
  const int64_t ic = rest % i_chunks;
  const int64_t o = rest / i_chunks;
  const int64_t i = (ic * 64 + threadIdx.x) * 4;
  if (i >= I) return;
  const Tin* xo = x + o * (int64_t)n_in * I + i;
#pragma unroll 1
  for (int t = 0; t < JT; ++t) {
    const int j = j_begin + jc * (4 * JT) + threadIdx.y + 4 * t;
    if (j >= j_end) break;
    Acc2 acc[4];
    taps4<Tin>(acc, xo, I, start[j], W, n_in, w + (int64_t)j * W);
    store4_ff(y, y32, (o * (int64_t)n_out + j) * I + i, acc);
  }
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Mode product on the outer layout (I < 32): a persistent CTA walks tiles of
// To consecutive (n_in x I) slabs, each one contiguous range of the input,
// staged in shared memory by cp.async (16-byte copies when VEC, element copies
// otherwise) through a ring of `stages` buffers, so the next tile's copy runs
// under the current tile's arithmetic.  Thread t of a tile computes output
// t, t + 256, ... in memory order: the stores are coalesced.
// MODE 0: one output per step (any I); 1: four consecutive inner lanes
// (I % 4 == 0); 2: four consecutive slabs of the same output row (I == 1).
template <typename Tin, bool VEC, int MODE>
__global__ void __launch_bounds__(256) band_ff_outer_kernel(const Tin* __restrict__ x, float2* __restrict__ y,
                                                            float* __restrict__ y32, int64_t O, int n_in, int n_out,
                                                            int I, const int32_t* __restrict__ start,
                                                            const float2* __restrict__ w, int W, int To, int stages) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int sin = n_in * I, sout = n_out * I;
  const int64_t tiles = (O + To - 1) / To;
  const int buf_elems = ((To * sin * (int)sizeof(Tin) + 15) / 16) * 16 / (int)sizeof(Tin);
  auto issue = [&](int64_t tile, int buf) {
    const int64_t o0 = tile * To;
    const int to = (int)((O - o0) < (int64_t)To ? (O - o0) : (int64_t)To);
    Tin* dst = reinterpret_cast<Tin*>(smem_raw) + (size_t)buf * buf_elems;
    const Tin* src = x + o0 * sin;
    if constexpr (VEC) {
      const int n16 = to * sin * (int)sizeof(Tin) / 16;
      for (int t = threadIdx.x; t < n16; t += blockDim.x)
        cp_async<16>(reinterpret_cast<unsigned char*>(dst) + 16 * t, reinterpret_cast<const unsigned char*>(src) + 16 * t);
    } else {
      for (int t = threadIdx.x; t < to * sin; t += blockDim.x) cp_async<(int)sizeof(Tin)>(dst + t, src + t);
    }
  };
  int64_t tile = blockIdx.x;
  for (int st = 0; st < stages - 1; ++st) {
    const int64_t tt = tile + (int64_t)st * gridDim.x;
    if (tt < tiles) issue(tt, st);
    cp_async_commit();
  }
  for (int64_t k = 0; tile < tiles; ++k, tile += gridDim.x) {
    if (stages > 1) {
      const int64_t tn = tile + (int64_t)(stages - 1) * gridDim.x;
      if (tn < tiles) issue(tn, (int)((k + stages - 1) % stages));
      cp_async_commit();
      cp_async_wait<1>();  // all but the newest group complete: this tile has landed
    } else {
      issue(tile, 0);
      cp_async_commit();
      cp_async_wait<0>();
    }
    __syncthreads();
    const Tin* xs = reinterpret_cast<const Tin*>(smem_raw) + (size_t)(k % stages) * buf_elems;
    const int64_t o0 = tile * To;
    const int to = (int)((O - o0) < (int64_t)To ? (O - o0) : (int64_t)To);
    if constexpr (MODE == 1) {
      // Groups of four inner lanes in output memory order (coalesced stores).
      const int gi = I / 4;
      for (int t = threadIdx.x; t < to * n_out * gi; t += blockDim.x) {
        const int oo = t / (n_out * gi);
        const int rem = t - oo * (n_out * gi);
        const int j = rem / gi;
        const int ii = 4 * (rem - j * gi);
        Acc2 acc[4];
        taps4<Tin>(acc, xs + oo * sin + ii, I, start[j], W, n_in, w + (int64_t)j * W);
        store4_ff(y, y32, o0 * sout + (int64_t)oo * sout + j * I + ii, acc);
      }
    } else if constexpr (MODE == 2) {
      // Four slabs (fibres) per thread for one output row j; j fastest across
      // threads, so each store instruction writes consecutive outputs.
      const int groups = (to + 3) / 4;
      for (int t = threadIdx.x; t < groups * n_out; t += blockDim.x) {
        const int g = t / n_out;
        const int j = t - g * n_out;
        const int s0 = start[j];
        const float2* wj = w + (int64_t)j * W;
        const int nq = min(4, to - 4 * g);
        const Tin* xf = xs + (4 * g) * sin;
        Acc2 acc[4];
        for (int e = 0; e < W; ++e) {
          const int l = s0 + e;
          if (l < 0 || l >= n_in) continue;
          const float2 c = wj[e];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const Tin v = q < nq ? xf[q * sin + l] : Tin{};
            acc_add(acc[q], c, v);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (q >= nq) break;
          const float2 r = acc[q].result();
          const int64_t oi = (o0 + 4 * g + q) * (int64_t)n_out + j;
          y[oi] = r;
          if (y32) y32[oi] = r.x;
        }
      }
    } else {
      for (int t = threadIdx.x; t < to * sout; t += blockDim.x) {
        const int oo = t / sout;
        const int rem = t - oo * sout;
        const int j = rem / I;
        const int ii = rem - j * I;
        const Tin* xf = xs + oo * sin + ii;
        Acc2 acc;
        const int s0 = start[j];
#pragma unroll 4
        for (int e = 0; e < W; ++e) {
          const int l = s0 + e;
          const bool ok = l >= 0 && l < n_in;
          const float2 c = ok ? w[(int64_t)j * W + e] : make_float2(0.f, 0.f);
          const Tin v = ok ? xf[l * I] : Tin{};
          acc_add(acc, c, v);
        }
        const float2 r = acc.result();
        const int64_t oi = o0 * sout + t;
        y[oi] = r;
        if (y32) y32[oi] = r.x;
      }
    }
    __syncthreads();  // the buffer is refilled by the next iteration's copy
  }
  cp_async_wait<0>();
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
          acc.add_x(-cf.x, -cf.y, __ldg(x + idx + (c - im) * reg.stride[m]));
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
    // Relative norm; the absolute one when the right-hand side is zero (0 for x = 0).
    const double rr = sqrt(((volatile double*)red2.partials)[red2.max_blocks - 1]);
    sc->aux = t_bb > 0.0 ? rr / sqrt(t_bb) : rr;
  }
}

// The same residual for runs of four consecutive elements along the
// innermost mode L (n_L a multiple of 4, 16-byte aligned vectors): one index
// decode and one 16-byte load per neighbouring run instead of one scalar load
// per tap, and the taps of each element accumulated in the order of
// residual_ff_kernel (so the two give the same values).
template <int L>
__global__ void __launch_bounds__(256, 4) residual_ff_vec_kernel(const float2* __restrict__ rhs,
                                                              const float2* __restrict__ kx,
                                                              const float* __restrict__ x, float* __restrict__ r_out,
                                                              int64_t total, RegFF reg, Scalars* sc, Reduce red,
                                                              Reduce red2) {
  __shared__ double sh[8];
  double a_rr = 0.0, a_bb = 0.0;
  const int64_t runs = total / 4;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < runs; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = 4 * v;
    int im[kMaxModes];
    unsigned rem = (unsigned)idx;  // the host keeps total below 2^32
#pragma unroll
    for (int m = kMaxModes - 1; m >= 0; --m) {
      im[m] = (int)(rem % (unsigned)reg.n[m]);
      rem /= (unsigned)reg.n[m];
    }
    const float4 b01 = reinterpret_cast<const float4*>(rhs + idx)[0];
    const float4 b23 = reinterpret_cast<const float4*>(rhs + idx)[1];
    const float4 k01 = reinterpret_cast<const float4*>(kx + idx)[0];
    const float4 k23 = reinterpret_cast<const float4*>(kx + idx)[1];
    const float2 bv[4] = {{b01.x, b01.y}, {b01.z, b01.w}, {b23.x, b23.y}, {b23.z, b23.w}};
    const float2 kv[4] = {{k01.x, k01.y}, {k01.z, k01.w}, {k23.x, k23.y}, {k23.z, k23.w}};
    Acc2 acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc[i].add(1.f, 0.f, bv[i].x, bv[i].y);
      acc[i].add(-1.f, 0.f, kv[i].x, kv[i].y);
    }
    const float4 xc4 = *reinterpret_cast<const float4*>(x + idx);
    const float xc[4] = {xc4.x, xc4.y, xc4.z, xc4.w};
#pragma unroll
    for (int m = kMaxModes - 1; m >= 0; --m) {
      if (!reg.w[m]) continue;
      if (m == L) {
        // Window x[idx - 4 .. idx + 8) along the run's own fibre.
        const int nL = (int)reg.n[m];
        const float4 lf = im[m] >= 4 ? *reinterpret_cast<const float4*>(x + idx - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 rf = im[m] + 4 < nL ? *reinterpret_cast<const float4*>(x + idx + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float win[12] = {lf.x, lf.y, lf.z, lf.w, xc[0], xc[1], xc[2], xc[3], rf.x, rf.y, rf.z, rf.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int row = im[m] + i;
          const float2* wm = reg.w[m] + (int64_t)row * 5;
#pragma unroll
          for (int e = 0; e < 5; ++e) {
            const int c = row - 2 + e;
            if (c >= 0 && c < nL) {
              const float2 cf = wm[e];
              acc[i].add_x(-cf.x, -cf.y, win[i + 2 + e]);
            }
          }
        }
      } else {
        const float2* wm = reg.w[m] + (int64_t)im[m] * 5;
#pragma unroll
        for (int e = 0; e < 5; ++e) {
          const int c = im[m] - 2 + e;
          if (c >= 0 && c < reg.n[m]) {
            const float2 cf = wm[e];
            float xv[4];
            if (e == 2) {
#pragma unroll
              for (int i = 0; i < 4; ++i) xv[i] = xc[i];
            } else {
              const float4 t = __ldg(reinterpret_cast<const float4*>(x + idx + (int64_t)(e - 2) * reg.stride[m]));
              xv[0] = t.x; xv[1] = t.y; xv[2] = t.z; xv[3] = t.w;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i].add_x(-cf.x, -cf.y, xv[i]);
          }
        }
      }
    }
    float ro[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 rv = acc[i].result();
      ro[i] = rv.x;
      const double rd = (double)rv.x + (double)rv.y;
      a_rr += rd * rd;
      const double bd = (double)bv[i].x + (double)bv[i].y;
      a_bb += bd * bd;
    }
    if (r_out) *reinterpret_cast<float4*>(r_out + idx) = make_float4(ro[0], ro[1], ro[2], ro[3]);
  }
  double t_rr, t_bb;
  const bool l1 = dev::grid_sum_last(a_rr, red, &t_rr, sh);
  if (l1) red2.partials[red2.max_blocks - 1] = t_rr;  // park the first total past the used slots
  const bool l2 = dev::grid_sum_last(a_bb, red2, &t_bb, sh);
  if (l2) {
    __threadfence();
    // Relative norm; the absolute one when the right-hand side is zero (0 for x = 0).
    const double rr = sqrt(((volatile double*)red2.partials)[red2.max_blocks - 1]);
    sc->aux = t_bb > 0.0 ? rr / sqrt(t_bb) : rr;
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
  const auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) % 16) == 0; };
  const bool aligned = al16(x) && al16(y) && (!y32 || al16(y32));
  if (I >= 32 && I % 4 == 0 && aligned) {
    const int64_t ich = (I / 4 + 63) / 64;
    const int jch = (n_out + 15) / 16;
    band_ff_inner4_kernel<Tin><<<(unsigned)(O * ich * jch), dim3(64, 4), 0, s>>>(x, y, y32, n_in, n_out, I, start,
                                                                                 w, W, ich, jch, 0, n_out);
  } else if (I >= 32) {
    const int64_t ich = (I + 63) / 64;
    const int jch = (n_out + 31) / 32;
    band_ff_inner_kernel<Tin><<<(unsigned)(O * ich * jch), dim3(64, 4), 0, s>>>(x, y, y32, O, n_in, n_out, I, start,
                                                                                w, W, ich, jch);
  } else {
    const size_t per = sizeof(Tin) * (size_t)n_in * (size_t)I;
    if (per > 200 * 1024) return TCA_ERR_UNSUPPORTED;
    int To = (int)std::max<size_t>(1, std::min<size_t>(256, (32 * 1024) / per));
    if ((int64_t)To > O) To = (int)O;
    const size_t buf = (per * To + 15) / 16 * 16;
    const int stages = 2 * buf <= 200 * 1024 ? 2 : 1;
    const size_t sm = buf * stages;
    const bool vec = (per % 16) == 0 && (reinterpret_cast<uintptr_t>(x) % 16) == 0;
    const int64_t tiles = (O + To - 1) / To;
    static int sms = 0;
    if (!sms) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 1;
    }
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)sms * 3);
    // Four-lane modes need 16-byte aligned rows in shared memory and output.
    const int mode = (I % 4 == 0 && vec && aligned) ? 1 : (I == 1 ? 2 : 0);
    auto k = mode == 1 ? band_ff_outer_kernel<Tin, true, 1>
                       : (mode == 2 ? (vec ? band_ff_outer_kernel<Tin, true, 2> : band_ff_outer_kernel<Tin, false, 2>)
                                    : (vec ? band_ff_outer_kernel<Tin, true, 0> : band_ff_outer_kernel<Tin, false, 0>));
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k<<<(unsigned)grid, 256, sm, s>>>(x, y, y32, O, n_in, n_out, (int)I, start, w, W, To, stages);
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

// A^T b for a host b (FP32), overlapped with its upload, in the plan's own
// mode order and arithmetic (bit-identical to chain_ff on a device copy of b).
// The first product of that order must run on the inner layout with O = 1
// (its mode is the outermost).  b arrives in `chunks` contiguous runs of that
// mode's rows (one copy each on cs, each with an event); after each run, the
// output rows of the first product whose band lies entirely in the rows
// received so far are computed, and so are those rows' slabs of every later
// product (the other modes act within a slab of the outermost index), so the
// chain trails the upload by one run.  TCA_ERR_UNSUPPORTED when the first
// product is not of that form (the caller uploads b whole).
tca_status chain_ff_rhs_from_host(tca_plan_s* p, const float* b_host, float* b_stage, float2* y, float* y32,
                                  float2* const* ws, int64_t ws_elems, cudaStream_t s, cudaStream_t cs,
                                  cudaEvent_t* ev, int chunks) {
  const int d = p->d;
  if (d < 2) return TCA_ERR_UNSUPPORTED;
  const int k0 = p->order_bwd[0];
  const ModeOp& op0 = p->mode[k0].bwd;
  if (k0 != 0 || op0.kind != OP_BAND || (int64_t)op0.band.start_host.size() != op0.band.n_out)
    return TCA_ERR_UNSUPPORTED;
  // Extents after each step and the per-step geometry (O and I per unit of the outermost index).
  int64_t cur[kMaxModes];
  for (int k = 0; k < d; ++k) cur[k] = p->m[k];
  int64_t Pk[kMaxModes], Ik[kMaxModes];
  int nin[kMaxModes], nout[kMaxModes];
  for (int st = 0; st < d; ++st) {
    const int k = p->order_bwd[st];
    const ModeOp& op = p->mode[k].bwd;
    int64_t P = 1, I = 1;
    for (int a = 1; a < k; ++a) P *= cur[a];
    for (int a = k + 1; a < d; ++a) I *= cur[a];
    Pk[st] = P;
    Ik[st] = I;
    nin[st] = (int)op.n_in();
    nout[st] = (int)op.n_out();
    cur[k] = nout[st];
    if (st < d - 1 && (k == 0 ? 1 : cur[0]) * P * I * nout[st] > ws_elems) return TCA_ERR_UNSUPPORTED;
  }
  const int64_t I0 = Ik[0];
  const int n_in0 = nin[0], n_out0 = nout[0];
  const auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) % 16) == 0; };
  if (I0 % 4 != 0 || I0 < 32 || n_in0 < chunks || !al16(b_stage) || !al16(ws[0]) || !al16(b_host))
    return TCA_ERR_UNSUPPORTED;
  const std::vector<int32_t>& st0 = op0.band.start_host;
  const int W0 = op0.band.W;
  const int64_t ich = (I0 / 4 + 63) / 64;
  int j_done = 0;
  for (int c = 0; c < chunks; ++c) {
    const int64_t r0 = (int64_t)n_in0 * c / chunks, r1 = (int64_t)n_in0 * (c + 1) / chunks;
    if (r1 <= r0) continue;
    TCA_CUDA_TRY(cudaMemcpyAsync(b_stage + r0 * I0, b_host + r0 * I0, sizeof(float) * (size_t)((r1 - r0) * I0),
                                 cudaMemcpyHostToDevice, cs));
    TCA_CUDA_TRY(cudaEventRecord(ev[c], cs));
    TCA_CUDA_TRY(cudaStreamWaitEvent(s, ev[c], 0));
    // Output rows whose taps (clipped to [0, n_in)) lie below row r1.
    int j_hi = j_done;
    if (c == chunks - 1) {
      j_hi = n_out0;
    } else {
      while (j_hi < n_out0 && std::min<int64_t>((int64_t)st0[j_hi] + W0, n_in0) <= r1) ++j_hi;
    }
    if (j_hi <= j_done) continue;
    const int jch = (j_hi - j_done + 15) / 16;
    band_ff_inner4_kernel<float><<<(unsigned)(ich * jch), dim3(64, 4), 0, s>>>(
        b_stage, ws[0], nullptr, n_in0, n_out0, I0, op0.band.start, op0.band.wff, W0, ich, jch, j_done, j_hi);
    TCA_LAUNCH_CHECK();
    // The slabs j_done .. j_hi - 1 of the outermost index through the other modes.
    const int64_t nj = j_hi - j_done;
    const float2* src = ws[0];
    for (int st = 1; st < d; ++st) {
      const int k = p->order_bwd[st];
      const bool last = st == d - 1;
      float2* dst = last ? y : ws[st % 2];
      const int64_t in_slab = Pk[st] * nin[st] * Ik[st], out_slab = Pk[st] * nout[st] * Ik[st];
      const int32_t* start;
      const float2* w;
      int W;
      op_band_ff(p->mode[k].bwd, &start, &w, &W);
      TCA_TRY(launch_ff<float2>(start, w, W, nin[st], nout[st], src + j_done * in_slab, dst + j_done * out_slab,
                                last ? y32 + j_done * out_slab : nullptr, nj * Pk[st], Ik[st], s));
      src = dst;
    }
    j_done = j_hi;
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
  const int L = p->d - 1;
  const auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) % 16) == 0; };
  if (p->n[L] % 4 == 0 && al16(x) && al16(rhs_ff) && al16(kx_ff) && (!r_out || al16(r_out))) {
    auto k = L == 3 ? residual_ff_vec_kernel<3>
                    : (L == 2 ? residual_ff_vec_kernel<2> : (L == 1 ? residual_ff_vec_kernel<1> : residual_ff_vec_kernel<0>));
    k<<<grid, 256, 0, s>>>(rhs_ff, kx_ff, x, r_out, p->N, reg, p->scal, red, red2);
  } else {
    residual_ff_kernel<<<grid, 256, 0, s>>>(rhs_ff, kx_ff, x, r_out, p->N, reg, p->scal, red, red2);
  }
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace tca
