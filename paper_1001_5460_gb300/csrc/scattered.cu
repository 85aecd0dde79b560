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
// Tiling.  The unknown grid is cut into tiles of anchor cells (a sample's
// anchor in mode k is col0_k + 1, clamped to the grid: its window col0 ..
// col0 + 3 starts one cell before it).  At plan time the samples are grouped
// by tile (a counting sort); the caller's order is kept at the boundary
// (apply, apply_T, b) by a permutation.  One CTA takes one tile and works in a
// shared-memory image of the tile's region - its anchor cells plus the cells
// their windows reach, at most kRegionMax elements:
//   gather:  the region of x is copied in once, then every sample of the tile
//            sums its window from shared memory;
//   scatter: every sample of the tile adds its window into the shared image
//            (shared-memory atomics), then the image is added to x with one
//            global atomic per nonzero region cell - instead of 4^d global
//            atomics per sample.
// Inside a tile the samples are ordered so that the 32 samples a warp takes
// together start their windows on distinct shared-memory banks
// (order_for_banks).  Per sample the window's weights are applied mode by
// mode (the separable window): gather sums the innermost mode first and folds
// the sums outwards (4^d + 4^(d-1) + .. + 4 fused multiply-adds), scatter
// forms the outer products outwards (the same count of multiplications).
// FP64 on every scattered plan (the operators of TCA_F64 plans and the true
// residual of TCA_F32 plans); FP32 on TCA_F32 plans.  The atomic additions make
// the order of the additions to one unknown vary from run to run in its last
// bits.
#include <algorithm>
#include <numeric>
#include <vector>

#include "tca_internal.cuh"

namespace tca {

namespace {

constexpr int kThreads = 256;
// Largest shared-memory region of a tile, in elements of the plan's type
// (48 KB in FP32, 96 KB in FP64).
constexpr int64_t kRegionMax = 12288;

template <typename T>
struct ScatArgs {
  int n[4];           // grid extents (1 beyond the plan's order)
  int ts[4], nt[4];   // tile extent (anchor cells) and tile count per mode
  int64_t m;
  const int32_t* col0;        // [k][m], grouped order
  const T* w;                 // [k][m][4]
  const int32_t* tile_start;  // [tiles + 1]
  const int32_t* perm;        // grouped position -> caller's sample index, or null (grouped order)
};

// A tile's region: per mode the cells [lo, lo + R) that its samples' windows
// can reach inside the grid, and the region's strides (mode 3 fastest).
struct Region {
  int lo[4], R[4];
  int S0, S1, S2;
  int total;
};

template <typename T>
__device__ __forceinline__ Region region_of(const ScatArgs<T>& a, int64_t tile) {
  Region r;
  int t[4];
  int64_t q = tile;
#pragma unroll
  for (int k = 3; k >= 0; --k) {
    t[k] = (int)(q % a.nt[k]);
    q /= a.nt[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // Anchors t ts .. t ts + ts - 1 reach cells anchor - 1 .. anchor + 2.
    const int lo = max(0, t[k] * a.ts[k] - 1);
    const int hi = min(a.n[k] - 1, t[k] * a.ts[k] + a.ts[k] + 1);
    r.lo[k] = lo;
    r.R[k] = hi - lo + 1;
  }
  r.S2 = r.R[3];
  r.S1 = r.R[2] * r.S2;
  r.S0 = r.R[1] * r.S1;
  r.total = r.R[0] * r.S0;
  return r;
}

// Calls f(e, g) for every region element e (flat, mode 3 fastest) handled by
// this thread (e = tid, tid + blockDim, ..) with g its index in the grid
// tensor.  The region digits of e advance by mixed-radix addition of the
// block size: no division inside the loop.
template <typename F>
__device__ __forceinline__ void walk_region(const Region& r, const int* n, F&& f) {
  const int B = blockDim.x;
  int q = threadIdx.x;
  int d3 = q % r.R[3];
  q /= r.R[3];
  int d2 = q % r.R[2];
  q /= r.R[2];
  int d1 = q % r.R[1];
  int d0 = q / r.R[1];
  int qb = B;
  const int b3 = qb % r.R[3];
  qb /= r.R[3];
  const int b2 = qb % r.R[2];
  qb /= r.R[2];
  const int b1 = qb % r.R[1];
  const int b0 = qb / r.R[1];
  for (int e = threadIdx.x; e < r.total; e += B) {
    const int64_t g =
        (((int64_t)(r.lo[0] + d0) * n[1] + (r.lo[1] + d1)) * n[2] + (r.lo[2] + d2)) * n[3] + (r.lo[3] + d3);
    f(e, g);
    // digit + step + carry <= 2 R - 1: one subtraction wraps each digit
    d3 += b3;
    int c = d3 >= r.R[3];
    if (c) d3 -= r.R[3];
    d2 += b2 + c;
    c = d2 >= r.R[2];
    if (c) d2 -= r.R[2];
    d1 += b1 + c;
    c = d1 >= r.R[1];
    if (c) d1 -= r.R[1];
    d0 += b0 + c;
  }
}

// One sample's window relative to the tile's region: per mode and tap the
// region offset of the tap's cell (clamped into the region) and the tap's
// weight, zeroed for a tap outside the region - so every window is 4^d taps
// with no branch per tap (a zeroed tap reads or adds 0 at a cell that the
// sample's valid taps in that mode also reach).  Returns false when some mode
// has no tap in the region (the sample touches nothing).
template <typename T, int D>
__device__ __forceinline__ bool load_sample(const ScatArgs<T>& a, const Region& r, int s, int (&off)[4][4],
                                            T (&w)[4][4]) {
  const int st[4] = {r.S0, r.S1, r.S2, 1};
  bool any = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k < D) {
      const int l = a.col0[(int64_t)k * a.m + s] - r.lo[k];  // region cell of tap 0
      T v[4];
      const T* wp = a.w + ((int64_t)k * a.m + s) * 4;
      if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(wp);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
      } else {
        const double2 q0 = reinterpret_cast<const double2*>(wp)[0];
        const double2 q1 = reinterpret_cast<const double2*>(wp)[1];
        v[0] = q0.x;
        v[1] = q0.y;
        v[2] = q1.x;
        v[3] = q1.y;
      }
      bool in_any = false;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const bool in = (unsigned)(l + t) < (unsigned)r.R[k];
        in_any = in_any || in;
        off[k][t] = min(max(l + t, 0), r.R[k] - 1) * st[k];
        w[k][t] = in ? v[t] : T(0);
      }
      any = any && in_any;
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        off[k][t] = 0;
        w[k][t] = t == 0 ? T(1) : T(0);
      }
    }
  }
  return any;
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads) gather_tiled_kernel(const ScatArgs<T> a, const T* __restrict__ x,
                                                                T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sx = reinterpret_cast<T*>(smem_raw);
  const int64_t tile = blockIdx.x;
  const int s_begin = a.tile_start[tile], s_end = a.tile_start[tile + 1];
  if (s_begin == s_end) return;
  const Region r = region_of(a, tile);
  walk_region(r, a.n, [&](int e, int64_t g) { sx[e] = x[g]; });
  __syncthreads();
  for (int s = s_begin + (int)threadIdx.x; s < s_end; s += blockDim.x) {
    int off[4][4];
    T w[4][4];
    T acc = T(0);
    if (load_sample<T, D>(a, r, s, off, w)) {
#pragma unroll
      for (int a0 = 0; a0 < 4; ++a0) {
        T s1 = T(0);
#pragma unroll
        for (int a1 = 0; a1 < 4; ++a1) {
          T s2 = T(0);
#pragma unroll
          for (int a2 = 0; a2 < 4; ++a2) {
            const T* row = sx + off[0][a0] + off[1][a1] + off[2][a2];
            T s3;
            if constexpr (D == 4) {
              s3 = T(0);
#pragma unroll
              for (int a3 = 0; a3 < 4; ++a3) s3 = fma(w[3][a3], row[off[3][a3]], s3);
            } else {
              s3 = row[0];
            }
            s2 = fma(w[2][a2], s3, s2);
          }
          s1 = fma(w[1][a1], s2, s1);
        }
        acc = fma(w[0][a0], s1, acc);
      }
    }
    y[a.perm ? a.perm[s] : s] = acc;
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads) scatter_tiled_kernel(const ScatArgs<T> a, const T* __restrict__ y,
                                                                 T* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sx = reinterpret_cast<T*>(smem_raw);
  const int64_t tile = blockIdx.x;
  const int s_begin = a.tile_start[tile], s_end = a.tile_start[tile + 1];
  if (s_begin == s_end) return;
  const Region r = region_of(a, tile);
  for (int e = threadIdx.x; e < r.total; e += blockDim.x) sx[e] = T(0);
  __syncthreads();
  for (int s = s_begin + (int)threadIdx.x; s < s_end; s += blockDim.x) {
    int off[4][4];
    T w[4][4];
    const T ys = y[a.perm ? a.perm[s] : s];
    if (!load_sample<T, D>(a, r, s, off, w)) continue;
#pragma unroll
    for (int a0 = 0; a0 < 4; ++a0) {
      const T c0 = ys * w[0][a0];
#pragma unroll
      for (int a1 = 0; a1 < 4; ++a1) {
        const T c1 = c0 * w[1][a1];
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) {
          const T c2 = c1 * w[2][a2];
          T* row = sx + off[0][a0] + off[1][a1] + off[2][a2];
          if constexpr (D == 4) {
#pragma unroll
            for (int a3 = 0; a3 < 4; ++a3) atomicAdd(row + off[3][a3], c2 * w[3][a3]);
          } else {
            atomicAdd(row, c2);
          }
        }
      }
    }
  }
  __syncthreads();
  walk_region(r, a.n, [&](int e, int64_t g) {
    const T v = sx[e];
    if (v != T(0)) atomicAdd(x + g, v);
  });
}

template <typename T>
const T* weights_of(const tca_plan_s* p) {
  if constexpr (sizeof(T) == 4) return p->sc_w32;
  else return p->sc_w;
}

template <typename T>
ScatArgs<T> args_of(const tca_plan_s* p, bool perm) {
  ScatArgs<T> a;
  for (int k = 0; k < 4; ++k) {
    a.n[k] = k < p->d ? (int)p->n[k] : 1;
    a.ts[k] = p->sc_ts[k];
    a.nt[k] = p->sc_nt[k];
  }
  a.m = p->sc_m;
  a.col0 = p->sc_col0;
  a.w = weights_of<T>(p);
  a.tile_start = p->sc_tile_start;
  a.perm = perm ? p->sc_perm : nullptr;
  return a;
}

// Dynamic shared memory above 48 KB needs the kernel's opt-in: once per
// kernel, for the largest region any plan can have.
template <typename T, typename K>
tca_status smem_opt_in(K kernel, size_t bytes, bool* done) {
  if (*done || bytes <= 48 * 1024) return TCA_OK;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(T) * kRegionMax));
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_CUDA;
  }
  *done = true;
  return TCA_OK;
}

// Tile extents: modes of at most 16 cells are not cut; the others share one
// extent, the largest whose region fits kRegionMax.  Should that not fit
// (several uncut modes), every mode is cut alike.
void choose_tiles(const int64_t* n, int d, int* ts) {
  auto region = [&](const int* t) {
    int64_t r = 1;
    for (int k = 0; k < d; ++k) r *= std::min<int64_t>(t[k] + 3, n[k]);
    return r;
  };
  for (int u = 64; u >= 1; --u) {
    for (int k = 0; k < d; ++k) ts[k] = n[k] <= 16 ? (int)n[k] : u;
    if (region(ts) <= kRegionMax) return;
  }
  for (int u = 16; u >= 1; --u) {
    for (int k = 0; k < d; ++k) ts[k] = (int)std::min<int64_t>(u, n[k]);
    if (region(ts) <= kRegionMax) return;
  }
}

// Order the samples inside each tile so that the 32 samples one warp takes
// together (tile-relative positions 32 g .. 32 g + 31) start their windows on
// distinct shared-memory banks: an interior sample's taps all lie at the same
// offsets from its window start, so a warp's accesses for one tap hit 32
// distinct banks (FP32; FP64 elements take two banks each, so each half-warp
// gets 16 distinct bank pairs) - no bank conflicts in the gather's loads, and
// no conflicts or same-address retries inside a warp in the scatter's atomic
// additions.  A sample's bank class is its window start's region offset,
// computed as the kernels compute it; classes are taken round-robin, and a
// group that runs out of distinct classes is filled from the largest classes.
void order_for_banks(const int64_t* n, int d, const int* ts, const int* nt, const tca_factor* rows, int classes,
                     const std::vector<int64_t>& start, std::vector<int32_t>& perm) {
  const int64_t tiles = (int64_t)start.size() - 1;
  std::vector<std::vector<int32_t>> bucket((size_t)classes);
  std::vector<size_t> head((size_t)classes);
  for (int64_t t = 0; t < tiles; ++t) {
    const int64_t b = start[(size_t)t], e = start[(size_t)t + 1];
    if (e - b <= 1) continue;
    // The tile's region, as region_of forms it (modes past the order have extent 1).
    int lo[kMaxModes], R[kMaxModes], tk[kMaxModes];
    int64_t q = t;
    for (int k = kMaxModes - 1; k >= 0; --k) {
      const int ntk = k < d ? nt[k] : 1;
      tk[k] = (int)(q % ntk);
      q /= ntk;
    }
    for (int k = 0; k < kMaxModes; ++k) {
      const int64_t nk = k < d ? n[k] : 1, tsk = k < d ? ts[k] : 1;
      lo[k] = (int)std::max<int64_t>(0, tk[k] * tsk - 1);
      R[k] = (int)(std::min<int64_t>(nk - 1, tk[k] * tsk + tsk + 1) - lo[k] + 1);
    }
    const int64_t st[kMaxModes] = {(int64_t)R[1] * R[2] * R[3], (int64_t)R[2] * R[3], R[3], 1};
    for (auto& v : bucket) v.clear();
    std::fill(head.begin(), head.end(), 0);
    for (int64_t i = b; i < e; ++i) {
      const int32_t s = perm[(size_t)i];
      int64_t base = 0;
      for (int k = 0; k < d; ++k) {
        const int64_t l = (int64_t)rows[k].col0[s] - lo[k];
        if (l >= -3 && l < R[k]) base += l * st[k];
      }
      bucket[(size_t)(((base % classes) + classes) % classes)].push_back(s);
    }
    int64_t out = b;
    const int per_pass = classes;  // distinct classes per pass (a warp, or a half-warp in FP64)
    while (out < e) {
      for (int pass = 0; pass < 32 / per_pass && out < e; ++pass) {
        int took = 0;
        for (int c = 0; c < classes && out < e; ++c) {
          if (head[(size_t)c] < bucket[(size_t)c].size()) {
            perm[(size_t)out++] = bucket[(size_t)c][head[(size_t)c]++];
            ++took;
          }
        }
        // Too few distinct classes left: fill the pass from the largest classes.
        while (took < per_pass && out < e) {
          size_t best = 0, left = 0;
          for (int c = 0; c < classes; ++c) {
            const size_t r = bucket[(size_t)c].size() - head[(size_t)c];
            if (r > left) {
              left = r;
              best = (size_t)c;
            }
          }
          perm[(size_t)out++] = bucket[best][head[best]++];
          ++took;
        }
      }
    }
  }
}

}  // namespace

template <typename T>
tca_status scattered_gather(const tca_plan_s* p, const T* x, T* y, bool perm, cudaStream_t s) {
  if (p->sc_m == 0) return TCA_OK;
  if (!weights_of<T>(p)) return TCA_ERR_UNSUPPORTED;
  const ScatArgs<T> a = args_of<T>(p, perm);
  const size_t bytes = sizeof(T) * (size_t)p->sc_region;
  if (p->d == 4) {
    static bool done = false;
    TCA_TRY(smem_opt_in<T>(gather_tiled_kernel<T, 4>, bytes, &done));
    gather_tiled_kernel<T, 4><<<(unsigned)p->sc_tiles, kThreads, bytes, s>>>(a, x, y);
  } else {
    static bool done = false;
    TCA_TRY(smem_opt_in<T>(gather_tiled_kernel<T, 3>, bytes, &done));
    gather_tiled_kernel<T, 3><<<(unsigned)p->sc_tiles, kThreads, bytes, s>>>(a, x, y);
  }
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template <typename T>
tca_status scattered_scatter(const tca_plan_s* p, const T* y, T* x, bool perm, cudaStream_t s) {
  TCA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * (size_t)p->N, s));
  if (p->sc_m == 0) return TCA_OK;
  if (!weights_of<T>(p)) return TCA_ERR_UNSUPPORTED;
  const ScatArgs<T> a = args_of<T>(p, perm);
  const size_t bytes = sizeof(T) * (size_t)p->sc_region;
  if (p->d == 4) {
    static bool done = false;
    TCA_TRY(smem_opt_in<T>(scatter_tiled_kernel<T, 4>, bytes, &done));
    scatter_tiled_kernel<T, 4><<<(unsigned)p->sc_tiles, kThreads, bytes, s>>>(a, y, x);
  } else {
    static bool done = false;
    TCA_TRY(smem_opt_in<T>(scatter_tiled_kernel<T, 3>, bytes, &done));
    scatter_tiled_kernel<T, 3><<<(unsigned)p->sc_tiles, kThreads, bytes, s>>>(a, y, x);
  }
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template tca_status scattered_gather<float>(const tca_plan_s*, const float*, float*, bool, cudaStream_t);
template tca_status scattered_gather<double>(const tca_plan_s*, const double*, double*, bool, cudaStream_t);
template tca_status scattered_scatter<float>(const tca_plan_s*, const float*, float*, bool, cudaStream_t);
template tca_status scattered_scatter<double>(const tca_plan_s*, const double*, double*, bool, cudaStream_t);

// Attach the scattered rows to a plan built over the grid (with identity
// per-mode factors, which give it the regulariser bands and workspace):
// validate, group the samples by tile, order them for the banks, upload.
tca_status scattered_attach(tca_plan_s* p, int64_t m, const tca_factor* rows) {
  const int d = p->d;
  for (int k = 0; k < d; ++k) {
    if (rows[k].kind != TCA_FACTOR_ELL4 || !rows[k].col0 || !rows[k].values || rows[k].reserved != 0)
      return TCA_ERR_INVALID_ARG;
    if (rows[k].m != m || rows[k].n != p->n[k]) return TCA_ERR_SHAPE;
  }
  if (m > INT32_MAX) return TCA_ERR_UNSUPPORTED;
  // Tiles of anchor cells and each sample's tile.
  int ts[kMaxModes], nt[kMaxModes];
  choose_tiles(p->n, d, ts);
  int64_t tiles = 1, region = 1;
  for (int k = 0; k < kMaxModes; ++k) {
    if (k < d) {
      nt[k] = (int)((p->n[k] + ts[k] - 1) / ts[k]);
      region *= std::min<int64_t>(ts[k] + 3, p->n[k]);
    } else {
      ts[k] = nt[k] = 1;
    }
    tiles *= nt[k];
  }
  if (tiles > INT32_MAX) return TCA_ERR_UNSUPPORTED;
  std::vector<int32_t> tile_of((size_t)m);
  std::vector<int64_t> start((size_t)tiles + 1, 0);
  for (int64_t s = 0; s < m; ++s) {
    int64_t t = 0;
    for (int k = 0; k < d; ++k) {
      const int64_t anchor = std::min<int64_t>(std::max<int64_t>((int64_t)rows[k].col0[s] + 1, 0), p->n[k] - 1);
      t = t * nt[k] + anchor / ts[k];
    }
    tile_of[(size_t)s] = (int32_t)t;
    ++start[(size_t)t + 1];
  }
  for (int64_t t = 0; t < tiles; ++t) start[(size_t)t + 1] += start[(size_t)t];
  std::vector<int32_t> perm((size_t)m), tstart((size_t)tiles + 1);
  for (int64_t t = 0; t <= tiles; ++t) tstart[(size_t)t] = (int32_t)start[(size_t)t];
  {
    std::vector<int64_t> next(start.begin(), start.end() - 1);
    for (int64_t s = 0; s < m; ++s) perm[(size_t)next[(size_t)tile_of[(size_t)s]]++] = (int32_t)s;
  }
  order_for_banks(p->n, d, ts, nt, rows, p->prec == TCA_F64 ? 16 : 32, start, perm);
  std::vector<int32_t> c0((size_t)d * m);
  std::vector<double> w((size_t)d * m * 4);
  for (int64_t s = 0; s < m; ++s) {
    const int64_t src = perm[(size_t)s];
    for (int k = 0; k < d; ++k) {
      // A window that starts at or below -4, or at or past n, has no tap in the
      // grid: clamping its start to [-4, n] changes nothing and keeps every
      // index the kernels form from it small.
      c0[(size_t)(k * m + s)] = (int32_t)std::min<int64_t>(std::max<int64_t>(rows[k].col0[src], -4), p->n[k]);
      for (int a = 0; a < 4; ++a) w[(size_t)((k * m + s) * 4 + a)] = rows[k].values[src * 4 + a];
    }
  }
  p->sc_m = m;
  p->sc_tiles = tiles;
  p->sc_region = region;
  for (int k = 0; k < kMaxModes; ++k) {
    p->sc_ts[k] = ts[k];
    p->sc_nt[k] = nt[k];
  }
  cudaError_t e = cudaMalloc((void**)&p->sc_tile_start, sizeof(int32_t) * tstart.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(p->sc_tile_start, tstart.data(), sizeof(int32_t) * tstart.size(), cudaMemcpyHostToDevice);
  if (m > 0) {
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->sc_col0, sizeof(int32_t) * c0.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->sc_w, sizeof(double) * w.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->sc_perm, sizeof(int32_t) * perm.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->sc_tmp, sizeof(double) * (size_t)m);
    if (e == cudaSuccess) e = cudaMemcpy(p->sc_col0, c0.data(), sizeof(int32_t) * c0.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->sc_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->sc_perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && p->prec == TCA_F32) {
      std::vector<float> w32(w.begin(), w.end());
      e = cudaMalloc((void**)&p->sc_w32, sizeof(float) * w32.size());
      if (e == cudaSuccess) e = cudaMemcpy(p->sc_w32, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  p->scattered = true;
  p->fused_ok = false;  // the grid plan's identity factors are not the operator
  p->M = m;
  return TCA_OK;
}

void scattered_release(tca_plan_s* p) {
  cudaFree(p->sc_col0);
  cudaFree(p->sc_w);
  cudaFree(p->sc_w32);
  cudaFree(p->sc_perm);
  cudaFree(p->sc_tile_start);
  cudaFree(p->sc_tmp);
  p->sc_col0 = nullptr;
  p->sc_w = nullptr;
  p->sc_w32 = nullptr;
  p->sc_perm = nullptr;
  p->sc_tile_start = nullptr;
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
  if (prec != TCA_F64 && prec != TCA_F32) {
    set_error_message("scattered plans compute in FP64 (TCA_F64) or FP32 (TCA_F32)");
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
