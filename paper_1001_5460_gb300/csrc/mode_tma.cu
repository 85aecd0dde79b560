// Single-mode banded products (one one-dimensional transformation of Eq.
// separable_transf) - the streaming kernels behind tca_apply, tca_apply_T,
// tca_apply_mode and the unfused normal operator.
//
// Row tiles (inner extent I a multiple of 4), TMA-staged: the tensor is viewed
// as a 3D array (I, n_in, O), innermost first.  A tile holds To outer slabs, Ti
// inner elements and the input rows read by kJB consecutive outputs along the
// mode.  One cp.async.bulk.tensor copies it into shared memory, completing on
// an mbarrier; rows outside [0, n_in) arrive as zeros, which is exactly the
// band's boundary.  Threads read 16-byte vectors along the inner index and
// write coalesced output rows.  The grid is k CTAs per SM (default 3,
// TCA_ROWS_CTAS_PER_SM overrides; 0 = one tile per CTA) and each CTA walks its
// tiles through a ring of up to 3 buffers, refilled as soon as a tile is done.  Waits on an
// mbarrier are bounded: a CTA that gives up sets g_wait_timeout (reported by
// tca_solve as TCA_ERR_TIMEOUT) and leaves uniformly.
//
// Fastest mode (I = 1, n_in and n_out small): the tiny band matrix is held
// densely in registers (static indices only) and each thread streams whole
// fibres with 16-byte loads and stores in a grid-stride loop.
#include <cuda.h>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "tca_internal.cuh"

namespace tca {

// Set by any kernel whose bounded wait gave up; read by tca_solve.
__device__ int g_wait_timeout = 0;

namespace {

constexpr int kThreads = 256;
constexpr int kJB = 32;                      // outputs per row tile along the mode
constexpr int kMaxStages = 12;               // deepest ring of a persistent CTA
constexpr long long kWaitLimit = 1ll << 26;  // mbarrier polls before giving up (seconds)

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ float* align128(unsigned char* p) {
  return reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
}

struct RowGeom {
  int64_t O, I, i_chunks, tiles;
  int n_in, n_out, W, Ti, To, RB, j_chunks, stage_floats, stages;
  int unit;  // 7-wide band with start[j] = start[0] + j: sliding-window path
};

// Sliding window over consecutive outputs of a unit-step 7-wide band: the JPG
// outputs j0 .. j0 + JPG - 1 of a thread read rows rs .. rs + JPG + 5 of the
// tile once (JPG + 6 loads instead of 7 JPG).
template <int JPG>
__device__ __forceinline__ void rows_window7(const float* ts, int Ti, int RB, int rs, int j0, int n_out,
                                             const float* __restrict__ w, float* yo, int64_t I, bool ok) {
  float4 win[JPG + 6];
  // Rows past the tile (RB rows) only feed outputs past n_out: never read them.
#pragma unroll
  for (int q = 0; q < JPG + 6; ++q)
    win[q] = rs + q < RB ? *reinterpret_cast<const float4*>(ts + (size_t)(rs + q) * Ti) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int q = 0; q < JPG; ++q) {
    const int j = j0 + q;
    if (j >= n_out) break;
    const float* wj = w + (int64_t)j * 7;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 7; ++e) {
      const float c = __ldg(wj + e);
      acc.x = fmaf(c, win[q + e].x, acc.x);
      acc.y = fmaf(c, win[q + e].y, acc.y);
      acc.z = fmaf(c, win[q + e].z, acc.z);
      acc.w = fmaf(c, win[q + e].w, acc.w);
    }
    if (ok) *reinterpret_cast<float4*>(yo + (int64_t)j * I) = acc;
  }
}

template <bool UNIT>
__global__ void __launch_bounds__(kThreads, 3) band_rows_kernel(const __grid_constant__ CUtensorMap tmap,
                                                             float* __restrict__ y, RowGeom g,
                                                             const int32_t* __restrict__ start,
                                                             const float* __restrict__ w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* base = align128(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + g.stages * g.stage_floats);
  const unsigned bytes = (unsigned)(sizeof(float) * g.Ti * g.RB * g.To);
  auto tile_of = [&](int64_t t, int64_t& oc, int64_t& ic, int& jc) {
    jc = (int)(t % g.j_chunks);
    const int64_t rest = t / g.j_chunks;
    ic = rest % g.i_chunks;
    oc = rest / g.i_chunks;
  };
  auto issue = [&](int64_t t, int buf) {
    int64_t oc, ic;
    int jc;
    tile_of(t, oc, ic, jc);
    mbar_expect(&bars[buf], bytes);
    tma_load_3d(base + buf * g.stage_floats, &tmap, (int)(ic * g.Ti), start[jc * kJB], (int)(oc * g.To), &bars[buf]);
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < g.stages; ++s) mbar_init(&bars[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < g.stages; ++s) {
      const int64_t t = blockIdx.x + (int64_t)s * gridDim.x;
      if (t < g.tiles) issue(t, s);
    }
  const int vl = g.Ti / 4;  // float4 lanes per slab
  const int lanes = vl * g.To;
  const int groups = kThreads / lanes;
  const int lane = threadIdx.x % lanes;
  const int grp = threadIdx.x / lanes;
  const int oo = lane / vl, v = lane % vl;
  for (int64_t k = 0;; ++k) {
    const int64_t t = blockIdx.x + k * gridDim.x;
    if (t >= g.tiles) break;
    const int buf = (int)(k % g.stages);
    const bool arrived = mbar_wait_bounded(&bars[buf], (unsigned)((k / g.stages) & 1));
    int64_t oc, ic;
    int jc;
    tile_of(t, oc, ic, jc);
    const int j0 = jc * kJB;
    const int r0 = start[j0];
    const int64_t o = oc * g.To + oo;
    const int64_t i = ic * g.Ti + 4 * v;
    const bool ok = arrived && grp < groups && o < g.O && i < g.I;
    const float* ts = base + buf * g.stage_floats + (size_t)oo * g.RB * g.Ti + 4 * v;
    float* yo = y + o * (int64_t)g.n_out * g.I + i;
    if (UNIT && grp < groups && (groups == 8 || groups == 4)) {
      // Contiguous outputs per thread group (kJB / groups = 4 or 8 of them).
      const int jpg = kJB / groups;
      const int jg = j0 + grp * jpg;
      const int rs = start[min(jg, g.n_out - 1)] - r0;
      if (jg < g.n_out) {
        if (jpg == 4) rows_window7<4>(ts, g.Ti, g.RB, rs, jg, g.n_out, w, yo, g.I, ok);
        else rows_window7<8>(ts, g.Ti, g.RB, rs, jg, g.n_out, w, yo, g.I, ok);
      }
    } else if (grp < groups) {
      for (int jj = grp; jj < kJB; jj += groups) {
        const int j = j0 + jj;
        if (j >= g.n_out) break;
        const int rs = start[j] - r0;
        const float* wj = w + (int64_t)j * g.W;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = 0; e < g.W; ++e) {
          const float c = __ldg(wj + e);
          const float4 xv = *reinterpret_cast<const float4*>(ts + (size_t)(rs + e) * g.Ti);
          acc.x = fmaf(c, xv.x, acc.x);
          acc.y = fmaf(c, xv.y, acc.y);
          acc.z = fmaf(c, xv.z, acc.z);
          acc.w = fmaf(c, xv.w, acc.w);
        }
        if (ok) *reinterpret_cast<float4*>(yo + (int64_t)j * g.I) = acc;
      }
    }
    // Every thread is done with this buffer; refill it with the tile `stages` ahead.
    if (__syncthreads_or(!arrived)) {
      if (threadIdx.x == 0) atomicExch(&g_wait_timeout, 1);
      return;
    }
    if (threadIdx.x == 0) {
      const int64_t t2 = t + (int64_t)g.stages * gridDim.x;
      if (t2 < g.tiles) issue(t2, buf);
    }
  }
}

// Fastest mode: y[o][j] = sum_l D[j][l] x[o][l] with the band expanded to a
// dense NOUT x NIN matrix held in registers.
template <int NIN, int NOUT>
__global__ void __launch_bounds__(kThreads) band_fibre_kernel(const float* __restrict__ x, float* __restrict__ y,
                                                              int64_t O, const int32_t* __restrict__ start,
                                                              const float* __restrict__ w, int W) {
  float d[NOUT][NIN];
#pragma unroll
  for (int j = 0; j < NOUT; ++j) {
    const int s0 = __ldg(start + j);
#pragma unroll
    for (int l = 0; l < NIN; ++l) {
      const int e = l - s0;
      d[j][l] = (e >= 0 && e < W) ? __ldg(w + j * W + e) : 0.f;
    }
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < O; o += stride) {
    float xf[NIN];
    const float* xo = x + o * NIN;
    if constexpr (NIN % 4 == 0) {
#pragma unroll
      for (int q = 0; q < NIN / 4; ++q) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(xo) + q);
        xf[4 * q] = f.x; xf[4 * q + 1] = f.y; xf[4 * q + 2] = f.z; xf[4 * q + 3] = f.w;
      }
    } else {
#pragma unroll
      for (int l = 0; l < NIN; ++l) xf[l] = __ldg(xo + l);
    }
    float yf[NOUT];
#pragma unroll
    for (int j = 0; j < NOUT; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int l = 0; l < NIN; ++l) acc = fmaf(d[j][l], xf[l], acc);
      yf[j] = acc;
    }
    float* yo = y + o * NOUT;
    if constexpr (NOUT % 4 == 0) {
#pragma unroll
      for (int q = 0; q < NOUT / 4; ++q)
        reinterpret_cast<float4*>(yo)[q] = make_float4(yf[4 * q], yf[4 * q + 1], yf[4 * q + 2], yf[4 * q + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < NOUT; ++j) yo[j] = yf[j];
    }
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static std::once_flag once;
  static EncodeFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : dflt;
}

// Row-tile geometry; false when the shape does not fit.
bool row_tile_shape(int64_t O, int64_t I, int RB, int* Ti, int* To) {
  if (I % 4 != 0 || RB <= 0 || RB > 256) return false;
  int ti = (int)std::min<int64_t>(128, I);
  ti = (ti / 4) * 4;
  if (ti <= 0) return false;
  const int lanes = ti / 4;
  int to = 1;
  while (lanes * to < 32 && to < 256 && to < O) to *= 2;  // fill a warp with slabs when I is short
  if (lanes * to > kThreads || kThreads % (lanes * to) != 0) return false;
  if (sizeof(float) * (size_t)ti * RB * to > 40 * 1024) return false;
  *Ti = ti;
  *To = to;
  return true;
}

template <int NIN, int NOUT>
tca_status launch_fibre(const Band& band, const float* x, float* y, int64_t O, cudaStream_t s, int sm_cap) {
  const int64_t want = (O + kThreads - 1) / kThreads;
  const int sms = sm_cap > 0 ? std::min(sm_cap, sm_count()) : sm_count();
  const int64_t grid = std::min<int64_t>(want, (int64_t)sms * 8);
  band_fibre_kernel<NIN, NOUT><<<(unsigned)grid, kThreads, 0, s>>>(x, y, O, band.start, band.w32, band.W);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace

tca_status launch_band_fast(const Band& band, const float* x, float* y, int64_t O, int64_t I, cudaStream_t s,
                            int sm_cap) {
  const int n_in = (int)band.n_in, n_out = (int)band.n_out, W = band.W;
  if ((uintptr_t)x % 16 != 0 || (uintptr_t)y % 16 != 0) return TCA_ERR_UNSUPPORTED;
  if (I == 1) {
#define TCA_FIBRE(a, b) \
  if (n_in == a && n_out == b) return launch_fibre<a, b>(band, x, y, O, s, sm_cap);
    TCA_FIBRE(8, 8)
    TCA_FIBRE(8, 12)
    TCA_FIBRE(12, 8)
    TCA_FIBRE(4, 4)
    TCA_FIBRE(4, 6)
    TCA_FIBRE(6, 4)
#undef TCA_FIBRE
    return TCA_ERR_UNSUPPORTED;
  }
  if (I > ((int64_t)1 << 31) || O > ((int64_t)1 << 31)) return TCA_ERR_UNSUPPORTED;
  int Ti = 0, To = 0;
  if (!row_tile_shape(O, I, band.rows32, &Ti, &To)) return TCA_ERR_UNSUPPORTED;
  EncodeFn enc = get_encode();
  if (!enc) return TCA_ERR_UNSUPPORTED;
  const int RB = band.rows32;
  CUtensorMap tmap;
  const cuuint64_t dims[3] = {(cuuint64_t)I, (cuuint64_t)n_in, (cuuint64_t)O};
  const cuuint64_t strides[2] = {(cuuint64_t)I * 4, (cuuint64_t)I * n_in * 4};
  const cuuint32_t box[3] = {(cuuint32_t)Ti, (cuuint32_t)RB, (cuuint32_t)To};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)x, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return TCA_ERR_UNSUPPORTED;
  RowGeom g;
  g.O = O;
  g.I = I;
  g.n_in = n_in;
  g.n_out = n_out;
  g.W = W;
  g.Ti = Ti;
  g.To = To;
  g.RB = RB;
  g.i_chunks = (I + Ti - 1) / Ti;
  g.j_chunks = (n_out + kJB - 1) / kJB;
  g.tiles = ((O + To - 1) / To) * g.i_chunks * g.j_chunks;
  g.stage_floats = ((Ti * RB * To + 31) / 32) * 32;
  g.unit = band.unit && W == 7;
  // Measured on GB300 (160^3 x 8 Gram and collocation sweeps): three persistent
  // CTAs per SM with a 3-deep ring beat one tile per CTA and deeper rings.
  static const int per_sm = env_int("TCA_ROWS_CTAS_PER_SM", 3);
  const size_t stage_bytes = sizeof(float) * (size_t)g.stage_floats;
  g.stages = per_sm > 0
                 ? (int)std::max<size_t>(2, std::min<size_t>(3, (200 * 1024) / (per_sm * stage_bytes)))
                 : 1;
  const int sms = sm_cap > 0 ? std::min(sm_cap, sm_count()) : sm_count();
  const int64_t grid = per_sm > 0 ? std::min<int64_t>(g.tiles, (int64_t)sms * per_sm) : g.tiles;
  if (grid > ((int64_t)1 << 31) - 1) return TCA_ERR_UNSUPPORTED;
  const size_t sm = sizeof(float) * (size_t)g.stages * g.stage_floats + 128 + 8 * g.stages;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(band_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(band_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  if (g.unit)
    band_rows_kernel<true><<<(unsigned)grid, kThreads, sm, s>>>(tmap, y, g, band.start, band.w32);
  else
    band_rows_kernel<false><<<(unsigned)grid, kThreads, sm, s>>>(tmap, y, g, band.start, band.w32);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

int rows_per_chunk(const int32_t* start_host, int64_t n_out, int W) {
  int rb = 0;
  for (int64_t j0 = 0; j0 < n_out; j0 += kJB) {
    const int64_t j1 = std::min<int64_t>(n_out, j0 + kJB) - 1;
    rb = std::max<int>(rb, (int)(start_host[j1] + W - start_host[j0]));
  }
  return rb;
}

bool encode_tmap_f32(CUtensorMap* map, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                     const uint32_t* box) {
  return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, rank, dims, strides, box);
}

bool encode_tmap(CUtensorMap* map, CUtensorMapDataType dtype, const void* base, int rank, const uint64_t* dims,
                 const uint64_t* strides, const uint32_t* box) {
  EncodeFn enc = get_encode();
  if (!enc || rank < 1 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) st[i] = strides[i];
  }
  return enc(map, dtype, (cuuint32_t)rank, const_cast<void*>(base), d, st, b, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int* wait_timeout_flag() {
  static int* addr = nullptr;
  if (!addr) {
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_wait_timeout) == cudaSuccess) addr = static_cast<int*>(a);
  }
  return addr;
}

// Give-up check of the wait machinery: one block waits on an mbarrier that
// nothing arrives at, `polls` times at most, then records the give-up like a
// real wait would.  Bounded by construction; touches no memory but its own.
__global__ void wait_selftest_kernel(long long polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool done = false;
  for (long long i = 0; i < polls && !done; ++i) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(&bar)), "r"(0u)
        : "memory");
    done = ok != 0;
  }
  if (!done && threadIdx.x == 0) atomicExch(&g_wait_timeout, 1);
}

// Pinned word the flag is read into (one per process; calls serialise on it).
static int* flag_host() {
  static int* h = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    if (cudaMallocHost((void**)&h, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      h = nullptr;
    }
  });
  return h;
}

tca_status check_wait_timeout(cudaStream_t s) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int* dflag = wait_timeout_flag();
  int* h = flag_host();
  if (!dflag || !h) return TCA_ERR_CUDA;
  TCA_CUDA_TRY(cudaMemcpyAsync(h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  if (*h == 0) return TCA_OK;
  TCA_CUDA_TRY(cudaMemsetAsync(dflag, 0, sizeof(int), s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  return TCA_ERR_TIMEOUT;
}

tca_status wait_selftest(long long polls, cudaStream_t s) {
  if (polls < 0) return TCA_ERR_INVALID_ARG;
  wait_selftest_kernel<<<1, 32, 0, s>>>(polls);
  TCA_LAUNCH_CHECK();
  return check_wait_timeout(s);
}


}  // namespace tca

extern "C" tca_status tca_check_timeout(cudaStream_t stream) { return tca::check_wait_timeout(stream); }

extern "C" tca_status tca_wait_selftest(int64_t polls, cudaStream_t stream) {
  return tca::wait_selftest((long long)polls, stream);
}
