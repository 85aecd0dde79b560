// Dense mode product on the 5th-generation tensor cores (tcgen05, TF32 operands,
// FP32 accumulation in tensor memory).
//
// y = x x_k A for a dense one-dimensional transformation A (n_out x n_in,
// Eq. separable_transf) is a GEMM over the positions of the other modes:
//   D[q][j] = sum_l X[q][l] A[j][l],   q = (o, i) flattened, l along mode k.
// A tile is 128 consecutive positions (M = 128), K = n_in (padded to 8) and
// N = n_out (padded to 16).  The factor is staged once per CTA in shared
// memory in the canonical K-major core-matrix layout (8 rows x 16 bytes).  A
// persistent CTA walks its tiles with three warp roles: twelve load warps
// (three threads per tile row) read X from HBM and write the A tile, one thread issues
// the tcgen05.mma chain into one of two TMEM accumulators and commits to
// mbarriers, and four epilogue warps read TMEM back (tcgen05.ld) and write y,
// so that loading tile t + 1, the MMAs of tile t and the epilogue of tile t - 1
// overlap.  Every mbarrier wait is bounded.
//
// split = 2 runs the 3xTF32 scheme: every operand is split into a TF32 head
// (round-to-nearest) and an FP32 tail, and D = Xh Ah + Xh At + Xt Ah, which
// recovers about FP32 accuracy; split = 1 is plain TF32 (for refinement).
#include <algorithm>
#include <cstdio>

#include "tca_internal.cuh"

namespace tca {

namespace {

constexpr int kM = 128;
constexpr int kLoadWarps = 12, kEpiWarps = 4;
constexpr int kKParts = kLoadWarps / 4;                                // load threads per tile row
constexpr int kMmaWarp = kLoadWarps;                                   // warp 12
constexpr int kTcThreads = (kLoadWarps + 1 + kEpiWarps) * 32;          // 544
constexpr long long kTcWaitLimit = 1ll << 26;
constexpr int kChunk = 32;  // K values a load thread holds per step

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = bytes between
// K-adjacent core matrices, sbo = bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ float tf32_head(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, k) in the canonical K-major no-swizzle layout.
__device__ __forceinline__ int canon(int row, int k, int sbo) {
  return (row >> 3) * sbo + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

struct TcGeom {
  int64_t O, I, P, tiles;  // P = O * I positions
  int n_in, n_out, Kp, Np, split, tmem_cols;
};

enum { BAR_AFULL = 0, BAR_AEMPTY = 1, BAR_ACCFULL = 2, BAR_ACCEMPTY = 4, NBARS = 6 };

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
// Bounded wait on an mbarrier phase; gives up (and raises the CTA's abort
// flag) after kTcWaitLimit polls, or returns early once another role aborted.
__device__ __forceinline__ bool bar_wait(uint64_t* b, int parity, volatile int* abort) {
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}

// Warp roles (one CTA per SM, persistent over tiles of 128 positions):
//   warps 0-11  load: three threads per tile row, each owning a third of the
//               row's n_in values; they read them from HBM (32 at a time, the
//               next chunk in flight while the current one is written), split
//               them into TF32 head and tail (3xTF32) and write the canonical
//               K-major A tile (many loads in flight per SM: the reads are
//               latency-bound otherwise);
//   warp 12     MMA: one thread issues the tcgen05.mma chain of a tile into
//               one of two TMEM accumulators and commits to two mbarriers (A
//               free, accumulator full);
//   warps 13-16 epilogue: TMEM -> registers (tcgen05.ld) -> y.
// Loading tile t + 1 overlaps the MMAs of tile t and the epilogue of t - 1.
__global__ void __launch_bounds__(kTcThreads, 1) dense_tc_kernel(const float* __restrict__ x, float* __restrict__ y,
                                                                 const float* __restrict__ a, TcGeom g,
                                                                 int* __restrict__ timeout_flag,
                                                                 const Scalars* __restrict__ stop) {
  // A CG preconditioner product after the iteration's stop flags are set
  // does no work (before any barrier or tensor-memory allocation).
  if (stop && cg_done(stop)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nsplit = g.split == 2 ? 2 : 1;
  const int sbo = (g.Kp / 4) * 128;  // A (kM rows) and B (Np rows) share the K extent
  const int bytesA = kM * g.Kp * 4;
  const int bytesB = g.Np * g.Kp * 4;
  unsigned char* sA[2] = {base, base + bytesA};
  unsigned char* sB[2] = {base + nsplit * bytesA, base + nsplit * bytesA + bytesB};
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + nsplit * (bytesA + bytesB));
  unsigned* tslot = reinterpret_cast<unsigned*>(bars + NBARS);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // Factor (n_out x n_in) as the K-major B operand, zero padded; head and tail.
  for (int idx = tid; idx < g.Np * g.Kp; idx += kTcThreads) {
    const int j = idx / g.Kp, l = idx % g.Kp;
    const float v = (j < g.n_out && l < g.n_in) ? __ldg(a + (int64_t)j * g.n_in + l) : 0.f;
    const int off = canon(j, l, sbo);
    const float h = nsplit == 2 ? tf32_head(v) : v;
    *reinterpret_cast<float*>(sB[0] + off) = h;
    if (nsplit == 2) *reinterpret_cast<float*>(sB[1] + off) = v - h;
  }
  if (tid == 0) {
    bar_init(&bars[BAR_AFULL], kLoadWarps * 32);
    bar_init(&bars[BAR_AEMPTY], 1);
    bar_init(&bars[BAR_ACCFULL], 1);
    bar_init(&bars[BAR_ACCFULL + 1], 1);
    bar_init(&bars[BAR_ACCEMPTY], kEpiWarps * 32);
    bar_init(&bars[BAR_ACCEMPTY + 1], kEpiWarps * 32);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(g.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B tile -> tensor-core reads
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = *tslot;

  if (warp < kLoadWarps) {
    // ---------------- load / split ----------------
    const int r = tid % kM;
    // K range of this thread: part kp of kKParts, a multiple of 4 wide.
    const int kp = tid / kM;
    const int kw = ((g.Kp / 4 + kKParts - 1) / kKParts) * 4;
    const int kb = kp * kw, ke = min(g.Kp, kb + kw);
    const bool fibre = g.I == 1 && (g.n_in % 4) == 0;
    int k = 0;
    for (int64_t t = blockIdx.x; t < g.tiles; t += gridDim.x, ++k) {
      const int64_t q = t * kM + r;
      const bool ok = q < g.P;
      const int64_t xb = ok ? (q / g.I) * (int64_t)g.n_in * g.I + q % g.I : 0;
      float cur[kChunk], nxt[kChunk];
      auto load = [&](int c0, float* dst) {
        if (fibre) {
#pragma unroll
          for (int u = 0; u < kChunk / 4; ++u) {
            const int l = c0 + 4 * u;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok && l < g.n_in) v = __ldg(reinterpret_cast<const float4*>(x + xb + l));
            dst[4 * u] = v.x; dst[4 * u + 1] = v.y; dst[4 * u + 2] = v.z; dst[4 * u + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int u = 0; u < kChunk; ++u) {
            const int l = c0 + u;
            dst[u] = (ok && l < g.n_in) ? __ldg(x + xb + (int64_t)l * g.I) : 0.f;
          }
        }
      };
      if (kb < ke) load(kb, cur);
      if (k > 0 && !bar_wait(&bars[BAR_AEMPTY], (k - 1) & 1, abort)) break;  // MMAs of tile k-1 read A
      for (int c0 = kb; c0 < ke; c0 += kChunk) {
        if (c0 + kChunk < ke) load(c0 + kChunk, nxt);
#pragma unroll
        for (int u = 0; u < kChunk / 4; ++u) {
          const int l = c0 + 4 * u;
          if (l >= ke) break;
          const int off = (r >> 3) * sbo + (l >> 2) * 128 + (r & 7) * 16;
          float4 h = make_float4(cur[4 * u], cur[4 * u + 1], cur[4 * u + 2], cur[4 * u + 3]);
          if (nsplit == 2) {
            const float4 v = h;
            h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
            *reinterpret_cast<float4*>(sA[1] + off) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
          }
          *reinterpret_cast<float4*>(sA[0] + off) = h;
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) cur[u] = nxt[u];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
      bar_arrive(&bars[BAR_AFULL]);
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      const unsigned idesc =
          (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(g.Np >> 3) << 17) | ((unsigned)(kM >> 4) << 24);
      int k = 0;
      for (int64_t t = blockIdx.x; t < g.tiles; t += gridDim.x, ++k) {
        const int slot = k & 1;
        if (k >= 2 && !bar_wait(&bars[BAR_ACCEMPTY + slot], ((k - 2) >> 1) & 1, abort)) break;
        if (!bar_wait(&bars[BAR_AFULL], k & 1, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const unsigned dtm = tmem + (unsigned)(slot * g.Np);
        int first = 1;
        for (int ks = 0; ks < g.Kp / 8; ++ks) {
          for (int term = 0; term < (nsplit == 2 ? 3 : 1); ++term) {
            const int ia = term == 2 ? 1 : 0, ib = term == 1 ? 1 : 0;
            const uint64_t ad = smem_desc(su32(sA[ia]) + ks * 256, 128, sbo);
            const uint64_t bd = smem_desc(su32(sB[ib]) + ks * 256, 128, sbo);
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
                "l"(ad), "l"(bd), "r"(idesc), "r"(first ? 0u : 1u));
            first = 0;
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&bars[BAR_AEMPTY])));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&bars[BAR_ACCFULL + slot])));
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int lq = warp & 3;  // TMEM lane quarter this warp may access
    const int row = 32 * lq + lane;
    int k = 0;
    for (int64_t t = blockIdx.x; t < g.tiles; t += gridDim.x, ++k) {
      const int slot = k & 1;
      const bool okw = __all_sync(0xffffffffu, bar_wait(&bars[BAR_ACCFULL + slot], (k >> 1) & 1, abort));
      if (!okw) {
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t q = t * kM + row;
      const bool ov = q < g.P;
      const int64_t oo = ov ? q / g.I : 0, io = ov ? q % g.I : 0;
      float* yr = y + oo * (int64_t)g.n_out * g.I + io;
      for (int c0 = 0; c0 < g.Np; c0 += 16) {
        unsigned v[16];
        const unsigned taddr = tmem + ((unsigned)(32 * lq) << 16) + (unsigned)(slot * g.Np + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (ov) {
          if (g.I == 1 && (g.n_out % 4) == 0 && c0 + 16 <= g.n_out) {
#pragma unroll
            for (int qq = 0; qq < 16; qq += 4)
              *reinterpret_cast<float4*>(yr + c0 + qq) = make_float4(__uint_as_float(v[qq]), __uint_as_float(v[qq + 1]),
                                                                     __uint_as_float(v[qq + 2]), __uint_as_float(v[qq + 3]));
          } else {
#pragma unroll
            for (int qq = 0; qq < 16; ++qq)
              if (c0 + qq < g.n_out) yr[(int64_t)(c0 + qq) * g.I] = __uint_as_float(v[qq]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      bar_arrive(&bars[BAR_ACCEMPTY + slot]);
    }
  }
  __syncthreads();
  if (*abort && tid == 0 && timeout_flag) atomicExch(timeout_flag, 1);
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols));
  }
}

int tc_sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

static size_t dense_tc_smem_bytes(int64_t n_in, int64_t n_out, int split) {
  const int64_t Kp = (n_in + 7) / 8 * 8, Np = (n_out + 15) / 16 * 16;
  const int nsplit = split == 2 ? 2 : 1;
  return (size_t)nsplit * ((size_t)kM * Kp * 4 + (size_t)Np * Kp * 4) + NBARS * 8 + 16 + 1024;
}

int dense_tc_max_split(int64_t n_in, int64_t n_out) {
  if (n_in <= 0 || n_out <= 0 || (n_out + 15) / 16 * 16 > 256) return 0;
  if (dense_tc_smem_bytes(n_in, n_out, 2) <= 220 * 1024) return 2;
  if (dense_tc_smem_bytes(n_in, n_out, 1) <= 220 * 1024) return 1;
  return 0;
}

tca_status launch_dense_tc(const Dense& d, const float* x, float* y, int64_t O, int64_t I, int split,
                           cudaStream_t s, int sm_cap, const Scalars* stop) {
  const int n_in = (int)d.n_in, n_out = (int)d.n_out;
  if (!d.a32 || n_in <= 0 || n_out <= 0) return TCA_ERR_UNSUPPORTED;
  if ((uintptr_t)x % 16 != 0) return TCA_ERR_UNSUPPORTED;
  TcGeom g;
  g.O = O;
  g.I = I;
  g.P = O * I;
  g.n_in = n_in;
  g.n_out = n_out;
  g.Kp = (n_in + 7) / 8 * 8;
  g.Np = (n_out + 15) / 16 * 16;
  g.split = split;
  if (g.Np > 256) return TCA_ERR_UNSUPPORTED;  // two accumulators of Np columns in 512
  int cols = 32;
  while (cols < 2 * g.Np) cols *= 2;  // two accumulators
  g.tmem_cols = cols;
  g.tiles = (g.P + kM - 1) / kM;
  const size_t bytes = dense_tc_smem_bytes(n_in, n_out, split);
  if (bytes > 220 * 1024) return TCA_ERR_UNSUPPORTED;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  // Persistent: at most one CTA per SM.  When the tile's shared memory leaves
  // room for a second CTA, both TMEM allocations fit (2 x 2 Np <= 512 columns
  // for Np <= 128) or the second waits for the first to free its columns.
  const int64_t grid = std::min<int64_t>(g.tiles, (int64_t)(sm_cap > 0 ? std::min(sm_cap, tc_sm_count()) : tc_sm_count()));
  dense_tc_kernel<<<(unsigned)std::max<int64_t>(grid, 1), kTcThreads, bytes, s>>>(x, y, d.a32, g,
                                                                                  wait_timeout_flag(), stop);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace tca
