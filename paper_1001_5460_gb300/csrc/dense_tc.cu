// Dense mode product on the 5th-generation tensor cores (tcgen05, TF32 operands,
// FP32 accumulation in tensor memory).
//
// y = x x_k A for a dense one-dimensional transformation A (n_out x n_in,
// Eq. separable_transf) is a GEMM over the positions of the other modes:
//   D[q][j] = sum_l X[q][l] A[j][l],   q = (o, i) flattened, l along mode k.
// A CTA owns 128 consecutive positions per tile (M = 128), K = n_in (padded
// to 8) and N = n_out (padded to 16).  The factor is staged once per CTA in
// shared memory, each X tile is gathered from HBM into the canonical K-major
// core-matrix layout (8 rows x 16 bytes), one elected thread issues the
// tcgen05.mma chain with the accumulator in tensor memory, tcgen05.commit
// arrives on an mbarrier, and the four warps read their 32 TMEM lanes back
// (tcgen05.ld) and write y.  Persistent: the grid is a multiple of the SM
// count and CTAs walk their tiles.
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
constexpr int kTcThreads = 256;
constexpr long long kTcWaitLimit = 1ll << 26;

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

__global__ void __launch_bounds__(kTcThreads, 1) dense_tc_kernel(const float* __restrict__ x, float* __restrict__ y,
                                                                 const float* __restrict__ a, TcGeom g,
                                                                 int* __restrict__ timeout_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nsplit = g.split == 2 ? 2 : 1;
  const int sboA = (g.Kp / 4) * 128;           // A (X tile): kM rows
  const int sboB = sboA;                       // B (factor): Np rows, same K extent
  const int bytesA = kM * g.Kp * 4;
  const int bytesB = g.Np * g.Kp * 4;
  unsigned char* sA[2] = {base, base + bytesA};
  unsigned char* sB[2] = {base + nsplit * bytesA, base + nsplit * bytesA + bytesB};
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + nsplit * (bytesA + bytesB));
  unsigned* tslot = reinterpret_cast<unsigned*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // Factor A (n_out x n_in) as the K-major B operand, zero padded; split into head and tail.
  for (int idx = tid; idx < g.Np * g.Kp; idx += kTcThreads) {
    const int j = idx / g.Kp, l = idx % g.Kp;
    const float v = (j < g.n_out && l < g.n_in) ? __ldg(a + (int64_t)j * g.n_in + l) : 0.f;
    const int off = canon(j, l, sboB);
    const float h = nsplit == 2 ? tf32_head(v) : v;
    *reinterpret_cast<float*>(sB[0] + off) = h;
    if (nsplit == 2) *reinterpret_cast<float*>(sB[1] + off) = v - h;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(g.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = *tslot;
  const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(g.Np >> 3) << 17) | ((unsigned)(kM >> 4) << 24);
  bool timed_out = false;
  int phase = 0;

  auto put = [&](int row, int l, float v) {
    const int off = canon(row, l, sboA);
    const float h = nsplit == 2 ? tf32_head(v) : v;
    *reinterpret_cast<float*>(sA[0] + off) = h;
    if (nsplit == 2) *reinterpret_cast<float*>(sA[1] + off) = v - h;
  };
  // Tile gather paths: rows along a contiguous inner index (I a multiple of
  // 128, one outer slab per tile), rows = whole fibres (I = 1), or generic.
  const bool rows_inner = (g.I % kM) == 0;
  const bool rows_fibre = g.I == 1 && (g.n_in % 4) == 0;
  for (int64_t t = blockIdx.x; t < g.tiles; t += gridDim.x) {
    const int64_t q0 = t * kM;
    if (rows_inner) {
      // 32 float4 per K row; 8 loads in flight per thread before any store.
      const int64_t o = q0 / g.I, i0 = q0 % g.I;
      const float* xo = x + o * (int64_t)g.n_in * g.I + i0;
      const int nv = g.Kp * (kM / 4);
      for (int base_idx = tid; base_idx < nv; base_idx += 8 * kTcThreads) {
        float4 buf[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base_idx + u * kTcThreads;
          const int l = idx >> 5, qd = idx & 31;
          buf[u] = (idx < nv && l < g.n_in) ? __ldg(reinterpret_cast<const float4*>(xo + (int64_t)l * g.I) + qd)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base_idx + u * kTcThreads;
          if (idx >= nv) break;
          const int l = idx >> 5, r = (idx & 31) * 4;
          put(r, l, buf[u].x);
          put(r + 1, l, buf[u].y);
          put(r + 2, l, buf[u].z);
          put(r + 3, l, buf[u].w);
        }
      }
    } else if (rows_fibre) {
      // Row r is fibre q0 + r: n_in contiguous floats, read as float4.
      const int kq = g.Kp / 4;
      for (int idx = tid; idx < kM * kq; idx += kTcThreads) {
        const int r = idx / kq, l = (idx % kq) * 4;
        const int64_t q = q0 + r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < g.P && l < g.n_in) v = __ldg(reinterpret_cast<const float4*>(x + q * g.n_in + l));
        put(r, l, v.x);
        put(r, l + 1, v.y);
        put(r, l + 2, v.z);
        put(r, l + 3, v.w);
      }
    } else {
      for (int idx = tid; idx < kM * g.Kp; idx += kTcThreads) {
        const int r = idx % kM, l = idx / kM;
        const int64_t q = q0 + r;
        float v = 0.f;
        if (q < g.P && l < g.n_in) v = __ldg(x + (q / g.I) * (int64_t)g.n_in * g.I + (int64_t)l * g.I + q % g.I);
        put(r, l, v);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      int first = 1;
      for (int ks = 0; ks < g.Kp / 8; ++ks) {
        for (int term = 0; term < (nsplit == 2 ? 3 : 1); ++term) {
          const int ia = term == 2 ? 1 : 0, ib = term == 1 ? 1 : 0;
          const uint64_t ad = smem_desc(su32(sA[ia]) + ks * 256, 128, sboA);
          const uint64_t bd = smem_desc(su32(sB[ib]) + ks * 256, 128, sboB);
          const unsigned acc = first ? 0u : 1u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          first = 0;
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)));
    }
    bool done = false;
    for (long long it = 0; it < kTcWaitLimit && !done; ++it) {
      unsigned ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(su32(bar)), "r"(phase)
          : "memory");
      done = ok;
    }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (done) {
      // Warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of the tile); warps
      // 0-3 take the first half of the columns, warps 4-7 the second.
      const int wl = warp & 3;
      const int row = 32 * wl + lane;
      const int64_t qo = t * kM + row;
      const bool ov = qo < g.P;
      const int64_t oo = ov ? qo / g.I : 0, io = ov ? qo % g.I : 0;
      float* yr = y + oo * (int64_t)g.n_out * g.I + io;
      const int half = g.Np / 2;  // a multiple of 8
      const int cb = (warp >> 2) * half;
      for (int c0 = cb; c0 < cb + half; c0 += 8) {
        unsigned v[8];
        const unsigned taddr = tmem + ((unsigned)(32 * wl) << 16) + (unsigned)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (ov) {
#pragma unroll
          for (int qq = 0; qq < 8; ++qq)
            if (c0 + qq < g.n_out) yr[(int64_t)(c0 + qq) * g.I] = __uint_as_float(v[qq]);
        }
      }
    } else {
      timed_out = true;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    if (__syncthreads_or(timed_out)) break;
  }
  if (timed_out && tid == 0 && timeout_flag) atomicExch(timeout_flag, 1);
  __syncthreads();
  if (warp == 0) {
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

tca_status launch_dense_tc(const Dense& d, const float* x, float* y, int64_t O, int64_t I, int split,
                           cudaStream_t s) {
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
  if (g.Np > 256) return TCA_ERR_UNSUPPORTED;
  int cols = 32;
  while (cols < g.Np) cols *= 2;
  g.tmem_cols = cols;
  g.tiles = (g.P + kM - 1) / kM;
  const int nsplit = split == 2 ? 2 : 1;
  const size_t bytes = (size_t)nsplit * ((size_t)kM * g.Kp * 4 + (size_t)g.Np * g.Kp * 4) + 16 + 1024;
  if (bytes > 220 * 1024) return TCA_ERR_UNSUPPORTED;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  // One CTA per SM: its shared memory and TMEM columns leave room for nothing else of this kernel.
  const int64_t grid = std::min<int64_t>(g.tiles, (int64_t)tc_sm_count());
  dense_tc_kernel<<<(unsigned)std::max<int64_t>(grid, 1), kTcThreads, bytes, s>>>(x, y, d.a32, g,
                                                                                  wait_timeout_flag());
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace tca
