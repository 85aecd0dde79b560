// Normal-operator sweep in bfloat16 on the tensor cores (the mixed-precision
// form's inner operator):
//   q = (G_1 kron G_2 kron G_3 kron G_4) p + lambda sum_k L_k p
// for banded factors, with p and q stored as bfloat16 and every sum in FP32.
//
// It is the "iterative application of the tensor multiplication" of each CG
// step (Sec. 4.1, Fig. 2, Q = A.P) with the separable structure of
// Eq. separable_transf, split by where each product runs best:
//   - modes 3 and 4, merged into one inner axis c = (i3, i4) of length n3 n4,
//     are one dense contraction per (plane, row): S = W p with
//     W = G_3 kron G_4 restricted to a tile of 128 outputs c' and the 128 + 2H
//     inputs c that reach them (H = 3 n4 rounded up to 8).  It runs on tcgen05
//     (kind::f16, BF16 operands, FP32 accumulators in tensor memory), as does
//     the regulariser of those modes, R = lambda (L_3 kron I + I kron L_4);
//   - mode 2 (G_2, lambda L_2) and mode 1 (G_1, lambda L_1, a 7-slot register
//     ring marching along mode 1) are short stencils applied in registers by
//     the threads that read the accumulators back, one thread per output c'.
//
// Tile: 16 rows of mode 2 x 128 values of the inner axis, marching along
// mode 1 over a chunk of planes.  Per plane j (22 halo rows x (128 + 2H)):
//   producer warp  TMA of the halo tiles of r and p_old (bfloat16, box
//                  {8 KC, 22, 1} of the view {n_c, n2, n1}: one request per
//                  halo row), 3-stage mbarrier ring; cp.async pieces when a
//                  box would be larger than the tensor;
//   worker warps   p = r + beta p_old (FP32 math, rounded to bfloat16) into the
//                  MMA operand buffer in the canonical no-swizzle K-major
//                  layout [chunk of 8 c][row][16 B] (rows 22..31 stay zero),
//                  p_new to HBM;
//   MMA warp       chain 1: D1[c'][row] = sum_c W[c'][c] P[row][c], N = 32 rows;
//                  chain 2: D2[c'][core row] = sum_c R[c'][c] P[3 + row][c],
//                  N = 16 (the operand shifted by three rows: a start address);
//                  one tcgen05.commit per plane, accumulators double-buffered;
//   worker warps   tcgen05.ld of D1 and D2, G_2 / lambda L_2 down the rows,
//                  the mode-1 ring, q of plane j - 3 (bfloat16) and <p, q>.
// Every mbarrier wait is bounded; a CTA that gives up sets the library's
// timeout flag, skips its stores and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "tca_internal.cuh"

namespace tca {

namespace {

namespace tb {

constexpr int kRows = 16;             // output rows of mode 2 per tile
constexpr int kHalo = kRows + 6;      // rows loaded per plane (G_2 reaches +-3)
constexpr int kOpRows = 32;           // operand rows of chain 1 (N = 32; rows 22..31 zero)
constexpr int kTileC = 128;           // outputs of the inner axis per tile (MMA M)
constexpr int kStages = 3;
constexpr int kMaxPlanes = 256;       // planes a CTA may visit (chunk + 6): size of the G_1 / L_1 table
constexpr int kPChunk = 33 * 16;      // operand chunk stride (33 rows: conflict-free column reads)
constexpr int kTmemCols = 128;        // two accumulator sets of 64 columns (D1: 32, D2: 16)
constexpr long long kWaitPolls = 1ll << 24;

struct Args {
  const __nv_bfloat16* r;     // CG: residual
  const __nv_bfloat16* pold;  // CG: previous direction; plain: the input
  __nv_bfloat16* pnew;        // CG: new direction
  __nv_bfloat16* q;
  const uint4* wt;            // per inner tile: W then R, each KC x 128 x 16 bytes
  const float* g1;            // G_1 band (n1 x 7), lambda L_1 band (n1 x 5)
  const float* l1;
  const float* g2;            // G_2 band (n2 x 7), lambda L_2 band (n2 x 5)
  const float* l2;
  int n1, n2, nc, H, KC;
  int ctiles, nchunks, chunk;
  Scalars* scal;
  Reduce red;
  int* timeout_flag;
  int tma;
  CUtensorMap tm_r, tm_p;
};

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// Bounded parity wait; gives up (returns false, marks the CTA) after kWaitPolls
// polls or as soon as another role of the CTA has given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort) {
  for (long long it = 0; it < kWaitPolls; ++it) {
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
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(su32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major: lbo = byte distance of
// K-adjacent core matrices, sbo = byte distance of the next 8 rows.
__device__ __forceinline__ uint64_t sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
__device__ __forceinline__ void mma_bf16(unsigned dtm, uint64_t ad, uint64_t bd, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

__device__ __forceinline__ float bf_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ unsigned pack_bf2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);  // a -> low half
  return *reinterpret_cast<const unsigned*>(&v);
}
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// Shared-memory carve-up (bytes) for KC chunks of the inner window.
struct Smem {
  int w, r, stg, stg_bytes, p, p_bytes, coef, g1l1, bar, misc, total;
  __host__ __device__ Smem(int KC, int nin, int nwarps) {
    stg_bytes = ((KC * kHalo * 16) + 127) / 128 * 128;
    p_bytes = ((KC * kPChunk) + 127) / 128 * 128;
    w = 0;
    r = w + KC * kTileC * 16;
    stg = r + KC * kTileC * 16;
    p = stg + kStages * nin * stg_bytes;
    coef = p + 2 * p_bytes;
    g1l1 = coef + 12 * kRows * 4;  // g2[7][16], l2[5][16] floats, then 16 floats per plane
    bar = g1l1 + kMaxPlanes * 16 * 4;
    misc = bar + (2 * kStages + 7) * 8;
    total = misc + 16 + 8 * nwarps + 128;  // flags, reduction scratch, alignment slack
  }
};
// barrier indices
enum { B_SFULL = 0, B_SEMPTY = kStages, B_PFULL = 2 * kStages, B_AFULL = 2 * kStages + 2,
       B_AEMPTY = 2 * kStages + 4, B_W = 2 * kStages + 6, NBARS = 2 * kStages + 7 };

// Bounded wait with a short sleep between polls, for the single-lane roles
// (producer, MMA issue), which would otherwise take issue slots from the workers.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* b, unsigned parity, volatile int* abort) {
  for (long long it = 0; it < kWaitPolls; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63 && *abort) return false;
    __nanosleep(32);
  }
  *abort = 1;
  return false;
}

template <int N>
__device__ __forceinline__ void tmem_ld(unsigned taddr, unsigned* v);
template <>
__device__ __forceinline__ void tmem_ld<2>(unsigned taddr, unsigned* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld<4>(unsigned taddr, unsigned* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld<8>(unsigned taddr, unsigned* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

// RPT core rows per worker thread: 16 / RPT groups of four warps (each warp
// reads its own TMEM lane quarter), one output c' per thread.
template <bool CG, int RPT>
__global__ void __launch_bounds__(64 + 128 * (kRows / RPT), 1) bf16_sweep_kernel(const __grid_constant__ Args a) {
  constexpr int NIN = CG ? 2 : 1;
  constexpr int kGroups = kRows / RPT;
  constexpr int kWorkers = 128 * kGroups;
  constexpr int kThreads = 64 + kWorkers;
  static_assert(RPT == 4 || RPT == 8, "rows per worker thread");
  if constexpr (CG) {
    if (cg_done(a.scal)) return;
  }
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int KC = a.KC, H = a.H;
  const Smem L(KC, NIN, kThreads / 32);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bar);
  unsigned* tslot = reinterpret_cast<unsigned*>(sm + L.misc);
  volatile int* abort = reinterpret_cast<volatile int*>(sm + L.misc + 4);
  volatile int* s_last = reinterpret_cast<volatile int*>(sm + L.misc + 8);
  double* s_red = reinterpret_cast<double*>(sm + L.misc + 16);
  float* g2s = reinterpret_cast<float*>(sm + L.coef);  // [7][16]
  float* l2s = g2s + 7 * kRows;                        // [5][16]
  float* g1l1 = reinterpret_cast<float*>(sm + L.g1l1);  // [plane][16]: G_1 taps 0..6, lambda L_1 taps 0..4

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float beta = CG ? (float)a.scal->beta : 0.f;
  const int n1 = a.n1, n2 = a.n2, nc = a.nc;
  const int bid = blockIdx.x;
  const int chunk_id = bid % a.nchunks;
  const int tile = bid / a.nchunks;
  const int ct = tile % a.ctiles, rt = tile / a.ctiles;
  const int i2_0 = rt * kRows, cc0 = ct * kTileC;
  const int c0 = chunk_id * a.chunk;
  const int c1 = min(n1, c0 + a.chunk);
  const int jb = max(0, c0 - kGramHalf);
  const int je = min(n1, c1 + kGramHalf);
  const int nplanes = je - jb;
  const int64_t plane = (int64_t)n2 * nc;

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&bars[B_SFULL + i], a.tma ? 1u : 32u);
      mbar_init(&bars[B_SEMPTY + i], kWorkers / 32);  // one arrival per worker warp
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars[B_PFULL + i], kWorkers / 32);
      mbar_init(&bars[B_AFULL + i], 1);
      mbar_init(&bars[B_AEMPTY + i], kWorkers / 32);
    }
    mbar_init(&bars[B_W], 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  // Coefficient tables (zero outside the domain): mode 2 of the tile's rows,
  // mode 1 of every plane the CTA visits; the zero rows 22..31 of both
  // operand buffers.
  for (int t = tid; t < 12 * kRows; t += kThreads) {
    const int e = t / kRows, rr = t % kRows, i2 = i2_0 + rr;
    float v = 0.f;
    if (i2 < n2) v = e < 7 ? a.g2[(int64_t)i2 * 7 + e] : a.l2[(int64_t)i2 * 5 + (e - 7)];
    g2s[t] = v;
  }
  for (int t = tid; t < nplanes * 16; t += kThreads) {
    const int pl = t >> 4, e = t & 15, jj = jb + pl;
    g1l1[t] = e < 7 ? a.g1[(int64_t)jj * 7 + e] : (e < 12 ? a.l1[(int64_t)jj * 5 + (e - 7)] : 0.f);
  }
  for (int t = tid; t < 2 * KC * (kOpRows - kHalo); t += kThreads) {
    const int b = t / (KC * (kOpRows - kHalo)), rem = t % (KC * (kOpRows - kHalo));
    const int kc = rem / (kOpRows - kHalo), row = kHalo + rem % (kOpRows - kHalo);
    *reinterpret_cast<uint4*>(sm + L.p + b * L.p_bytes + kc * kPChunk + row * 16) = make_uint4(0, 0, 0, 0);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // zero rows -> tensor-core reads
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = *tslot;

  float dotf = 0.f;
  if (warp == 0) {
    // ======================= producer =======================
    const unsigned stg_tx = (unsigned)(KC * kHalo * 16);
    if (a.tma) {
      if (lane == 0) {
        int issued = 0;
        mbar_expect_tx(&bars[B_W], (unsigned)(2 * KC * kTileC * 16));
        bulk_load(sm + L.w, a.wt + (size_t)ct * 2 * KC * kTileC, (unsigned)(KC * kTileC * 16), &bars[B_W]);
        bulk_load(sm + L.r, a.wt + ((size_t)ct * 2 + 1) * KC * kTileC, (unsigned)(KC * kTileC * 16), &bars[B_W]);
        for (int it = 0; it < nplanes && !*abort; ++it) {
          const int s = it % kStages;
          if (it >= kStages && !mbar_wait_sleep(&bars[B_SEMPTY + s], (unsigned)(((it / kStages) - 1) & 1), abort))
            break;
          mbar_expect_tx(&bars[B_SFULL + s], NIN * stg_tx);
          unsigned char* dst = sm + L.stg + s * NIN * L.stg_bytes;
          if (CG) tma_load_3d(dst, &a.tm_r, cc0 - H, i2_0 - 3, jb + it, &bars[B_SFULL + s]);
          tma_load_3d(dst + (NIN - 1) * L.stg_bytes, &a.tm_p, cc0 - H, i2_0 - 3, jb + it, &bars[B_SFULL + s]);
          issued = it + 1;
        }
        // No copy may outlive the CTA: after a give-up, wait (bounded) for the
        // stages still in flight and for the operand tiles.
        if (*abort) {
          for (int k = max(0, issued - kStages); k < issued; ++k)
            (void)mbar_wait_sleep(&bars[B_SFULL + k % kStages], (unsigned)((k / kStages) & 1), abort);
          for (long long it = 0; it < kWaitPolls; ++it) {
            unsigned ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, "
                "p;\n\t}"
                : "=r"(ok)
                : "r"(su32(&bars[B_W])), "r"(0u)
                : "memory");
            if (ok) break;
          }
        }
      }
      __syncwarp();
    } else {
      // cp.async pieces: the whole warp copies; W and R with plain loads.
      for (int k = lane; k < 2 * KC * kTileC; k += 32)
        reinterpret_cast<uint4*>(sm + L.w)[k] = a.wt[(size_t)ct * 2 * KC * kTileC + k];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[B_W]);
      const int units = KC * kHalo;
      for (int it = 0; it < nplanes; ++it) {
        const int s = it % kStages;
        if (it >= kStages && !mbar_wait_sleep(&bars[B_SEMPTY + s], (unsigned)(((it / kStages) - 1) & 1), abort))
          break;
        if (__any_sync(0xffffffffu, *abort)) break;
        const int j = jb + it;
        const unsigned dst = su32(sm + L.stg + s * NIN * L.stg_bytes);
        for (int src_i = 0; src_i < NIN; ++src_i) {
          const __nv_bfloat16* g = (CG && src_i == 0) ? a.r : a.pold;
          for (int u = lane; u < units; u += 32) {
            const int kc = u / kHalo, row = u % kHalo;
            const int i2 = i2_0 - 3 + row, c = cc0 - H + kc * 8;
            const bool ok = i2 >= 0 && i2 < n2 && c >= 0 && c < nc;
            const __nv_bfloat16* src = ok ? g + (int64_t)j * plane + (int64_t)i2 * nc + c : g;
            cp_async16(dst + (unsigned)(src_i * L.stg_bytes + row * KC * 16 + kc * 16), src, ok);
          }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(&bars[B_SFULL + s]))
                     : "memory");
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
  } else if (warp == 1) {
    // ======================= MMA (one lane) =======================
    // kind::f16, D = F32, A = B = BF16, both K-major; M = 128, N = 32 / 16.
    if (lane == 0) {
      const unsigned idesc1 = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kOpRows >> 3) << 17) |
                              ((unsigned)(kTileC >> 4) << 24);
      const unsigned idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kRows >> 3) << 17) |
                              ((unsigned)(kTileC >> 4) << 24);
      const uint64_t wdesc = sdesc(su32(sm + L.w), kTileC * 16, 128);
      const uint64_t rdesc = sdesc(su32(sm + L.r), kTileC * 16, 128);
      bool ok = mbar_wait_sleep(&bars[B_W], 0, abort);
      int issued = 0;
      for (int it = 0; it < nplanes && ok; ++it) {
        const int b = it & 1;
        ok = mbar_wait_sleep(&bars[B_PFULL + b], (unsigned)((it >> 1) & 1), abort);
        if (ok && it >= 2) ok = mbar_wait_sleep(&bars[B_AEMPTY + b], (unsigned)(((it - 2) >> 1) & 1), abort);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint64_t pdesc = sdesc(su32(sm + L.p + b * L.p_bytes), kPChunk, 128);
        const unsigned d1 = tmem + (unsigned)(b * 64), d2 = d1 + 32u;
        // One MMA takes K = 16 (two chunks of 8); the two chains alternate so
        // that consecutive instructions write different accumulators.
        for (int s = 0; s < KC / 2; ++s) {
          mma_bf16(d1, wdesc + (uint64_t)(s * 2 * kTileC), pdesc + (uint64_t)(s * 2 * kPChunk / 16), idesc1,
                   s > 0 ? 1u : 0u);
          mma_bf16(d2, rdesc + (uint64_t)(s * 2 * kTileC), pdesc + (uint64_t)(s * 2 * kPChunk / 16 + 3), idesc2,
                   s > 0 ? 1u : 0u);
        }
        mma_commit(&bars[B_AFULL + b]);
        issued = it + 1;
      }
      // The last commit must land before the accumulators are freed.
      if (issued > 0)
        (void)mbar_wait_sleep(&bars[B_AFULL + ((issued - 1) & 1)], (unsigned)(((issued - 1) >> 1) & 1), abort);
    }
    __syncwarp();
  } else {
    // ======================= workers =======================
    const int wt = tid - 64;                   // 0 .. kWorkers - 1
    const int grp = (warp - 2) >> 2;           // row group
    const int quarter = warp & 3;              // TMEM lane quarter this warp may read
    const int cl = 32 * quarter + lane;        // this thread's output c' in the tile
    const int r0 = RPT * grp;                  // first core row
    const int cg_ = cc0 + cl;                  // global inner index
    const bool c_ok = cg_ < nc;
    const int pcol_off = ((cl + H) >> 3) * kPChunk + ((cl + H) & 7) * 2;  // column cl + H in the operand
    const int64_t out_base = (int64_t)(i2_0 + r0) * nc + cg_;
    unsigned row_ok = 0;
#pragma unroll
    for (int k = 0; k < RPT; ++k) row_ok |= (c_ok && (i2_0 + r0 + k) < n2) ? (1u << k) : 0u;

    constexpr int NP = RPT / 2;  // row pairs
    float2 acc[NP][7];
    unsigned pring[NP][7];  // p of the plane in each ring slot (bfloat16 pairs)
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < 7; ++e) {
        acc[k][e] = make_float2(0.f, 0.f);
        pring[k][e] = 0u;
      }
    float2 w2[NP], lin2[NP], pc2[NP];

    // p pass of plane it: operand buffer it & 1, p_new of owned planes.
    auto ppass = [&](int it) -> bool {
      const int s = it % kStages, b = it & 1, j = jb + it;
      bool ok = mbar_wait(&bars[B_SFULL + s], (unsigned)((it / kStages) & 1), abort);
      const unsigned char* st = sm + L.stg + s * NIN * L.stg_bytes;
      unsigned char* pb = sm + L.p + b * L.p_bytes;
      const bool own = j >= c0 && j < c1;
      const int units = KC * kHalo;
      if (ok) {
        for (int u = wt; u < units; u += kWorkers) {
          const int row = u / KC, kc = u % KC;  // consecutive threads: consecutive chunks of one row
          const int so = row * KC * 16 + kc * 16;  // stage rows: [row][KC chunks of 16 bytes]
          uint4 pv;
          if constexpr (CG) {
            const uint4 rv = *reinterpret_cast<const uint4*>(st + so);
            const uint4 ov = *reinterpret_cast<const uint4*>(st + L.stg_bytes + so);
            pv.x = pack_bf2(fmaf(beta, bf_lo(ov.x), bf_lo(rv.x)), fmaf(beta, bf_hi(ov.x), bf_hi(rv.x)));
            pv.y = pack_bf2(fmaf(beta, bf_lo(ov.y), bf_lo(rv.y)), fmaf(beta, bf_hi(ov.y), bf_hi(rv.y)));
            pv.z = pack_bf2(fmaf(beta, bf_lo(ov.z), bf_lo(rv.z)), fmaf(beta, bf_hi(ov.z), bf_hi(rv.z)));
            pv.w = pack_bf2(fmaf(beta, bf_lo(ov.w), bf_lo(rv.w)), fmaf(beta, bf_hi(ov.w), bf_hi(rv.w)));
          } else {
            pv = *reinterpret_cast<const uint4*>(st + so);
          }
          *reinterpret_cast<uint4*>(pb + kc * kPChunk + row * 16) = pv;
          if constexpr (CG) {
            const int i2 = i2_0 - 3 + row, c = cc0 - H + kc * 8;
            if (own && row >= 3 && row < 3 + kRows && i2 < n2 && c >= cc0 && c < cc0 + kTileC && c < nc)
              *reinterpret_cast<uint4*>(a.pnew + (int64_t)j * plane + (int64_t)i2 * nc + c) = pv;
          }
        }
      }
      // The warp's reads of the stage and writes of the operand are done (and
      // the writes made visible to the tensor cores) before one lane arrives.
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars[B_SEMPTY + s]);
        mbar_arrive(&bars[B_PFULL + b]);
      }
      return ok;
    };

    bool ok = nplanes > 0 ? ppass(0) : true;
#pragma unroll 1
    for (int j = jb; j < c1 + kGramHalf; ++j) {
      const int it = j - jb;
      const bool have = j < je;
      float g1r[7], l1r[5];
      if (have) {
        if (it + 1 < nplanes) ok = ppass(it + 1) && ok;
        const int b = it & 1;
        // Accumulators of plane j.
        const bool got = mbar_wait(&bars[B_AFULL + b], (unsigned)((it >> 1) & 1), abort);
        ok = got && ok;
        asm volatile("tcgen05.fence::after_thread_sync;");
        unsigned s1u[RPT + 8], d2u[RPT];  // D1 columns r0 .. r0 + RPT + 5 (+ unused), D2 columns r0 .. r0 + RPT - 1
        const unsigned taddr = tmem + ((unsigned)(32 * quarter) << 16) + (unsigned)(b * 64) + (unsigned)r0;
        tmem_ld<8>(taddr, s1u);
        if constexpr (RPT == 8) tmem_ld<8>(taddr + 8u, s1u + 8);
        else tmem_ld<2>(taddr + 8u, s1u + 8);
        tmem_ld<RPT>(taddr + 32u, d2u);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[B_AEMPTY + b]);
        // Centre column of p, halo rows r0 + 1 .. r0 + RPT + 4 (core rows r0 - 2 .. r0 + RPT + 1).
        const unsigned char* pb = sm + L.p + b * L.p_bytes + pcol_off;
        float pc[RPT + 4];
#pragma unroll
        for (int t = 0; t < RPT + 4; ++t)
          pc[t] = __uint_as_float((unsigned)*reinterpret_cast<const unsigned short*>(pb + (r0 + 1 + t) * 16) << 16);
        {
          const float4* cr = reinterpret_cast<const float4*>(g1l1 + it * 16);
          const float4 c0v = cr[0], c1v = cr[1], c2v = cr[2];
          g1r[0] = c0v.x; g1r[1] = c0v.y; g1r[2] = c0v.z; g1r[3] = c0v.w;
          g1r[4] = c1v.x; g1r[5] = c1v.y; g1r[6] = c1v.z;
          l1r[0] = c1v.w; l1r[1] = c2v.x; l1r[2] = c2v.y; l1r[3] = c2v.z; l1r[4] = c2v.w;
        }
#pragma unroll
        for (int h = 0; h < RPT / 4; ++h) {
          // Coefficients of rows r0 + 4h .. r0 + 4h + 3, one 128-bit load per tap.
          float4 g2f[7], l2f[5];
#pragma unroll
          for (int e = 0; e < 7; ++e) g2f[e] = *reinterpret_cast<const float4*>(g2s + e * kRows + r0 + 4 * h);
#pragma unroll
          for (int e = 0; e < 5; ++e) l2f[e] = *reinterpret_cast<const float4*>(l2s + e * kRows + r0 + 4 * h);
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int k2 = 2 * h + hh, k = 2 * k2;
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 7; ++e) {
              const float2 cf = hh ? make_float2(g2f[e].z, g2f[e].w) : make_float2(g2f[e].x, g2f[e].y);
              w = ffma2(cf, make_float2(__uint_as_float(s1u[k + e]), __uint_as_float(s1u[k + 1 + e])), w);
            }
            float2 lin = make_float2(__uint_as_float(d2u[k]), __uint_as_float(d2u[k + 1]));
#pragma unroll
            for (int e = 0; e < 5; ++e) {
              const float2 cf = hh ? make_float2(l2f[e].z, l2f[e].w) : make_float2(l2f[e].x, l2f[e].y);
              lin = ffma2(cf, make_float2(pc[k + e], pc[k + 1 + e]), lin);
            }
            w2[k2] = w;
            lin2[k2] = lin;
            pc2[k2] = make_float2(pc[k + 2], pc[k + 3]);
          }
        }
      }
      // Scatter plane j into the ring along mode 1; plane j - 3 is complete.
      const int c = j - kGramHalf;
      auto step = [&](auto tag) {
        constexpr int S = decltype(tag)::value;  // j mod 7
        if (have) {
#pragma unroll
          for (int k2 = 0; k2 < NP; ++k2) {
#pragma unroll
            for (int d = -3; d <= 3; ++d)
              acc[k2][(S + d + 7) % 7] = ffma2(bc2(g1r[3 + d]), w2[k2], acc[k2][(S + d + 7) % 7]);
#pragma unroll
            for (int d = -2; d <= 2; ++d)
              acc[k2][(S + d + 7) % 7] = ffma2(bc2(l1r[2 + d]), pc2[k2], acc[k2][(S + d + 7) % 7]);
            acc[k2][S].x += lin2[k2].x;
            acc[k2][S].y += lin2[k2].y;
            pring[k2][S] = pack_bf2(pc2[k2].x, pc2[k2].y);
          }
        }
        constexpr int E = (S + 4) % 7;
        if (c >= c0 && ok) {
          __nv_bfloat16* qo = a.q + (int64_t)c * plane + out_base;
#pragma unroll
          for (int k2 = 0; k2 < NP; ++k2) {
            const unsigned qv = pack_bf2(acc[k2][E].x, acc[k2][E].y);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int k = 2 * k2 + h;
              if ((row_ok >> k) & 1u) {
                const unsigned short qs = (unsigned short)(h ? (qv >> 16) : (qv & 0xffffu));
                *reinterpret_cast<unsigned short*>(qo + (int64_t)k * nc) = qs;
                if constexpr (CG) {
                  const float pv = h ? bf_hi(pring[k2][E]) : bf_lo(pring[k2][E]);
                  dotf = fmaf(h ? bf_hi(qv) : bf_lo(qv), pv, dotf);
                }
              }
            }
          }
        }
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) acc[k2][E] = make_float2(0.f, 0.f);
      };
      switch (j % 7) {
        case 0: step(std::integral_constant<int, 0>{}); break;
        case 1: step(std::integral_constant<int, 1>{}); break;
        case 2: step(std::integral_constant<int, 2>{}); break;
        case 3: step(std::integral_constant<int, 3>{}); break;
        case 4: step(std::integral_constant<int, 4>{}); break;
        case 5: step(std::integral_constant<int, 5>{}); break;
        default: step(std::integral_constant<int, 6>{}); break;
      }
    }
  }
  __syncthreads();
  if (*abort && tid == 0 && a.timeout_flag) atomicExch(a.timeout_flag, 1);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
  if constexpr (CG) {
    double total;
    if (dev::grid_sum_last_at((double)dotf, a.red, &total, s_red, s_last)) {
      Scalars* sc = a.scal;
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

// ---- vector kernels of the bfloat16 inner CG ----------------------------------
constexpr int kVT = 256;

// r = bf16(src) (src: the FP32 outer residual); rho = <r, r>; bnorm = ||r||;
// beta = 0 and fresh stop flags.  n % 8 == 0.
__global__ void __launch_bounds__(kVT) bf16_start_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ r,
                                                         int64_t n, Scalars* sc, Reduce red) {
  __shared__ double sh[kVT / 32];
  double acc = 0.0;
  const int64_t nv = n / 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a0 = reinterpret_cast<const float4*>(src)[2 * i];
    const float4 a1 = reinterpret_cast<const float4*>(src)[2 * i + 1];
    uint4 o;
    o.x = pack_bf2(a0.x, a0.y);
    o.y = pack_bf2(a0.z, a0.w);
    o.z = pack_bf2(a1.x, a1.y);
    o.w = pack_bf2(a1.z, a1.w);
    reinterpret_cast<uint4*>(r)[i] = o;
    float part = 0.f;
    const unsigned u[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      part = fmaf(bf_lo(u[k]), bf_lo(u[k]), part);
      part = fmaf(bf_hi(u[k]), bf_hi(u[k]), part);
    }
    acc += (double)part;
  }
  double t;
  if (dev::grid_sum_last(acc, red, &t, sh)) {
    sc->rho = t;
    sc->rho_new = t;
    sc->beta = 0.0;
    sc->bnorm = sqrt(t);
    sc->converged = 0;
    sc->breakdown = 0;
  }
}

struct BDir {
  const uint4* p[kDirBufs];  // direction written at group position i: p[(i + 1) % kDirBufs]
};

__device__ __forceinline__ void axpy8(float* x, float a, uint4 v) {
  const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    x[2 * k] = fmaf(a, bf_lo(u[k]), x[2 * k]);
    x[2 * k + 1] = fmaf(a, bf_hi(u[k]), x[2 * k + 1]);
  }
}

// r = bf16(r - alpha q); rho1 = <r, r> -> beta, stop test; grouped update of
// the correction d (FP32) over kDirBufs iterations, in iteration order (the
// same scheme as the FP32 update kernel).  n % 8 == 0.
template <bool XUPD>
__global__ void __launch_bounds__(kVT) bf16_update_kernel(float* __restrict__ d, __nv_bfloat16* __restrict__ r,
                                                          const __nv_bfloat16* __restrict__ p,
                                                          const __nv_bfloat16* __restrict__ q, int64_t n, Scalars* sc,
                                                          Reduce red, BDir pb, int pos) {
  __shared__ double sh[kVT / 32];
  if (cg_done(sc)) return;
  const double alpha_d = sc->alpha;
  const float alpha = (float)alpha_d;
  float ah[kDirBufs - 1];
  if constexpr (XUPD) {
#pragma unroll
    for (int k = 0; k < kDirBufs - 1; ++k) ah[k] = (float)sc->alpha_hist[k];
  }
  double acc = 0.0;
  const int64_t nv = n / 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 rv = reinterpret_cast<const uint4*>(r)[i];
    const uint4 qv = reinterpret_cast<const uint4*>(q)[i];
    const unsigned ru[4] = {rv.x, rv.y, rv.z, rv.w}, qu[4] = {qv.x, qv.y, qv.z, qv.w};
    unsigned o[4];
    float part = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float lo = fmaf(-alpha, bf_lo(qu[k]), bf_lo(ru[k]));
      const float hi = fmaf(-alpha, bf_hi(qu[k]), bf_hi(ru[k]));
      o[k] = pack_bf2(lo, hi);
      part = fmaf(bf_lo(o[k]), bf_lo(o[k]), part);
      part = fmaf(bf_hi(o[k]), bf_hi(o[k]), part);
    }
    reinterpret_cast<uint4*>(r)[i] = make_uint4(o[0], o[1], o[2], o[3]);
    acc += (double)part;
    if constexpr (XUPD) {
      float4 x0 = reinterpret_cast<float4*>(d)[2 * i], x1 = reinterpret_cast<float4*>(d)[2 * i + 1];
      float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int k = 0; k < kDirBufs - 1; ++k) axpy8(xs, ah[k], pb.p[k + 1][i]);
      axpy8(xs, alpha, reinterpret_cast<const uint4*>(p)[i]);
      reinterpret_cast<float4*>(d)[2 * i] = make_float4(xs[0], xs[1], xs[2], xs[3]);
      reinterpret_cast<float4*>(d)[2 * i + 1] = make_float4(xs[4], xs[5], xs[6], xs[7]);
    }
  }
  double total;
  if (dev::grid_sum_last(acc, red, &total, sh)) {
    const double rho = sc->rho;
    sc->rho_new = total;
    sc->beta = total / rho;
    sc->rho = total;
    sc->iters += 1;
    if constexpr (XUPD) {
      sc->npend = 0;
    } else {
      sc->alpha_hist[pos] = alpha_d;
      sc->npend = pos + 1;
    }
    if (!isfinite(total)) sc->breakdown = 1;
    if (sqrt(total) <= sc->rtol * sc->bnorm) sc->converged = 1;
  }
}

// The grouped update still pending when the loop stops: d += alpha_k p_k.
__global__ void __launch_bounds__(kVT) bf16_flush_kernel(float* __restrict__ d, int64_t n, Scalars* sc, Reduce red,
                                                         BDir pb) {
  __shared__ double sh[kVT / 32];
  const int np = sc->npend;
  if (np > 0) {
    const int64_t nv = n / 8;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
      float4 x0 = reinterpret_cast<float4*>(d)[2 * i], x1 = reinterpret_cast<float4*>(d)[2 * i + 1];
      float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      for (int k = 0; k < np; ++k) axpy8(xs, (float)sc->alpha_hist[k], pb.p[k + 1][i]);
      reinterpret_cast<float4*>(d)[2 * i] = make_float4(xs[0], xs[1], xs[2], xs[3]);
      reinterpret_cast<float4*>(d)[2 * i + 1] = make_float4(xs[4], xs[5], xs[6], xs[7]);
    }
  }
  double total;
  if (dev::grid_sum_last(0.0, red, &total, sh)) sc->npend = 0;
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}
__global__ void bf16_to_f32_kernel(const __nv_bfloat16* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __bfloat162float(x[i]);
}

}  // namespace tb

// Round a double to the nearest bfloat16 (ties to even), as raw bits: the
// value is first rounded to float (nearest), then its 16 low bits are rounded
// off by the IEEE rule; NaN stays NaN.
uint16_t host_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x7fffffu)) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

}  // namespace

// Shapes the tensor-core sweep takes: banded factors, the inner axis n3 n4 (or
// n3 for order 3) a multiple of 8 (16-byte rows of bfloat16), n4 <= 8 (the
// inner window stays within 22 chunks of 8).
bool bf16_shape_ok(const tca_plan_s* p) {
  if (!p->all_band) return false;
  const int64_t n4 = p->d == 4 ? p->n[3] : 1;
  const int64_t nc = p->d == 4 ? p->n[2] * p->n[3] : p->n[2];
  if (n4 > 8 || nc % 8 != 0) return false;
  if (p->n[0] > INT32_MAX || p->n[1] > INT32_MAX || nc > INT32_MAX / 2) return false;
  return true;
}

static bool encode_bf16_view(CUtensorMap* map, const void* base, int64_t n1, int64_t n2, int64_t nc, int KC) {
  // {n_c, n2 rows, n1 planes}; box {8 KC, 22, 1}: one 16 KC-byte run per halo row.
  const uint64_t dims[3] = {(uint64_t)nc, (uint64_t)n2, (uint64_t)n1};
  const uint64_t strides[2] = {(uint64_t)nc * 2, (uint64_t)n2 * nc * 2};
  const uint32_t box[3] = {(uint32_t)(8 * KC), (uint32_t)tb::kHalo, 1};
  return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, 3, dims, strides, box);
}

// Build (once) the bfloat16 state of a plan: the W = G_3 kron G_4 and
// R = lambda (L_3 kron I + I kron L_4) tiles of every inner tile in the MMA
// operand layout (computed in FP64 on the host from the plan's FP64 bands,
// rounded to bfloat16), the bfloat16 CG vectors and their tensor maps.
tca_status bf16_prepare(tca_plan_s* p) {
  Bf16State& B = p->bf;
  if (B.wt) return TCA_OK;
  if (!bf16_shape_ok(p)) return TCA_ERR_UNSUPPORTED;
  const int d = p->d;
  const int64_t n3 = p->n[2], n4 = d == 4 ? p->n[3] : 1;
  B.nc = n3 * n4;
  B.H = (int)(((3 * n4) + 7) / 8 * 8);
  B.KC = (tb::kTileC + 2 * B.H) / 8;
  B.ctiles = (int)((B.nc + tb::kTileC - 1) / tb::kTileC);
  // FP64 bands of modes 3 and 4 (mode 4 of an order-3 plan: the identity).
  std::vector<double> g3(n3 * 7), l3(n3 * 5), g4(n4 * 7, 0.0), l4(n4 * 5, 0.0);
  TCA_CUDA_TRY(cudaMemcpy(g3.data(), p->mode[2].gram.band.w64, sizeof(double) * g3.size(), cudaMemcpyDeviceToHost));
  TCA_CUDA_TRY(cudaMemcpy(l3.data(), p->mode[2].lap.w64, sizeof(double) * l3.size(), cudaMemcpyDeviceToHost));
  if (d == 4) {
    TCA_CUDA_TRY(cudaMemcpy(g4.data(), p->mode[3].gram.band.w64, sizeof(double) * g4.size(), cudaMemcpyDeviceToHost));
    TCA_CUDA_TRY(cudaMemcpy(l4.data(), p->mode[3].lap.w64, sizeof(double) * l4.size(), cudaMemcpyDeviceToHost));
  } else {
    g4[3] = 1.0;
  }
  const int KC = B.KC, H = B.H;
  const size_t tile_elems = (size_t)KC * tb::kTileC * 8;  // bfloat16 per operand tile
  std::vector<uint16_t> host((size_t)B.ctiles * 2 * tile_elems, 0);
  for (int t = 0; t < B.ctiles; ++t) {
    uint16_t* W = host.data() + (size_t)t * 2 * tile_elems;
    uint16_t* R = W + tile_elems;
    for (int cl = 0; cl < tb::kTileC; ++cl) {
      const int64_t co = (int64_t)t * tb::kTileC + cl;
      if (co >= B.nc) continue;
      const int64_t i3o = co / n4, i4o = co % n4;
      for (int kc = 0; kc < KC; ++kc)
        for (int e = 0; e < 8; ++e) {
          const int64_t ci = (int64_t)t * tb::kTileC - H + kc * 8 + e;
          if (ci < 0 || ci >= B.nc) continue;
          const int64_t i3 = ci / n4, i4 = ci % n4, d3 = i3 - i3o, d4 = i4 - i4o;
          double w = 0.0, rr = 0.0;
          if (std::abs(d3) <= 3 && std::abs(d4) <= 3) w = g3[i3o * 7 + d3 + 3] * g4[i4o * 7 + d4 + 3];
          if (d4 == 0 && std::abs(d3) <= 2) rr += l3[i3o * 5 + d3 + 2];
          if (d3 == 0 && std::abs(d4) <= 2) rr += l4[i4o * 5 + d4 + 2];
          const size_t off = ((size_t)kc * tb::kTileC + cl) * 8 + e;  // [chunk][c'][8]
          W[off] = host_bf16(w);
          R[off] = host_bf16(rr);
        }
    }
  }
  const size_t N = (size_t)p->N;
  cudaError_t e = cudaMalloc((void**)&B.wt, sizeof(uint16_t) * host.size());
  if (e == cudaSuccess) e = cudaMemcpy(B.wt, host.data(), sizeof(uint16_t) * host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.r, 2 * N);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.q, 2 * N);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.x, 2 * N);
  for (int k = 0; k < kDirBufs && e == cudaSuccess; ++k) e = cudaMalloc((void**)&B.p[k], 2 * N);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  // TMA when every box fits inside the tensor; cp.async pieces otherwise.
  const int64_t n1 = p->n[0], n2 = p->n[1];
  B.tma = n2 >= tb::kHalo && B.nc / 8 >= KC && encode_bf16_view(&B.tm_r, B.r, n1, n2, B.nc, KC) &&
          encode_bf16_view(&B.tm_x, B.x, n1, n2, B.nc, KC);
  for (int k = 0; k < kDirBufs && B.tma; ++k) B.tma = encode_bf16_view(&B.tm_p[k], B.p[k], n1, n2, B.nc, KC);
  return TCA_OK;
}

void bf16_release(tca_plan_s* p) {
  Bf16State& B = p->bf;
  cudaFree(B.wt);
  cudaFree(B.r);
  cudaFree(B.q);
  cudaFree(B.x);
  for (int k = 0; k < kDirBufs; ++k) cudaFree(B.p[k]);
  B = Bf16State{};
}

// One sweep.  CG (pold_idx >= 0): p_new = r + beta p[pold_idx], q = K p_new,
// <p_new, q> -> alpha.  Plain (pold_idx < 0): q = K x for the plan's bfloat16
// staging buffer x.
tca_status bf16_sweep(tca_plan_s* p, int pold_idx, __nv_bfloat16* pnew, __nv_bfloat16* q, cudaStream_t s) {
  Bf16State& B = p->bf;
  if (!B.wt) return TCA_ERR_UNSUPPORTED;
  const bool cg = pold_idx >= 0;
  tb::Args a{};
  a.r = B.r;
  a.pold = cg ? B.p[pold_idx] : B.x;
  a.pnew = pnew;
  a.q = q;
  a.wt = reinterpret_cast<const uint4*>(B.wt);
  a.g1 = p->mode[0].gram.band.w32;
  a.l1 = p->mode[0].lap.w32;
  a.g2 = p->mode[1].gram.band.w32;
  a.l2 = p->mode[1].lap.w32;
  a.n1 = (int)p->n[0];
  a.n2 = (int)p->n[1];
  a.nc = (int)B.nc;
  a.H = B.H;
  a.KC = B.KC;
  a.ctiles = B.ctiles;
  a.scal = p->scal;
  a.red = p->red;
  a.timeout_flag = wait_timeout_flag();
  a.tma = B.tma ? 1 : 0;
  if (B.tma) {
    a.tm_r = B.tm_r;
    a.tm_p = cg ? B.tm_p[pold_idx] : B.tm_x;
  }
  const int rtiles = (a.n2 + tb::kRows - 1) / tb::kRows;
  const int tiles = rtiles * a.ctiles;
  // Chunks along mode 1: whole waves of one CTA per SM against the +-3 plane
  // halo each chunk reloads (the same model as the FP32 sweep), unless the
  // autotuner chose them.
  int best_nc = 1;
  double best_cost = 1e30;
  for (int nch = 1; nch <= a.n1; ++nch) {
    const int len = (a.n1 + nch - 1) / nch;
    if ((int64_t)tiles * nch > p->red.max_blocks) break;
    if (len + 2 * kGramHalf > tb::kMaxPlanes) continue;
    const int64_t waves = ((int64_t)tiles * nch + p->num_sms - 1) / p->num_sms;
    const double cost = (double)waves * (len + 2 * kGramHalf);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best_nc = nch;
    }
  }
  if (B.nchunks > 0 && (int64_t)tiles * B.nchunks <= p->red.max_blocks &&
      (a.n1 + B.nchunks - 1) / B.nchunks + 2 * kGramHalf <= tb::kMaxPlanes)
    best_nc = std::min(B.nchunks, a.n1);
  a.chunk = (a.n1 + best_nc - 1) / best_nc;
  if (a.chunk + 2 * kGramHalf > tb::kMaxPlanes) return TCA_ERR_UNSUPPORTED;
  a.nchunks = (a.n1 + a.chunk - 1) / a.chunk;
  B.model_nchunks = best_nc;
  const int grid = tiles * a.nchunks;
  if (grid > p->red.max_blocks) return TCA_ERR_UNSUPPORTED;
  // Worker layout: 8 rows per thread (8 worker warps) or 4 (16 worker warps).
  const int rpt = B.rpt == 8 ? 8 : 4;
  const int threads = 64 + 128 * (tb::kRows / rpt);
  const tb::Smem L(B.KC, cg ? 2 : 1, threads / 32);
  const size_t bytes = (size_t)L.total;
  void (*kfn)(tb::Args);
  if (rpt == 8) kfn = cg ? tb::bf16_sweep_kernel<true, 8> : tb::bf16_sweep_kernel<false, 8>;
  else kfn = cg ? tb::bf16_sweep_kernel<true, 4> : tb::bf16_sweep_kernel<false, 4>;
  static bool attr_done[2][2] = {};
  bool& done = attr_done[cg ? 1 : 0][rpt == 8 ? 1 : 0];
  if (!done) {
    const tb::Smem Lmax(22, cg ? 2 : 1, threads / 32);
    TCA_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, Lmax.total));
    done = true;
  }
  kfn<<<grid, threads, bytes, s>>>(a);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// y = K x through the bfloat16 sweep, for a float x and y (tca_apply_normal on
// a TCA_BF16_IR plan): x rounded to bfloat16, one plain sweep, q widened.
tca_status normal_bf16(tca_plan_s* p, const float* x, float* y, cudaStream_t s) {
  TCA_TRY(bf16_prepare(p));
  const int grid = std::min<int64_t>((p->N + 255) / 256, (int64_t)p->num_sms * 8);
  tb::f32_to_bf16_kernel<<<grid, 256, 0, s>>>(x, p->bf.x, p->N);
  TCA_LAUNCH_CHECK();
  TCA_TRY(bf16_sweep(p, -1, nullptr, p->bf.q, s));
  tb::bf16_to_f32_kernel<<<grid, 256, 0, s>>>(p->bf.q, y, p->N);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// Inner-CG vector kernels (launch helpers used by the solver).
tca_status bf16_start(tca_plan_s* p, const float* src, Reduce red, cudaStream_t s) {
  const int grid = std::min<int64_t>(std::max<int64_t>(1, (p->N / 8 + 255) / 256),
                                     std::min<int64_t>((int64_t)p->num_sms * 8, red.max_blocks));
  tb::bf16_start_kernel<<<grid, tb::kVT, 0, s>>>(src, p->bf.r, p->N, p->scal, red);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

tca_status bf16_update(tca_plan_s* p, float* d, int pos, Reduce red, cudaStream_t s) {
  Bf16State& B = p->bf;
  const int grid = std::min<int64_t>(std::max<int64_t>(1, (p->N / 8 + 255) / 256),
                                     std::min<int64_t>((int64_t)p->num_sms * 8, red.max_blocks));
  tb::BDir pb;
  for (int k = 0; k < kDirBufs; ++k) pb.p[k] = reinterpret_cast<const uint4*>(B.p[k]);
  const __nv_bfloat16* pnew = B.p[(pos + 1) % kDirBufs];
  if (pos == kDirBufs - 1)
    tb::bf16_update_kernel<true><<<grid, tb::kVT, 0, s>>>(d, B.r, pnew, B.q, p->N, p->scal, red, pb, pos);
  else
    tb::bf16_update_kernel<false><<<grid, tb::kVT, 0, s>>>(d, B.r, pnew, B.q, p->N, p->scal, red, pb, pos);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

tca_status bf16_flush(tca_plan_s* p, float* d, Reduce red, cudaStream_t s) {
  const int grid = std::min<int64_t>(std::max<int64_t>(1, (p->N / 8 + 255) / 256),
                                     std::min<int64_t>((int64_t)p->num_sms * 8, red.max_blocks));
  tb::BDir pb;
  for (int k = 0; k < kDirBufs; ++k) pb.p[k] = reinterpret_cast<const uint4*>(p->bf.p[k]);
  tb::bf16_flush_kernel<<<grid, tb::kVT, 0, s>>>(d, p->N, p->scal, red, pb);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace tca
