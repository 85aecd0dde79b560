// Fused normal-operator sweep:  q = (G_1 kron G_2 kron G_3 kron G_4) p + lambda sum_k L_k p
// for banded factors, in one pass over p (FP32 data, FP32 arithmetic).
//
// This is the "iterative application of the tensor multiplication" that every
// CG step performs (Sec. 4.1, Fig. 2, Q = A.P), with the separable structure of
// Eq. separable_transf applied mode by mode inside one tile (Sec. 4.1 Poisson
// example: sequential one-dimensional transformations along each dimension).
// G_k = A_k^T A_k is 7-banded, L_k = D2_k^T D2_k is 5-banded (lambda folded in).
//
// Schedule.  A CTA owns an in-plane tile (T2 x T3 x n4, full fastest mode) and a
// run of planes along mode 1, and marches along mode 1:
//   load plane j of p with a +-3 halo in modes 2 and 3  (cp.async, STAGES deep)
//   stage A: G_3 then G_4 along rows of the halo tile      -> S1 (halo rows kept)
//            lambda (L_3 + L_4) p on core rows              -> SL
//   stage B: G_2 down each column -> w;  lambda L_2 p + SL -> lin
//            scatter into 7 register accumulators: plane j contributes
//            G_1[j+d][j] w (|d|<=3) and lambda L_1[j+d][j] p (|d|<=2);
//            plane j-3 is then complete and is written out.
// In CG mode the kernel also forms the new direction p = r + beta p_old on the
// fly (halo included), stores it, and reduces <p, q> to alpha = rho / <p, q>
// (last block; Fig. 2, alpha := rho/(P+*Q)).
//
// Shared-memory layout is chosen for conflict-free access: every row pitch holds
// an odd number of 16-byte chunks and stage A maps consecutive lanes to
// consecutive rows, so eight lanes of a 128-bit access phase hit eight distinct
// bank quads; the per-stage buffers are double-buffered so that a plane costs
// two block barriers (three in CG mode).  Products are issued as packed FP32
// pairs (fma.rn.f32x2) wherever both operands pair up naturally, and the
// accumulator ring along mode 1 is indexed by compile-time slots (a switch on
// j mod 7) so it never moves between registers.
#include <cuda.h>
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "tca_internal.cuh"

namespace tca {

namespace {

struct FusedArgs {
  const float* r;      // CG: residual (may be null otherwise)
  const float* pold;   // CG: previous direction; plain: the input x
  float* pnew;         // CG: new direction out
  float* q;            // output
  const float* g[4];   // G_k bands, n_k x 7 (zeros outside [0, n_k))
  const float* l[4];   // lambda L_k bands, n_k x 5
  int n1, n2, n3;
  int chunk;           // planes per CTA along mode 1
  int tiles3;
  int nchunks;
  Scalars* scal;
  Reduce red;
  // Warp-specialised sweep (n4 = 8): G_4 and lambda L_4 by tap, then lane,
  // read straight from the parameter bank (the same for every CTA and plane).
  float g4c[7 * 8];
  float l4c[5 * 8];
  // Warp-specialised sweep with TMA halo loads: 3D maps (n3 n4, n2, n1) of r
  // and p_old, box (176, 22, 1) = one halo tile; set by the TMA launch only.
  CUtensorMap tm_r;
  CUtensorMap tm_p;
  int* timeout_flag;
  const Scalars* stop;  // plain sweep as a CG preconditioner: no work once these stop flags are set
  int pdot;             // plain warp-specialised sweep as the preconditioner of PCG: 1 / 2 also forms
                        // rho1 = <input, output> and the PCG scalars (1: a fresh start, beta = 0)
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// mbarrier and TMA (cp.async.bulk.tensor) helpers for the warp-specialised sweep.
constexpr long long kTmaWaitPolls = 1ll << 24;  // try_wait polls before a wait gives up
__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait_parity(uint64_t* bar, unsigned parity) {
  for (long long it = 0; it < kTmaWaitPolls; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(float* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// d = a * b + c on a pair of FP32 lanes (one packed FMA instruction).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

template <int N4, int T2, int T3, int T3P, int NT, int STAGES, bool CG>
struct Cfg {
  static constexpr int H2 = T2 + 6, H3 = T3 + 6;
  // Row pitches (floats) with an odd number of 16-byte chunks (odd word count
  // for N4 = 1): eight lanes on eight consecutive rows then hit eight distinct
  // bank quads.
  static constexpr int pitch(int cols) {
    return N4 == 1 ? (cols | 1) : (cols * N4 + (((cols * N4 / 4) % 2 == 0) ? 4 : 0));
  }
  static constexpr int ROW = pitch(H3);            // floats per halo-tile row
  static constexpr int TILE = ((H2 * ROW + 31) / 32) * 32;
  static constexpr int ROW1 = pitch(T3);           // floats per S1 / SL row
  static constexpr int S1N = ((H2 * ROW1 + 31) / 32) * 32;
  static constexpr int SLN = ((T2 * ROW1 + 31) / 32) * 32;
  static constexpr int CORE = T2 * T3 * N4;        // thread-private ring slots
  static constexpr int NIN = CG ? 2 : 1;
  static constexpr int RB = NT / (N4 * T3);        // row blocks in stage B
  static constexpr int P = T2 / RB;                // rows per thread in stage B
  static constexpr int NBQ = T3 / T3P;             // pencils per halo row
  static constexpr int RPB = ((H2 + 7) / 8) * 8;   // pencil slots per column block
  static_assert(NT % (N4 * T3) == 0, "stage-B mapping");
  static_assert(T2 % RB == 0 && P % 4 == 0, "stage-B rows come in pairs of pairs");
  static_assert(T3 % T3P == 0, "stage-A pencils");
  static_assert(N4 == 1 || N4 % 4 == 0, "fastest mode 1, 4 or 8");
  static constexpr int NB = CG ? 2 : 1;            // double-buffered p tile in CG mode
  // shared memory carve-up (floats)
  static constexpr int OFF_IN = 0;
  static constexpr int OFF_P = OFF_IN + STAGES * NIN * TILE;
  static constexpr int OFF_S1 = OFF_P + (CG ? NB * TILE : 0);
  static constexpr int OFF_SL = OFF_S1 + 2 * S1N;
  static constexpr int OFF_RING = OFF_SL + 2 * SLN;
  static constexpr int OFF_G3 = OFF_RING + (CG ? 4 * CORE : 0);   // [T3][8]
  static constexpr int OFF_L3 = OFF_G3 + T3 * 8;                  // [T3][8]
  static constexpr int OFF_G4 = OFF_L3 + T3 * 8;                  // [7][N4]  (offset-major)
  static constexpr int OFF_L4 = OFF_G4 + 7 * N4;                  // [5][N4]
  static constexpr int OFF_G2 = ((OFF_L4 + 5 * N4 + 3) / 4) * 4;  // [7][T2]  (offset-major)
  static constexpr int OFF_L2 = OFF_G2 + 7 * T2;                  // [5][T2]
  static constexpr int OFF_RED = ((OFF_L2 + 5 * T2 + 3) / 4) * 4; // doubles
  static constexpr int FLOATS = OFF_RED + 2 * (NT / 32);
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

template <int N4, int T2, int T3, int T3P, int NT, int STAGES, bool CG>
__global__ void __launch_bounds__(NT, 1) fused_normal_kernel(FusedArgs a) {
  using C = Cfg<N4, T2, T3, T3P, NT, STAGES, CG>;
  constexpr int H2 = C::H2, ROW = C::ROW, ROW1 = C::ROW1, P = C::P;
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;

  if constexpr (CG) {
    if (cg_done(a.scal)) return;
  } else {
    if (a.stop && cg_done(a.stop)) return;
  }
  const float beta = CG ? (float)a.scal->beta : 0.f;

  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const int bid = blockIdx.x;
  const int chunk_id = bid % a.nchunks;
  const int tile = bid / a.nchunks;
  const int t3i = tile % a.tiles3, t2i = tile / a.tiles3;
  const int i2_0 = t2i * T2, i3_0 = t3i * T3;
  const int c0 = chunk_id * a.chunk;
  const int c1 = min(n1, c0 + a.chunk);
  const int jb = max(0, c0 - kGramHalf);
  const int je = min(n1, c1 + kGramHalf);

  float* s_in = sm + C::OFF_IN;
  float* s_ring = sm + C::OFF_RING;
  float* g3s = sm + C::OFF_G3;
  float* l3s = sm + C::OFF_L3;
  float* g4s = sm + C::OFF_G4;
  float* l4s = sm + C::OFF_L4;
  float* g2s = sm + C::OFF_G2;
  float* l2s = sm + C::OFF_L2;
  double* s_red = reinterpret_cast<double*>(sm + C::OFF_RED);

  // Tile coefficient tables (entries outside the domain are zero).
  for (int t = tid; t < T3 * 8; t += NT) {
    const int r = t >> 3, e = t & 7, i3 = i3_0 + r;
    g3s[t] = (i3 < n3 && e < 7) ? a.g[2][(int64_t)i3 * 7 + e] : 0.f;
    l3s[t] = (i3 < n3 && e < 5) ? a.l[2][(int64_t)i3 * 5 + e] : 0.f;
  }
  for (int t = tid; t < 7 * T2; t += NT) {
    const int e = t / T2, r = t % T2, i2 = i2_0 + r;
    g2s[t] = i2 < n2 ? a.g[1][(int64_t)i2 * 7 + e] : 0.f;
    if (e < 5) l2s[t] = i2 < n2 ? a.l[1][(int64_t)i2 * 5 + e] : 0.f;
  }
  if constexpr (N4 > 1) {
    for (int t = tid; t < 7 * N4; t += NT) {
      const int e = t / N4, i4 = t % N4;
      g4s[t] = a.g[3][i4 * 7 + e];
      if (e < 5) l4s[t] = a.l[3][i4 * 5 + e];
    }
  }

  const int64_t plane = (int64_t)n2 * n3 * N4;

  // Asynchronous copies of plane jj (halo tile) into stage buffer buf.
  // Each thread's share of the halo-tile copy is the same for every plane:
  // its shared-memory offsets and in-plane source offsets (-1: outside the
  // domain, zero fill) are computed once.
  constexpr int CW = (N4 % 4 == 0) ? 4 : 1;             // floats per copy
  constexpr int ELEMS = H2 * C::H3 * (N4 / CW);         // copies per tensor and plane
  constexpr int NCP = (ELEMS + NT - 1) / NT;
  int cp_dst[NCP], cp_src[NCP];
#pragma unroll
  for (int i = 0; i < NCP; ++i) {
    const int t = tid + i * NT;
    cp_dst[i] = -1;
    cp_src[i] = -1;
    if (t < ELEMS) {
      const int v = t % (N4 / CW), rc = t / (N4 / CW);
      const int cc = rc % C::H3, rr = rc / C::H3;
      const int i2 = i2_0 - 3 + rr, i3 = i3_0 - 3 + cc;
      const bool ok = (unsigned)i2 < (unsigned)n2 && (unsigned)i3 < (unsigned)n3;
      cp_dst[i] = rr * ROW + cc * N4 + CW * v;
      cp_src[i] = ok ? (i2 * n3 + i3) * N4 + CW * v : -1;
    }
  }
  auto issue = [&](int jj, int buf) {
#pragma unroll
    for (int src_i = 0; src_i < C::NIN; ++src_i) {
      const float* g = (CG && src_i == 0) ? a.r : a.pold;
      float* dst = s_in + (buf * C::NIN + src_i) * C::TILE;
      const float* gp = g + (int64_t)jj * plane;
#pragma unroll
      for (int i = 0; i < NCP; ++i) {
        if (cp_dst[i] < 0) continue;
        const bool ok = cp_src[i] >= 0;
        if constexpr (CW == 4) cp_async16(dst + cp_dst[i], ok ? gp + cp_src[i] : g, ok);
        else cp_async4(dst + cp_dst[i], ok ? gp + cp_src[i] : g, ok);
      }
    }
  };

  // Stage-B thread mapping: one column (bcol, i4b), P consecutive core rows.
  const int i4b = tid % N4;
  const int bcol = (tid / N4) % T3;
  const int a0 = (tid / (N4 * T3)) * P;
  const bool col_ok = (i3_0 + bcol) < n3;
  // In-plane offset of the thread's first row and a bit per row inside the domain.
  const int64_t out_base = ((int64_t)(i2_0 + a0) * n3 + i3_0 + bcol) * N4 + i4b;
  const int64_t row_step = (int64_t)n3 * N4;
  unsigned row_ok = 0;
#pragma unroll
  for (int k = 0; k < P; ++k) row_ok |= (col_ok && (i2_0 + a0 + k) < n2) ? (1u << k) : 0u;

  float2 acc[P / 2][7];
#pragma unroll
  for (int k = 0; k < P / 2; ++k)
#pragma unroll
    for (int e = 0; e < 7; ++e) acc[k][e] = make_float2(0.f, 0.f);
  double dot = 0.0;
  // Per-plane stage-B results (pairs of rows) consumed by the ring update.
  float2 w2[P / 2], lin2[P / 2], pc2[P / 2];
  float g1r[7], l1r[5];
#pragma unroll
  for (int k2 = 0; k2 < P / 2; ++k2) w2[k2] = lin2[k2] = pc2[k2] = make_float2(0.f, 0.f);
#pragma unroll
  for (int e = 0; e < 7; ++e) g1r[e] = 0.f;
#pragma unroll
  for (int e = 0; e < 5; ++e) l1r[e] = 0.f;

#pragma unroll 1
  for (int s = 0; s < STAGES - 1; ++s) {
    if (jb + s < je) issue(jb + s, s);
    cp_async_commit();
  }

#pragma unroll 1
  for (int j = jb; j < c1 + kGramHalf; ++j) {
    const int it = j - jb;
    const bool have = j < je;
    const int par = it & 1;
    if (have) {
      cp_async_wait<STAGES - 2>();
      // Plane j landed for every thread; every thread is also done with plane
      // j-1, whose stage buffer the next copy reuses.  (On the first pass this
      // barrier also publishes the coefficient tables.)
      __syncthreads();
      {
        const int jn = j + STAGES - 1;
        if (jn < je) issue(jn, (it + STAGES - 1) % STAGES);
        cp_async_commit();
      }
      const int buf = it % STAGES;
      const float* src;
      if constexpr (CG) {
        const float4* rr = reinterpret_cast<const float4*>(s_in + (buf * 2 + 0) * C::TILE);
        const float4* pp = reinterpret_cast<const float4*>(s_in + (buf * 2 + 1) * C::TILE);
        float* pdst = sm + C::OFF_P + par * C::TILE;
        float4* out = reinterpret_cast<float4*>(pdst);
        for (int t = tid; t < C::TILE / 4; t += NT) {
          const float4 x = rr[t], y = pp[t];
          out[t] = make_float4(fmaf(beta, y.x, x.x), fmaf(beta, y.y, x.y), fmaf(beta, y.z, x.z),
                               fmaf(beta, y.w, x.w));
        }
        __syncthreads();
        src = pdst;
      } else {
        src = s_in + buf * C::TILE;
      }
      float* s_s1 = sm + C::OFF_S1 + par * C::S1N;
      float* s_sl = sm + C::OFF_SL + par * C::SLN;

      // ---- stage A: G_3 then G_4 along rows of the halo tile; L_3 + L_4 on core rows ----
#pragma unroll 1
      for (int slot = tid; slot < C::RPB * C::NBQ; slot += NT) {
        const int ar = slot % C::RPB;
        const int bq = slot / C::RPB;
        if (ar >= H2) continue;
        const int b0 = bq * T3P;
        constexpr int NV = (N4 + 1) / 2;  // pairs per column (N4 = 1 keeps one lane in .x)
        float2 v[T3P + 6][NV];
        const float* rowp = src + ar * ROW + b0 * N4;
        if constexpr (N4 == 8) {
#pragma unroll
          for (int t = 0; t < T3P + 6; ++t) {
            const float4 lo = reinterpret_cast<const float4*>(rowp + t * N4)[0];
            const float4 hi = reinterpret_cast<const float4*>(rowp + t * N4)[1];
            v[t][0] = make_float2(lo.x, lo.y); v[t][1] = make_float2(lo.z, lo.w);
            v[t][2] = make_float2(hi.x, hi.y); v[t][3] = make_float2(hi.z, hi.w);
          }
        } else if constexpr (N4 == 4) {
#pragma unroll
          for (int t = 0; t < T3P + 6; ++t) {
            const float4 f = *reinterpret_cast<const float4*>(rowp + t * N4);
            v[t][0] = make_float2(f.x, f.y); v[t][1] = make_float2(f.z, f.w);
          }
        } else {
#pragma unroll
          for (int t = 0; t < T3P + 6; ++t) v[t][0] = make_float2(rowp[t], 0.f);
        }
        // G_3 along the row, pairs over the fastest mode.
        float2 u[T3P][NV];
#pragma unroll
        for (int t = 0; t < T3P; ++t) {
          const float4 ga = *reinterpret_cast<const float4*>(g3s + (b0 + t) * 8);
          const float4 gb = *reinterpret_cast<const float4*>(g3s + (b0 + t) * 8 + 4);
          const float gc[7] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z};
#pragma unroll
          for (int m = 0; m < NV; ++m) {
            float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 7; ++e) s2 = ffma2(bc2(gc[e]), v[t + e][m], s2);
            u[t][m] = s2;
          }
        }
        // G_4 along the fastest mode: output pair (2m, 2m+1) at offset d reads
        // (u[2m+d], u[2m+d+1]) - an aligned pair for even d, an odd pair otherwise.
        float2 o[T3P][NV];
        if constexpr (N4 > 1) {
          float2 od[T3P][NV + 1];  // od[t][k] = (u[t][2k-1], u[t][2k]), zero outside
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            od[t][0] = make_float2(0.f, u[t][0].x);
#pragma unroll
            for (int k = 1; k < NV; ++k) od[t][k] = make_float2(u[t][k - 1].y, u[t][k].x);
            od[t][NV] = make_float2(u[t][NV - 1].y, 0.f);
#pragma unroll
            for (int m = 0; m < NV; ++m) o[t][m] = make_float2(0.f, 0.f);
          }
          // One 128-bit coefficient load serves output pairs 2mm and 2mm+1 of every row t.
#pragma unroll
          for (int mm = 0; mm < NV / 2; ++mm) {
#pragma unroll
            for (int e = 0; e < 7; ++e) {
              const int d = e - 3;
              const float4 c4 = *reinterpret_cast<const float4*>(g4s + e * N4 + 4 * mm);
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const int m = 2 * mm + hh;
                const float2 cf = hh ? make_float2(c4.z, c4.w) : make_float2(c4.x, c4.y);
#pragma unroll
                for (int t = 0; t < T3P; ++t) {
                  if ((d & 1) == 0) {
                    const int pi = m + d / 2;
                    if (pi >= 0 && pi < NV) o[t][m] = ffma2(cf, u[t][pi], o[t][m]);
                  } else {
                    const int pi = m + (d + 1) / 2;
                    if (pi >= 0 && pi <= NV) o[t][m] = ffma2(cf, od[t][pi], o[t][m]);
                  }
                }
              }
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < T3P; ++t) o[t][0] = u[t][0];
        }
#pragma unroll
        for (int t = 0; t < T3P; ++t) {
          float* dst = s_s1 + ar * ROW1 + (b0 + t) * N4;
          if constexpr (N4 == 8) {
            reinterpret_cast<float4*>(dst)[0] = make_float4(o[t][0].x, o[t][0].y, o[t][1].x, o[t][1].y);
            reinterpret_cast<float4*>(dst)[1] = make_float4(o[t][2].x, o[t][2].y, o[t][3].x, o[t][3].y);
          } else if constexpr (N4 == 4) {
            *reinterpret_cast<float4*>(dst) = make_float4(o[t][0].x, o[t][0].y, o[t][1].x, o[t][1].y);
          } else {
            dst[0] = o[t][0].x;
          }
        }
        if (ar >= 3 && ar < 3 + T2) {
          float2 lin[T3P][NV];
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            const float4 la = *reinterpret_cast<const float4*>(l3s + (b0 + t) * 8);
            const float lc[5] = {la.x, la.y, la.z, la.w, l3s[(b0 + t) * 8 + 4]};
#pragma unroll
            for (int m = 0; m < NV; ++m) {
              float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
              for (int e = 0; e < 5; ++e) s2 = ffma2(bc2(lc[e]), v[t + 1 + e][m], s2);
              lin[t][m] = s2;
            }
          }
          if constexpr (N4 > 1) {
            float2 od[T3P][NV + 1];  // odd pairs of the centre column v[t + 3]
#pragma unroll
            for (int t = 0; t < T3P; ++t) {
              od[t][0] = make_float2(0.f, v[t + 3][0].x);
#pragma unroll
              for (int k = 1; k < NV; ++k) od[t][k] = make_float2(v[t + 3][k - 1].y, v[t + 3][k].x);
              od[t][NV] = make_float2(v[t + 3][NV - 1].y, 0.f);
            }
#pragma unroll
            for (int mm = 0; mm < NV / 2; ++mm) {
#pragma unroll
              for (int e = 0; e < 5; ++e) {
                const int d = e - 2;
                const float4 c4 = *reinterpret_cast<const float4*>(l4s + e * N4 + 4 * mm);
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                  const int m = 2 * mm + hh;
                  const float2 cf = hh ? make_float2(c4.z, c4.w) : make_float2(c4.x, c4.y);
#pragma unroll
                  for (int t = 0; t < T3P; ++t) {
                    if ((d & 1) == 0) {
                      const int pi = m + d / 2;
                      if (pi >= 0 && pi < NV) lin[t][m] = ffma2(cf, v[t + 3][pi], lin[t][m]);
                    } else {
                      const int pi = m + (d + 1) / 2;
                      if (pi >= 0 && pi <= NV) lin[t][m] = ffma2(cf, od[t][pi], lin[t][m]);
                    }
                  }
                }
              }
            }
          }
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            float* dst = s_sl + (ar - 3) * ROW1 + (b0 + t) * N4;
            if constexpr (N4 == 8) {
              reinterpret_cast<float4*>(dst)[0] = make_float4(lin[t][0].x, lin[t][0].y, lin[t][1].x, lin[t][1].y);
              reinterpret_cast<float4*>(dst)[1] = make_float4(lin[t][2].x, lin[t][2].y, lin[t][3].x, lin[t][3].y);
            } else if constexpr (N4 == 4) {
              *reinterpret_cast<float4*>(dst) = make_float4(lin[t][0].x, lin[t][0].y, lin[t][1].x, lin[t][1].y);
            } else {
              dst[0] = lin[t][0].x;
            }
          }
        }
      }
      __syncthreads();

      // ---- stage B: G_2 down columns and L_2; per-row results for the scatter ----
      {
        float s1c[P + 6];
#pragma unroll
        for (int k = 0; k < P + 6; ++k) s1c[k] = s_s1[(a0 + k) * ROW1 + bcol * N4 + i4b];
        float s0c[P + 4];
#pragma unroll
        for (int k = 0; k < P + 4; ++k) s0c[k] = src[(a0 + 1 + k) * ROW + (bcol + 3) * N4 + i4b];
#pragma unroll
        for (int e = 0; e < 7; ++e) g1r[e] = __ldg(a.g[0] + (int64_t)j * 7 + e);
#pragma unroll
        for (int e = 0; e < 5; ++e) l1r[e] = __ldg(a.l[0] + (int64_t)j * 5 + e);
        const bool own_plane = (j >= c0) && (j < c1);
        float* pn = CG ? a.pnew + (int64_t)j * plane + out_base : nullptr;
#pragma unroll
        for (int h = 0; h < P / 4; ++h) {
          // Coefficients of rows a0+4h .. a0+4h+3, one 128-bit load per offset.
          float4 g2f[7], l2f[5];
#pragma unroll
          for (int e = 0; e < 7; ++e) g2f[e] = *reinterpret_cast<const float4*>(g2s + e * T2 + a0 + 4 * h);
#pragma unroll
          for (int e = 0; e < 5; ++e) l2f[e] = *reinterpret_cast<const float4*>(l2s + e * T2 + a0 + 4 * h);
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int k2 = 2 * h + hh;
            const int k = 2 * k2;
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 7; ++e) {
              const float2 cf = hh ? make_float2(g2f[e].z, g2f[e].w) : make_float2(g2f[e].x, g2f[e].y);
              w = ffma2(cf, make_float2(s1c[k + e], s1c[k + 1 + e]), w);
            }
            float2 lin = make_float2(s_sl[(a0 + k) * ROW1 + bcol * N4 + i4b],
                                     s_sl[(a0 + k + 1) * ROW1 + bcol * N4 + i4b]);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
              const float2 cf = hh ? make_float2(l2f[e].z, l2f[e].w) : make_float2(l2f[e].x, l2f[e].y);
              lin = ffma2(cf, make_float2(s0c[k + e], s0c[k + 1 + e]), lin);
            }
            const float2 pcv = make_float2(s0c[k + 2], s0c[k + 3]);
            w2[k2] = w;
            lin2[k2] = lin;
            pc2[k2] = pcv;
            if constexpr (CG) {
              float* ring = s_ring + (j & 3) * C::CORE;
              ring[(k) * NT + tid] = pcv.x;
              ring[(k + 1) * NT + tid] = pcv.y;
              if (own_plane && ((row_ok >> k) & 1u)) pn[k * row_step] = pcv.x;
              if (own_plane && ((row_ok >> (k + 1)) & 1u)) pn[(k + 1) * row_step] = pcv.y;
            }
          }
        }
      }
    }
    // ---- scatter plane j into the ring along mode 1, emit plane j-3 ----
    // acc[.][s] accumulates plane c with s = c mod 7; the switch makes every
    // slot index a compile-time constant so the ring stays in registers.
    const int c = j - kGramHalf;
    auto step = [&](auto tag) {
      constexpr int S = decltype(tag)::value;  // j mod 7
      if (have) {
#pragma unroll
        for (int k2 = 0; k2 < P / 2; ++k2) {
#pragma unroll
          for (int d = -3; d <= 3; ++d)
            acc[k2][(S + d + 7) % 7] = ffma2(bc2(g1r[3 + d]), w2[k2], acc[k2][(S + d + 7) % 7]);
#pragma unroll
          for (int d = -2; d <= 2; ++d)
            acc[k2][(S + d + 7) % 7] = ffma2(bc2(l1r[2 + d]), pc2[k2], acc[k2][(S + d + 7) % 7]);
          acc[k2][S].x += lin2[k2].x;
          acc[k2][S].y += lin2[k2].y;
        }
      }
      constexpr int E = (S + 4) % 7;  // slot of plane j-3
      if (c >= c0) {
        float part = 0.f;
        float* qo = a.q + (int64_t)c * plane + out_base;
        const float* ring = s_ring + (c & 3) * C::CORE + tid;
#pragma unroll
        for (int k2 = 0; k2 < P / 2; ++k2) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int k = 2 * k2 + h;
            if ((row_ok >> k) & 1u) {
              const float qv = h ? acc[k2][E].y : acc[k2][E].x;
              qo[k * row_step] = qv;
              if constexpr (CG) part = fmaf(qv, ring[k * NT], part);
            }
          }
        }
        dot += (double)part;
      }
#pragma unroll
      for (int k2 = 0; k2 < P / 2; ++k2) acc[k2][E] = make_float2(0.f, 0.f);
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
  cp_async_wait<0>();

  if constexpr (CG) {
    double total;
    if (dev::grid_sum_last(dot, a.red, &total, s_red)) {
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

// ---------------------------------------------------------------------------
// Warp-specialised variant for n4 = 8 (the 4D workloads): the same sweep with
// the work of a plane split between two warp groups that run one plane apart.
//   loader/in-plane warps (A, 8 warps): copy the halo tiles of r and p_old
//     (one TMA box per tensor and plane into a 3-stage mbarrier ring, or
//     cp.async when the tile is wider than the tensor or a tensor is not
//     16-byte aligned), form p = r + beta p_old, apply G_3, G_4 along the
//     rows of the halo tile (S1) and lambda (L_3 + L_4) on the core rows (SL);
//   column/ring warps (B, 8 warps): G_2 and lambda L_2 down the columns, the
//     scatter into the 7-slot register ring along mode 1, the outputs q and
//     p_new and the partial <p, q>.
// A hands plane j to B through the double-buffered P / S1 / SL tiles and two
// pairs of named barriers (FULL: A -> B, EMPTY: B -> A), so A's in-plane work
// on plane j + 1 overlaps B's column and ring work on plane j.  The groups
// rebalance the register file (setmaxnreg): only B holds the ring.
namespace ws {

constexpr int NA = 256, NB = 256, NT = NA + NB;
constexpr int REG_A = 104, REG_B = 152;  // 256 x 112 + 256 x 144 = 65536 = 512 x 128 at launch
constexpr int BAR_A = 1, BAR_FULL = 2, BAR_EMPTY = 4;
constexpr int kMaxPlanes = 256;  // planes a CTA may visit (chunk + 6): size of the G1 / L1 table

__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <bool CG, bool TMA, bool PDOT>
__global__ void __launch_bounds__(NT, 1) fused_ws_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int N4 = 8, T2 = 16, T3 = 16, T3P = 2, STAGES = 3;
  using C = Cfg<N4, T2, T3, T3P, NB, STAGES, true>;  // smem layout of the CG configuration (P tiles, ring)
  constexpr int H2 = C::H2, ROW = C::ROW, ROW1 = C::ROW1, P = C::P;
  constexpr int NIN = CG ? 2 : 1;
  // No static shared memory in this kernel (the reduction's flag lives in the
  // dynamic block too), so the dynamic block starts at the 128-byte aligned
  // base that the TMA stages need; checked below.
  extern __shared__ __align__(128) float sm[];
  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  if constexpr (CG) {
    if (cg_done(a.scal)) return;
  } else {
    if (a.stop && cg_done(a.stop)) return;
  }
  const float beta = CG ? (float)a.scal->beta : 0.f;

  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const int bid = blockIdx.x;
  const int chunk_id = bid % a.nchunks;
  const int tile = bid / a.nchunks;
  const int t3i = tile % a.tiles3, t2i = tile / a.tiles3;
  const int i2_0 = t2i * T2, i3_0 = t3i * T3;
  const int c0 = chunk_id * a.chunk;
  const int c1 = min(n1, c0 + a.chunk);
  const int jb = max(0, c0 - kGramHalf);
  const int je = min(n1, c1 + kGramHalf);
  const int nplanes = je - jb;

  float* s_in = sm + C::OFF_IN;
  float* s_ring = sm + C::OFF_RING;
  float* g3s = sm + C::OFF_G3;
  float* l3s = sm + C::OFF_L3;
  float* g4s = sm + C::OFF_G4;
  float* l4s = sm + C::OFF_L4;
  float* g2s = sm + C::OFF_G2;
  float* l2s = sm + C::OFF_L2;
  double* s_red = reinterpret_cast<double*>(sm + C::OFF_RED);
  // TMA: one mbarrier per stage and a CTA-wide give-up flag after the reduction scratch.
  uint64_t* tbar = reinterpret_cast<uint64_t*>(sm + C::OFF_RED + 2 * (NT / 32));
  volatile int* s_abort = reinterpret_cast<volatile int*>(tbar + STAGES);
  volatile int* s_last = s_abort + 1;
  // Plain sweep: G1 (7 taps) and lambda L1 (5 taps) of every plane this CTA
  // visits, one 16-float row per plane (read by B with three broadcast 16-byte
  // loads).  The CG sweep, short of registers in B, reads them from global.
  float* s_g1l1 = reinterpret_cast<float*>(tbar + 4);
  if (TMA && tid == 0) {
    for (int b = 0; b < STAGES; ++b) mbar_init1(&tbar[b]);
    // A stage off the 128-byte grid would fault the copy: give up instead
    // (no copies, no waits, error flag set; the sweep's output is invalid).
    const bool misaligned = (smem_u32(sm) & 127u) != 0;
    *s_abort = misaligned ? 1 : 0;
    if (misaligned && a.timeout_flag) atomicExch(a.timeout_flag, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  for (int t = tid; t < T3 * 8; t += NT) {
    const int r = t >> 3, e = t & 7, i3 = i3_0 + r;
    g3s[t] = (i3 < n3 && e < 7) ? a.g[2][(int64_t)i3 * 7 + e] : 0.f;
    l3s[t] = (i3 < n3 && e < 5) ? a.l[2][(int64_t)i3 * 5 + e] : 0.f;
  }
  for (int t = tid; t < 7 * T2; t += NT) {
    const int e = t / T2, r = t % T2, i2 = i2_0 + r;
    g2s[t] = i2 < n2 ? a.g[1][(int64_t)i2 * 7 + e] : 0.f;
    if (e < 5) l2s[t] = i2 < n2 ? a.l[1][(int64_t)i2 * 5 + e] : 0.f;
  }
  for (int t = tid; t < 7 * N4; t += NT) {
    const int e = t / N4, i4 = t % N4;
    g4s[t] = a.g[3][i4 * 7 + e];
    if (e < 5) l4s[t] = a.l[3][i4 * 5 + e];
  }
  for (int t = tid; !CG && t < nplanes * 16; t += NT) {
    const int pl = t >> 4, e = t & 15, jj = jb + pl;
    s_g1l1[t] = e < 7 ? a.g[0][(int64_t)jj * 7 + e] : (e < 12 ? a.l[0][(int64_t)jj * 5 + (e - 7)] : 0.f);
  }
  __syncthreads();

  const int64_t plane = (int64_t)n2 * n3 * N4;
  double dot = 0.0;

  if (warp < NA / 32) {
    // ======================= A: loads, p, stage A =======================
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_A));
    constexpr int ELEMS = H2 * C::H3 * 2;  // 16-byte copies per tensor and plane
    constexpr int NCP = TMA ? 1 : (ELEMS + NA - 1) / NA;
    int cp_dst[NCP], cp_src[NCP];
    // TMA: one thread of warp 7 (idle in stage A) copies each tensor's 22 x 22
    // x 8 halo tile as one box into its stage, densely packed (row pitch
    // H3 * N4); the p pass re-pitches it into the padded P tile.
    constexpr int TMA_WARP = NA / 32 - 1;
    constexpr unsigned TMA_BYTES = NIN * H2 * C::H3 * N4 * sizeof(float);
    static_assert((C::TILE * sizeof(float)) % 128 == 0, "TMA stages must stay 128-byte aligned");
    int n_issued = 0;  // issuing thread: planes jb .. jb + n_issued - 1 copied (in order)
    auto issue_tma = [&](int jj, int b) {
      if ((tid & 31) == 0 && !*s_abort) {
        n_issued = jj - jb + 1;
        mbar_expect_tx(&tbar[b], TMA_BYTES);
#pragma unroll
        for (int src_i = 0; src_i < NIN; ++src_i)
          tma_load_3d(s_in + (b * 2 + src_i) * C::TILE, (CG && src_i == 0) ? &a.tm_r : &a.tm_p, (i3_0 - 3) * N4,
                      i2_0 - 3, jj, &tbar[b]);
      }
    };
#pragma unroll
    for (int i = 0; i < NCP; ++i) {
      const int t = tid + i * NA;
      cp_dst[i] = -1;
      cp_src[i] = -1;
      if (t < ELEMS) {
        const int v = t & 1, rc = t >> 1;
        const int cc = rc % C::H3, rr = rc / C::H3;
        const int i2 = i2_0 - 3 + rr, i3 = i3_0 - 3 + cc;
        const bool ok = (unsigned)i2 < (unsigned)n2 && (unsigned)i3 < (unsigned)n3;
        cp_dst[i] = rr * ROW + cc * N4 + 4 * v;
        cp_src[i] = ok ? (i2 * n3 + i3) * N4 + 4 * v : -1;
      }
    }
    auto issue = [&](int jj, int buf) {
#pragma unroll
      for (int src_i = 0; src_i < NIN; ++src_i) {
        const float* g = (CG && src_i == 0) ? a.r : a.pold;
        float* dst = s_in + (buf * 2 + src_i) * C::TILE;
        const float* gp = g + (int64_t)jj * plane;
#pragma unroll
        for (int i = 0; i < NCP; ++i) {
          if (cp_dst[i] < 0) continue;
          const bool ok = cp_src[i] >= 0;
          cp_async16(dst + cp_dst[i], ok ? gp + cp_src[i] : g, ok);
        }
      }
    };
#pragma unroll 1
    for (int s = 0; s < STAGES - 1; ++s) {
      if constexpr (TMA) {
        if (warp == TMA_WARP && jb + s < je) issue_tma(jb + s, s);
      } else {
        if (jb + s < je) issue(jb + s, s);
        cp_async_commit();
      }
    }
    static_assert(H2 == 22 && T2 == 16 && C::NBQ == 8 && NA == 256, "stage-A slot map");
    int slot_ar = -1, slot_bq = 0;
    if (tid < 128) {
      slot_ar = 3 + (tid & 15);
      slot_bq = tid >> 4;
    } else if (tid < 176) {
      const int h = tid - 128;  // 0 .. 47
      const int hr = h % 6;
      slot_ar = hr < 3 ? hr : hr + T2;
      slot_bq = h / 6;
    }
    // G3 and lambda L3 coefficients of this slot's two columns, the same for every plane.
    float gc3[T3P][7], lc3[T3P][5];
#pragma unroll
    for (int t = 0; t < T3P; ++t) {
      const int col = (slot_ar >= 0 ? slot_bq * T3P : 0) + t;
#pragma unroll
      for (int e = 0; e < 7; ++e) gc3[t][e] = g3s[col * 8 + e];
#pragma unroll
      for (int e = 0; e < 5; ++e) lc3[t][e] = l3s[col * 8 + e];
    }
#pragma unroll 1
    for (int it = 0; it < nplanes; ++it) {
      const int j = jb + it;
      const int par = it & 1;
      const int buf = it % STAGES;
      if constexpr (TMA) {
        // Plane j's rows have landed once its stage barrier completes.  Every
        // A thread passed the barrier after the p pass of plane j - 1, so its
        // stage (the one refilled next) is free.  A wait that gives up marks
        // the CTA and the kernel runs on without waiting (garbage out, flag set).
        if (!*s_abort && !mbar_wait_parity(&tbar[buf], (unsigned)((it / STAGES) & 1))) {
          *s_abort = 1;
          if (a.timeout_flag) atomicExch(a.timeout_flag, 1);
        }
        const int jn = j + STAGES - 1;
        if (warp == TMA_WARP && jn < je) issue_tma(jn, (it + STAGES - 1) % STAGES);
      } else {
        cp_async_wait<STAGES - 2>();
        bar_sync(BAR_A, NA);  // plane j landed for every A thread; all are done with plane j - 1's stage
        const int jn = j + STAGES - 1;
        if (jn < je) issue(jn, (it + STAGES - 1) % STAGES);
        cp_async_commit();
      }
      if (it >= 2) bar_sync(BAR_EMPTY + par, NT);  // B is done with the buffers of plane j - 2
      float* pdst = sm + C::OFF_P + par * C::TILE;
      {
        const float4* pp = reinterpret_cast<const float4*>(s_in + (buf * 2 + (CG ? 1 : 0)) * C::TILE);
        float4* out = reinterpret_cast<float4*>(pdst);
        if constexpr (TMA) {
          // Dense stage rows (H3 * N4 / 4 vectors) into padded P rows (ROW / 4).
          constexpr int DR = C::H3 * N4 / 4, PR = ROW / 4;
          const float4* rr = reinterpret_cast<const float4*>(s_in + (buf * 2 + 0) * C::TILE);
          for (int t = tid; t < H2 * DR; t += NA) {
            const int o = (t / DR) * PR + t % DR;
            if constexpr (CG) {
              const float4 x = rr[t], y = pp[t];
              out[o] = make_float4(fmaf(beta, y.x, x.x), fmaf(beta, y.y, x.y), fmaf(beta, y.z, x.z),
                                   fmaf(beta, y.w, x.w));
            } else {
              out[o] = pp[t];
            }
          }
        } else if constexpr (CG) {
          const float4* rr = reinterpret_cast<const float4*>(s_in + (buf * 2 + 0) * C::TILE);
          for (int t = tid; t < C::TILE / 4; t += NA) {
            const float4 x = rr[t], y = pp[t];
            out[t] = make_float4(fmaf(beta, y.x, x.x), fmaf(beta, y.y, x.y), fmaf(beta, y.z, x.z),
                                 fmaf(beta, y.w, x.w));
          }
        } else {
          for (int t = tid; t < C::TILE / 4; t += NA) out[t] = pp[t];
        }
      }
      bar_sync(BAR_A, NA);
      const float* src = pdst;
      float* s_s1 = sm + C::OFF_S1 + par * C::S1N;
      float* s_sl = sm + C::OFF_SL + par * C::SLN;
      // ---- stage A (one halo row, two columns, eight lanes per thread) ----
      // Slots of core rows (G3, G4 and lambda (L3 + L4)) fill warps 0-3, one
      // per scheduler; the lighter halo-row slots (G3, G4 only) fill warp 4
      // and half of warp 5.  No warp mixes the two kinds, and the fewest
      // warps issue the light work (issue slots, not lanes, are the limit).
      if (slot_ar >= 0) {
        const int ar = slot_ar;
        const int bq = slot_bq;
        const int b0 = bq * T3P;
        constexpr int NV = 4;
        float2 v[T3P + 6][NV];
        const float* rowp = src + ar * ROW + b0 * N4;
#pragma unroll
        for (int t = 0; t < T3P + 6; ++t) {
          const float4 lo = reinterpret_cast<const float4*>(rowp + t * N4)[0];
          const float4 hi = reinterpret_cast<const float4*>(rowp + t * N4)[1];
          v[t][0] = make_float2(lo.x, lo.y); v[t][1] = make_float2(lo.z, lo.w);
          v[t][2] = make_float2(hi.x, hi.y); v[t][3] = make_float2(hi.z, hi.w);
        }
        float2 u[T3P][NV];
#pragma unroll
        for (int t = 0; t < T3P; ++t) {
          const float* gc = gc3[t];
#pragma unroll
          for (int m = 0; m < NV; ++m) {
            float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 7; ++e) s2 = ffma2(bc2(gc[e]), v[t + e][m], s2);
            u[t][m] = s2;
          }
        }
        float2 o[T3P][NV];
        {
          float2 od[T3P][NV + 1];
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            od[t][0] = make_float2(0.f, u[t][0].x);
#pragma unroll
            for (int k = 1; k < NV; ++k) od[t][k] = make_float2(u[t][k - 1].y, u[t][k].x);
            od[t][NV] = make_float2(u[t][NV - 1].y, 0.f);
#pragma unroll
            for (int m = 0; m < NV; ++m) o[t][m] = make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int mm = 0; mm < NV / 2; ++mm) {
#pragma unroll
            for (int e = 0; e < 7; ++e) {
              const int d = e - 3;
              const float4 c4 = make_float4(a.g4c[e * N4 + 4 * mm], a.g4c[e * N4 + 4 * mm + 1],
                                            a.g4c[e * N4 + 4 * mm + 2], a.g4c[e * N4 + 4 * mm + 3]);
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const int m = 2 * mm + hh;
                const float2 cf = hh ? make_float2(c4.z, c4.w) : make_float2(c4.x, c4.y);
#pragma unroll
                for (int t = 0; t < T3P; ++t) {
                  if ((d & 1) == 0) {
                    const int pi = m + d / 2;
                    if (pi >= 0 && pi < NV) o[t][m] = ffma2(cf, u[t][pi], o[t][m]);
                  } else {
                    const int pi = m + (d + 1) / 2;
                    if (pi >= 0 && pi <= NV) o[t][m] = ffma2(cf, od[t][pi], o[t][m]);
                  }
                }
              }
            }
          }
        }
#pragma unroll
        for (int t = 0; t < T3P; ++t) {
          float* dst = s_s1 + ar * ROW1 + (b0 + t) * N4;
          reinterpret_cast<float4*>(dst)[0] = make_float4(o[t][0].x, o[t][0].y, o[t][1].x, o[t][1].y);
          reinterpret_cast<float4*>(dst)[1] = make_float4(o[t][2].x, o[t][2].y, o[t][3].x, o[t][3].y);
        }
        if (ar >= 3 && ar < 3 + T2) {
          float2 lin[T3P][NV];
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            const float* lc = lc3[t];
#pragma unroll
            for (int m = 0; m < NV; ++m) {
              float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
              for (int e = 0; e < 5; ++e) s2 = ffma2(bc2(lc[e]), v[t + 1 + e][m], s2);
              lin[t][m] = s2;
            }
          }
          float2 od[T3P][NV + 1];
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            od[t][0] = make_float2(0.f, v[t + 3][0].x);
#pragma unroll
            for (int k = 1; k < NV; ++k) od[t][k] = make_float2(v[t + 3][k - 1].y, v[t + 3][k].x);
            od[t][NV] = make_float2(v[t + 3][NV - 1].y, 0.f);
          }
#pragma unroll
          for (int mm = 0; mm < NV / 2; ++mm) {
#pragma unroll
            for (int e = 0; e < 5; ++e) {
              const int d = e - 2;
              const float4 c4 = make_float4(a.l4c[e * N4 + 4 * mm], a.l4c[e * N4 + 4 * mm + 1],
                                            a.l4c[e * N4 + 4 * mm + 2], a.l4c[e * N4 + 4 * mm + 3]);
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const int m = 2 * mm + hh;
                const float2 cf = hh ? make_float2(c4.z, c4.w) : make_float2(c4.x, c4.y);
#pragma unroll
                for (int t = 0; t < T3P; ++t) {
                  if ((d & 1) == 0) {
                    const int pi = m + d / 2;
                    if (pi >= 0 && pi < NV) lin[t][m] = ffma2(cf, v[t + 3][pi], lin[t][m]);
                  } else {
                    const int pi = m + (d + 1) / 2;
                    if (pi >= 0 && pi <= NV) lin[t][m] = ffma2(cf, od[t][pi], lin[t][m]);
                  }
                }
              }
            }
          }
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            float* dst = s_sl + (ar - 3) * ROW1 + (b0 + t) * N4;
            reinterpret_cast<float4*>(dst)[0] = make_float4(lin[t][0].x, lin[t][0].y, lin[t][1].x, lin[t][1].y);
            reinterpret_cast<float4*>(dst)[1] = make_float4(lin[t][2].x, lin[t][2].y, lin[t][3].x, lin[t][3].y);
          }
        }
      }
      __threadfence_block();
      bar_arrive(BAR_FULL + par, NT);  // plane j's P, S1 and SL tiles are ready for B
    }
    if constexpr (TMA) {
      // After a give-up, wait (bounded) for the last copy into each stage so
      // that no transfer into shared memory outlives the CTA.
      if (*s_abort && warp == TMA_WARP && (tid & 31) == 0) {
        // Plane k went to stage k % STAGES in phase (k / STAGES) & 1.
        for (int k = max(0, n_issued - STAGES); k < n_issued; ++k)
          (void)mbar_wait_parity(&tbar[k % STAGES], (unsigned)((k / STAGES) & 1));
      }
    } else {
      cp_async_wait<0>();
    }
    for (int it = max(0, nplanes - 2); it < nplanes; ++it) bar_sync(BAR_EMPTY + (it & 1), NT);
  } else {
    // ======================= B: columns, ring, outputs =======================
    // Thread = two adjacent core rows x four consecutive mode-4 lanes of one
    // column: every shared-memory read and global store is 16 bytes wide and
    // every tap is a packed pair FMA across lanes.  A warp covers all 16
    // columns of one row pair (512 contiguous bytes per row).
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_B));
    static_assert(NB == 2 * T3 * (T2 / 2), "B mapping: 2 lane quads x T3 columns x T2/2 row pairs");
    const int tb = tid - NA;
    const int lq = tb & 1;
    const int bcol = (tb >> 1) % T3;
    const int a0 = 2 * (tb / (2 * T3));
    const bool col_ok = (i3_0 + bcol) < n3;
    const int64_t out_base = ((int64_t)(i2_0 + a0) * n3 + i3_0 + bcol) * N4 + 4 * lq;
    const int64_t row_step = (int64_t)n3 * N4;
    const bool ok0 = col_ok && (i2_0 + a0) < n2;
    const bool ok1 = col_ok && (i2_0 + a0 + 1) < n2;

    // Ring of accumulators along mode 1: [row][lane pair][slot].
    float2 acc[2][2][7];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 7; ++e) acc[k][h][e] = make_float2(0.f, 0.f);
    float2 w2[2][2], lin2[2][2], pc2[2][2];
    float g1r[7], l1r[5];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) w2[k][h] = lin2[k][h] = pc2[k][h] = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 7; ++e) g1r[e] = 0.f;
#pragma unroll
    for (int e = 0; e < 5; ++e) l1r[e] = 0.f;
    const int c_off = bcol * N4 + 4 * lq;
    float2 g2c[7], l2c[5];  // (row a0, row a0 + 1) coefficient pairs, the same for every plane
#pragma unroll
    for (int e = 0; e < 7; ++e) g2c[e] = *reinterpret_cast<const float2*>(g2s + e * T2 + a0);
#pragma unroll
    for (int e = 0; e < 5; ++e) l2c[e] = *reinterpret_cast<const float2*>(l2s + e * T2 + a0);

#pragma unroll 1
    for (int j = jb; j < c1 + kGramHalf; ++j) {
      const int it = j - jb;
      const bool have = j < je;
      const int par = it & 1;
      if (have) {
        bar_sync(BAR_FULL + par, NT);
        const float* src = sm + C::OFF_P + par * C::TILE;
        const float* s_s1 = sm + C::OFF_S1 + par * C::S1N;
        const float* s_sl = sm + C::OFF_SL + par * C::SLN;
        // S1 rows a0 .. a0 + 7 (G2 taps of both rows), P rows a0 + 1 .. a0 + 6
        // of the core column (lambda L2 taps and centres), SL rows a0, a0 + 1.
        float4 s1v[8], s0v[6], slv[2];
#pragma unroll
        for (int r = 0; r < 8; ++r) s1v[r] = *reinterpret_cast<const float4*>(s_s1 + (a0 + r) * ROW1 + c_off);
#pragma unroll
        for (int r = 0; r < 6; ++r)
          s0v[r] = *reinterpret_cast<const float4*>(src + (a0 + 1 + r) * ROW + 3 * N4 + c_off);
#pragma unroll
        for (int r = 0; r < 2; ++r) slv[r] = *reinterpret_cast<const float4*>(s_sl + (a0 + r) * ROW1 + c_off);
        __threadfence_block();
        bar_arrive(BAR_EMPTY + par, NT);  // everything B reads of plane j is in registers
        if constexpr (CG) {
#pragma unroll
          for (int e = 0; e < 7; ++e) g1r[e] = __ldg(a.g[0] + (int64_t)j * 7 + e);
#pragma unroll
          for (int e = 0; e < 5; ++e) l1r[e] = __ldg(a.l[0] + (int64_t)j * 5 + e);
        } else {
          const float4* cr = reinterpret_cast<const float4*>(s_g1l1 + (j - jb) * 16);
          const float4 c0v = cr[0], c1v = cr[1], c2v = cr[2];
          g1r[0] = c0v.x; g1r[1] = c0v.y; g1r[2] = c0v.z; g1r[3] = c0v.w;
          g1r[4] = c1v.x; g1r[5] = c1v.y; g1r[6] = c1v.z;
          l1r[0] = c1v.w; l1r[1] = c2v.x; l1r[2] = c2v.y; l1r[3] = c2v.z; l1r[4] = c2v.w;
        }
        const bool own_plane = (j >= c0) && (j < c1);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 7; ++e) {
              const float cf = k ? g2c[e].y : g2c[e].x;
              const float4 v = s1v[k + e];
              w = ffma2(bc2(cf), h ? make_float2(v.z, v.w) : make_float2(v.x, v.y), w);
            }
            float2 lin = h ? make_float2(slv[k].z, slv[k].w) : make_float2(slv[k].x, slv[k].y);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
              const float cf = k ? l2c[e].y : l2c[e].x;
              const float4 v = s0v[k + e];
              lin = ffma2(bc2(cf), h ? make_float2(v.z, v.w) : make_float2(v.x, v.y), lin);
            }
            const float4 pv = s0v[k + 2];
            w2[k][h] = w;
            lin2[k][h] = lin;
            pc2[k][h] = h ? make_float2(pv.z, pv.w) : make_float2(pv.x, pv.y);
          }
          if constexpr (CG || PDOT) {
            const float4 pc4 = make_float4(pc2[k][0].x, pc2[k][0].y, pc2[k][1].x, pc2[k][1].y);
            float* ring = s_ring + (j & 3) * C::CORE;
            reinterpret_cast<float4*>(ring)[k * NB + tb] = pc4;
            if constexpr (CG) {
              if (own_plane && (k ? ok1 : ok0))
                *reinterpret_cast<float4*>(a.pnew + (int64_t)j * plane + out_base + k * row_step) = pc4;
            }
          }
        }
      }
      const int c = j - kGramHalf;
      auto step = [&](auto tag) {
        constexpr int S = decltype(tag)::value;
        if (have) {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
              for (int d = -3; d <= 3; ++d)
                acc[k][h][(S + d + 7) % 7] = ffma2(bc2(g1r[3 + d]), w2[k][h], acc[k][h][(S + d + 7) % 7]);
#pragma unroll
              for (int d = -2; d <= 2; ++d)
                acc[k][h][(S + d + 7) % 7] = ffma2(bc2(l1r[2 + d]), pc2[k][h], acc[k][h][(S + d + 7) % 7]);
              acc[k][h][S].x += lin2[k][h].x;
              acc[k][h][S].y += lin2[k][h].y;
            }
          }
        }
        constexpr int E = (S + 4) % 7;
        if (c >= c0) {
          float part = 0.f;
          float* qo = a.q + (int64_t)c * plane + out_base;
          const float4* ring = reinterpret_cast<const float4*>(s_ring + (c & 3) * C::CORE);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            if (k ? ok1 : ok0) {
              const float4 qv = make_float4(acc[k][0][E].x, acc[k][0][E].y, acc[k][1][E].x, acc[k][1][E].y);
              *reinterpret_cast<float4*>(qo + k * row_step) = qv;
              if constexpr (CG || PDOT) {
                const float4 pv = ring[k * NB + tb];
                part = fmaf(qv.x, pv.x, part);
                part = fmaf(qv.y, pv.y, part);
                part = fmaf(qv.z, pv.z, part);
                part = fmaf(qv.w, pv.w, part);
              }
            }
          }
          dot += (double)part;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int h = 0; h < 2; ++h) acc[k][h][E] = make_float2(0.f, 0.f);
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
  if constexpr (CG) {
    double total;
    if (dev::grid_sum_last_at(dot, a.red, &total, s_red, s_last)) {
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
  } else if constexpr (PDOT) {
    // rho1 = <r, z> of the preconditioned CG (r the input, z = M^-1 r the output),
    // with the scalar logic of the separate preconditioner dot.
    double total;
    if (dev::grid_sum_last_at(dot, a.red, &total, s_red, s_last)) {
      Scalars* sc = a.scal;
      const bool bad = !isfinite(total) || (!(total > 0.0) && sc->rho_new > 0.0);
      if (bad) sc->breakdown = 1;
      sc->beta = a.pdot == 1 ? 0.0 : total / sc->rho;
      sc->rho = total;
    }
  }
}

constexpr size_t ws_bytes() {
  using C = Cfg<8, 16, 16, 2, NB, 3, true>;
  // reduction scratch for 16 warps, then 3 stage mbarriers, the give-up flag,
  // the reduction's last-block flag and the G1 / L1 table (kMaxPlanes rows)
  return sizeof(float) * (size_t)(C::OFF_RED + 2 * (NT / 32)) + 4 * sizeof(uint64_t) +
         sizeof(float) * 16 * kMaxPlanes;
}

}  // namespace ws

template <int N4, int T2, int T3, int T3P, int NT, int STAGES, bool CG>
tca_status launch_fused(tca_plan_s* p, const FusedArgs& base, cudaStream_t s) {
  using C = Cfg<N4, T2, T3, T3P, NT, STAGES, CG>;
  static_assert(C::BYTES <= 227 * 1024, "shared memory budget");
  auto kfn = fused_normal_kernel<N4, T2, T3, T3P, NT, STAGES, CG>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return TCA_ERR_CUDA;
    }
    attr_done = true;
  }
  FusedArgs a = base;
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const int tiles2 = (n2 + T2 - 1) / T2, tiles3 = (n3 + T3 - 1) / T3;
  const int tiles = tiles2 * tiles3;
  // Chunk count along mode 1: balance whole waves (one CTA per SM) against the
  // +-3 plane halo each chunk reloads.
  int best_nc = 1;
  double best_cost = 1e30;
  for (int nc = 1; nc <= n1; ++nc) {
    const int len = (n1 + nc - 1) / nc;
    if ((int64_t)tiles * nc > p->red.max_blocks) break;
    const int64_t waves = ((int64_t)tiles * nc + p->num_sms - 1) / p->num_sms;
    const double cost = (double)waves * (len + 2 * kGramHalf);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best_nc = nc;
    }
  }
  // An autotuned chunk count (tca_autotune) overrides the wave model.
  if (p->fused_nchunks > 0 && (int64_t)tiles * p->fused_nchunks <= p->red.max_blocks)
    best_nc = std::min(p->fused_nchunks, n1);
  p->fused_model_nchunks = best_nc;
  a.chunk = (n1 + best_nc - 1) / best_nc;
  a.nchunks = (n1 + a.chunk - 1) / a.chunk;
  a.tiles3 = tiles3;
  const int grid = tiles * a.nchunks;
  if (grid > p->red.max_blocks) return TCA_ERR_UNSUPPORTED;
  kfn<<<grid, NT, C::BYTES, s>>>(a);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template <bool CG, bool PDOT>
tca_status launch_ws(tca_plan_s* p, const FusedArgs& base, cudaStream_t s) {
  constexpr size_t bytes = ws::ws_bytes();
  static_assert(bytes <= 227 * 1024, "shared memory budget");
  static_assert(!(CG && PDOT), "the preconditioner dot belongs to the plain sweep");
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(ws::fused_ws_kernel<CG, false, PDOT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ws::fused_ws_kernel<CG, true, PDOT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bytes);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return TCA_ERR_CUDA;
    }
    attr_done = true;
  }
  FusedArgs a = base;
  // Halo tiles by TMA when both maps encode (16-byte aligned tensors); else cp.async.
  bool tma = true;
  {
    // Modes 3 and 4 merged into one contiguous row of n3 * 8 floats: a halo
    // row is one 704-byte run of the box, so a plane's tile is 22 row
    // requests (a 32-byte innermost box dimension would take 484).
    const uint64_t dims[3] = {(uint64_t)a.n3 * 8, (uint64_t)a.n2, (uint64_t)a.n1};
    const uint64_t strides[2] = {(uint64_t)a.n3 * 8 * sizeof(float), (uint64_t)a.n2 * a.n3 * 8 * sizeof(float)};
    // One box per tensor and plane; boxes wider than the tensor are left to cp.async.
    const uint32_t box[3] = {22 * 8, 22, 1};
    tma = a.n2 >= 22 && a.n3 >= 22 && encode_tmap_f32(&a.tm_p, a.pold, 3, dims, strides, box);
    if (tma && CG) tma = encode_tmap_f32(&a.tm_r, a.r, 3, dims, strides, box);
  }
  a.timeout_flag = wait_timeout_flag();
  auto kfn = tma ? ws::fused_ws_kernel<CG, true, PDOT> : ws::fused_ws_kernel<CG, false, PDOT>;
  const int n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const int tiles2 = (n2 + 15) / 16, tiles3 = (n3 + 15) / 16;
  const int tiles = tiles2 * tiles3;
  int best_nc = 1;
  double best_cost = 1e30;
  for (int nc = 1; nc <= n1; ++nc) {
    const int len = (n1 + nc - 1) / nc;
    if ((int64_t)tiles * nc > p->red.max_blocks) break;
    if (len + 2 * kGramHalf > ws::kMaxPlanes) continue;
    const int64_t waves = ((int64_t)tiles * nc + p->num_sms - 1) / p->num_sms;
    const double cost = (double)waves * (len + 2 * kGramHalf);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best_nc = nc;
    }
  }
  if (p->fused_nchunks > 0 && (int64_t)tiles * p->fused_nchunks <= p->red.max_blocks &&
      (n1 + p->fused_nchunks - 1) / p->fused_nchunks + 2 * kGramHalf <= ws::kMaxPlanes)
    best_nc = std::min(p->fused_nchunks, n1);
  p->fused_model_nchunks = best_nc;
  a.chunk = (n1 + best_nc - 1) / best_nc;
  if (a.chunk + 2 * kGramHalf > ws::kMaxPlanes) return TCA_ERR_UNSUPPORTED;
  a.nchunks = (n1 + a.chunk - 1) / a.chunk;
  a.tiles3 = tiles3;
  const int grid = tiles * a.nchunks;
  if (grid > p->red.max_blocks) return TCA_ERR_UNSUPPORTED;
  kfn<<<grid, ws::NT, bytes, s>>>(a);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace

tca_status normal_fused_f32(tca_plan_s* p, const float* r, const float* p_old, float* p_new, float* q,
                            bool cg_mode, cudaStream_t s, const FusedBands* bands, const Scalars* stop, int pdot) {
  if (!p->fused_ok) return TCA_ERR_UNSUPPORTED;
  if (pdot && (cg_mode || p->d != 4 || p->n[3] != 8)) return TCA_ERR_UNSUPPORTED;
  FusedArgs a{};
  a.r = r;
  a.pold = p_old;
  a.pnew = p_new;
  a.q = q;
  const int d = p->d;
  int64_t dims[4];
  for (int k = 0; k < 4; ++k) dims[k] = k < d ? p->n[k] : 1;
  for (int k = 0; k < d; ++k) {
    a.g[k] = bands ? bands->g[k] : p->mode[k].gram.band.w32;
    a.l[k] = bands ? bands->l[k] : p->mode[k].lap.w32;
  }
  a.stop = stop;
  a.pdot = pdot;
  for (int k = d; k < 4; ++k) {
    a.g[k] = nullptr;
    a.l[k] = nullptr;
  }
  if (dims[0] > INT32_MAX || dims[1] > INT32_MAX || dims[2] > INT32_MAX) return TCA_ERR_UNSUPPORTED;
  a.n1 = (int)dims[0];
  a.n2 = (int)dims[1];
  a.n3 = (int)dims[2];
  a.scal = p->scal;
  a.red = p->red;
  const int64_t n4 = dims[3];
  if (n4 == 8) {
    const float* g4 = bands ? bands->g4 : p->ws_g4;
    const float* l4 = bands ? bands->l4 : p->ws_l4;
    for (int i4 = 0; i4 < 8; ++i4) {
      for (int e = 0; e < 7; ++e) a.g4c[e * 8 + i4] = g4[i4 * 7 + e];
      for (int e = 0; e < 5; ++e) a.l4c[e * 8 + i4] = l4[i4 * 5 + e];
    }
    if (cg_mode) return launch_ws<true, false>(p, a, s);
    return pdot ? launch_ws<false, true>(p, a, s) : launch_ws<false, false>(p, a, s);
  } else if (n4 == 4) {
    return cg_mode ? launch_fused<4, 16, 32, 4, 256, 3, true>(p, a, s) : launch_fused<4, 16, 32, 4, 256, 3, false>(p, a, s);
  } else if (n4 == 1) {
    return cg_mode ? launch_fused<1, 32, 64, 8, 256, 3, true>(p, a, s) : launch_fused<1, 32, 64, 8, 256, 3, false>(p, a, s);
  }
  return TCA_ERR_UNSUPPORTED;
}

}  // namespace tca
