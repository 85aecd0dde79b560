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
#include <algorithm>
#include <cstdio>

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

template <int N4, int T2, int T3, int T3P, int NT, int STAGES, bool CG>
struct Cfg {
  static constexpr int H2 = T2 + 6, H3 = T3 + 6;
  static constexpr int TILE = H2 * H3 * N4;   // halo tile, floats
  static constexpr int CORE = T2 * T3 * N4;
  static constexpr int S1N = H2 * T3 * N4;
  static constexpr int NIN = CG ? 2 : 1;      // loaded tensors per plane
  static constexpr int RB = NT / (N4 * T3);   // row blocks in stage B
  static constexpr int P = T2 / RB;           // rows per thread in stage B
  static constexpr int PENC = H2 * (T3 / T3P);
  static_assert(NT % (N4 * T3) == 0, "stage-B mapping");
  static_assert(T2 % RB == 0, "stage-B rows");
  static_assert(T3 % T3P == 0, "stage-A pencils");
  // shared memory carve-up (floats)
  static constexpr int OFF_IN = 0;
  static constexpr int OFF_P = OFF_IN + STAGES * NIN * TILE;
  static constexpr int OFF_S1 = OFF_P + (CG ? TILE : 0);
  static constexpr int OFF_SL = OFF_S1 + S1N;
  static constexpr int OFF_RING = OFF_SL + CORE;
  static constexpr int OFF_G2 = OFF_RING + (CG ? 4 * CORE : 0);
  static constexpr int OFF_L2 = OFF_G2 + T2 * 7;
  static constexpr int OFF_G3 = OFF_L2 + T2 * 5;
  static constexpr int OFF_L3 = OFF_G3 + T3 * 7;
  static constexpr int OFF_G4 = OFF_L3 + T3 * 5;
  static constexpr int OFF_L4 = OFF_G4 + N4 * 7;
  static constexpr int OFF_RED = ((OFF_L4 + N4 * 5 + 1) / 2) * 2;  // doubles, 8B aligned
  static constexpr int FLOATS = OFF_RED + 2 * (NT / 32);
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

template <int N4, int T2, int T3, int T3P, int NT, int STAGES, bool CG>
__global__ void __launch_bounds__(NT, 1) fused_normal_kernel(FusedArgs a) {
  using C = Cfg<N4, T2, T3, T3P, NT, STAGES, CG>;
  constexpr int H3 = C::H3, P = C::P;
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;

  if constexpr (CG) {
    if (cg_done(a.scal)) return;
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
  float* s_p = CG ? sm + C::OFF_P : nullptr;
  float* s_s1 = sm + C::OFF_S1;
  float* s_sl = sm + C::OFF_SL;
  float* s_ring = sm + C::OFF_RING;
  float* g2s = sm + C::OFF_G2;
  float* l2s = sm + C::OFF_L2;
  float* g3s = sm + C::OFF_G3;
  float* l3s = sm + C::OFF_L3;
  float* g4s = sm + C::OFF_G4;
  float* l4s = sm + C::OFF_L4;
  double* s_red = reinterpret_cast<double*>(sm + C::OFF_RED);

  // Tile coefficient tables (rows outside the domain are zero).
  for (int t = tid; t < T2 * 7; t += NT) {
    const int r = t / 7, i2 = i2_0 + r;
    g2s[t] = i2 < n2 ? a.g[1][(int64_t)i2 * 7 + t % 7] : 0.f;
  }
  for (int t = tid; t < T2 * 5; t += NT) {
    const int r = t / 5, i2 = i2_0 + r;
    l2s[t] = i2 < n2 ? a.l[1][(int64_t)i2 * 5 + t % 5] : 0.f;
  }
  for (int t = tid; t < T3 * 7; t += NT) {
    const int r = t / 7, i3 = i3_0 + r;
    g3s[t] = i3 < n3 ? a.g[2][(int64_t)i3 * 7 + t % 7] : 0.f;
  }
  for (int t = tid; t < T3 * 5; t += NT) {
    const int r = t / 5, i3 = i3_0 + r;
    l3s[t] = i3 < n3 ? a.l[2][(int64_t)i3 * 5 + t % 5] : 0.f;
  }
  if constexpr (N4 > 1) {
    for (int t = tid; t < N4 * 7; t += NT) g4s[t] = a.g[3][t];
    for (int t = tid; t < N4 * 5; t += NT) l4s[t] = a.l[3][t];
  }

  const int64_t plane = (int64_t)n2 * n3 * N4;

  // Issue the asynchronous copies of plane jj (halo tile) into stage buffer buf.
  auto issue = [&](int jj, int buf) {
#pragma unroll 1
    for (int src_i = 0; src_i < C::NIN; ++src_i) {
      const float* g = (CG && src_i == 0) ? a.r : a.pold;
      float* dst = s_in + (buf * C::NIN + src_i) * C::TILE;
      const float* gp = g + (int64_t)jj * plane;
      if constexpr (N4 % 4 == 0) {
        constexpr int V = N4 / 4;  // float4 per (row, col)
        for (int t = tid; t < C::H2 * H3 * V; t += NT) {
          const int v = t % V, rc = t / V;
          const int cc = rc % H3, rr = rc / H3;
          const int i2 = i2_0 - 3 + rr, i3 = i3_0 - 3 + cc;
          const bool ok = (unsigned)i2 < (unsigned)n2 && (unsigned)i3 < (unsigned)n3;
          const float* src = ok ? gp + ((int64_t)i2 * n3 + i3) * N4 + 4 * v : g;
          cp_async16(dst + (rr * H3 + cc) * N4 + 4 * v, src, ok);
        }
      } else {
        for (int t = tid; t < C::H2 * H3 * N4; t += NT) {
          const int i4 = t % N4, rc = t / N4;
          const int cc = rc % H3, rr = rc / H3;
          const int i2 = i2_0 - 3 + rr, i3 = i3_0 - 3 + cc;
          const bool ok = (unsigned)i2 < (unsigned)n2 && (unsigned)i3 < (unsigned)n3;
          const float* src = ok ? gp + ((int64_t)i2 * n3 + i3) * N4 + i4 : g;
          cp_async4(dst + t, src, ok);
        }
      }
    }
  };

  // Stage-B thread mapping.
  const int i4b = tid % N4;
  const int bcol = (tid / N4) % T3;
  const int a0 = (tid / (N4 * T3)) * P;
  const bool col_ok = (i3_0 + bcol) < n3;

  float acc[P][7];
#pragma unroll
  for (int k = 0; k < P; ++k)
#pragma unroll
    for (int e = 0; e < 7; ++e) acc[k][e] = 0.f;
  double dot = 0.0;

  // Prologue: planes jb .. jb+STAGES-2.
#pragma unroll 1
  for (int s = 0; s < STAGES - 1; ++s) {
    if (jb + s < je) issue(jb + s, s);
    cp_async_commit();
  }
  __syncthreads();  // coefficient tables visible

#pragma unroll 1
  for (int j = jb; j < c1 + kGramHalf; ++j) {
    const int it = j - jb;
    const bool have = j < je;
    {
      const int jn = j + STAGES - 1;
      if (jn < je) issue(jn, (it + STAGES - 1) % STAGES);
      cp_async_commit();
    }
    if (have) {
      cp_async_wait<STAGES - 1>();
      __syncthreads();
      const int buf = it % STAGES;
      const float* src;
      if constexpr (CG) {
        const float4* rr = reinterpret_cast<const float4*>(s_in + (buf * 2 + 0) * C::TILE);
        const float4* pp = reinterpret_cast<const float4*>(s_in + (buf * 2 + 1) * C::TILE);
        float4* out = reinterpret_cast<float4*>(s_p);
        static_assert(C::TILE % 4 == 0, "tile must hold whole float4");
        for (int t = tid; t < C::TILE / 4; t += NT) {
          const float4 x = rr[t], y = pp[t];
          out[t] = make_float4(fmaf(beta, y.x, x.x), fmaf(beta, y.y, x.y), fmaf(beta, y.z, x.z),
                               fmaf(beta, y.w, x.w));
        }
        __syncthreads();
        src = s_p;
      } else {
        src = s_in + buf * C::TILE;
      }

      // ---- stage A: G_3 then G_4 along the rows of the halo tile ----
#pragma unroll 1
      for (int pc = tid; pc < C::PENC; pc += NT) {
        const int ar = pc / (T3 / T3P);
        const int b0 = (pc % (T3 / T3P)) * T3P;
        float v[T3P + 6][N4];
#pragma unroll
        for (int t = 0; t < T3P + 6; ++t) {
          const float* row = src + (ar * H3 + b0 + t) * N4;
          if constexpr (N4 % 4 == 0) {
#pragma unroll
            for (int q4 = 0; q4 < N4 / 4; ++q4) {
              const float4 f = reinterpret_cast<const float4*>(row)[q4];
              v[t][4 * q4 + 0] = f.x; v[t][4 * q4 + 1] = f.y; v[t][4 * q4 + 2] = f.z; v[t][4 * q4 + 3] = f.w;
            }
          } else {
#pragma unroll
            for (int i4 = 0; i4 < N4; ++i4) v[t][i4] = row[i4];
          }
        }
        float u[T3P][N4];
#pragma unroll
        for (int t = 0; t < T3P; ++t) {
          float gc[7];
#pragma unroll
          for (int e = 0; e < 7; ++e) gc[e] = g3s[(b0 + t) * 7 + e];
#pragma unroll
          for (int i4 = 0; i4 < N4; ++i4) {
            float s = 0.f;
#pragma unroll
            for (int e = 0; e < 7; ++e) s = fmaf(gc[e], v[t + e][i4], s);
            u[t][i4] = s;
          }
        }
#pragma unroll
        for (int t = 0; t < T3P; ++t) {
          float o[N4];
          if constexpr (N4 > 1) {
#pragma unroll
            for (int i4 = 0; i4 < N4; ++i4) {
              float s = 0.f;
#pragma unroll
              for (int e = 0; e < 7; ++e) {
                const int c = i4 - 3 + e;
                if (c >= 0 && c < N4) s = fmaf(g4s[i4 * 7 + e], u[t][c], s);
              }
              o[i4] = s;
            }
          } else {
            o[0] = u[t][0];
          }
          float* dst = s_s1 + (ar * T3 + b0 + t) * N4;
#pragma unroll
          for (int i4 = 0; i4 < N4; ++i4) dst[i4] = o[i4];
        }
        if (ar >= 3 && ar < 3 + T2) {
#pragma unroll
          for (int t = 0; t < T3P; ++t) {
            float lc[5];
#pragma unroll
            for (int e = 0; e < 5; ++e) lc[e] = l3s[(b0 + t) * 5 + e];
            float* dst = s_sl + ((ar - 3) * T3 + b0 + t) * N4;
#pragma unroll
            for (int i4 = 0; i4 < N4; ++i4) {
              float s = 0.f;
#pragma unroll
              for (int e = 0; e < 5; ++e) s = fmaf(lc[e], v[t + 1 + e][i4], s);
              if constexpr (N4 > 1) {
#pragma unroll
                for (int e = 0; e < 5; ++e) {
                  const int c = i4 - 2 + e;
                  if (c >= 0 && c < N4) s = fmaf(l4s[i4 * 5 + e], v[t + 3][c], s);
                }
              }
              dst[i4] = s;
            }
          }
        }
      }
      __syncthreads();

      // ---- stage B: G_2 down columns, L_2, scatter along mode 1 ----
      {
        float s1c[P + 6];
#pragma unroll
        for (int k = 0; k < P + 6; ++k) s1c[k] = s_s1[((a0 + k) * T3 + bcol) * N4 + i4b];
        float s0c[P + 4];
#pragma unroll
        for (int k = 0; k < P + 4; ++k) s0c[k] = src[((a0 + 1 + k) * H3 + bcol + 3) * N4 + i4b];
        float g1r[7], l1r[5];
#pragma unroll
        for (int e = 0; e < 7; ++e) g1r[e] = __ldg(a.g[0] + (int64_t)j * 7 + e);
#pragma unroll
        for (int e = 0; e < 5; ++e) l1r[e] = __ldg(a.l[0] + (int64_t)j * 5 + e);
        const bool own_plane = (j >= c0) && (j < c1);
#pragma unroll
        for (int k = 0; k < P; ++k) {
          float w = 0.f;
#pragma unroll
          for (int e = 0; e < 7; ++e) w = fmaf(g2s[(a0 + k) * 7 + e], s1c[k + e], w);
          float lin = s_sl[((a0 + k) * T3 + bcol) * N4 + i4b];
#pragma unroll
          for (int e = 0; e < 5; ++e) lin = fmaf(l2s[(a0 + k) * 5 + e], s0c[k + e], lin);
          const float pcv = s0c[k + 2];
#pragma unroll
          for (int e = 0; e < 7; ++e) acc[k][e] = fmaf(g1r[e], w, acc[k][e]);
#pragma unroll
          for (int e = 0; e < 5; ++e) acc[k][e + 1] = fmaf(l1r[e], pcv, acc[k][e + 1]);
          acc[k][3] += lin;
          if constexpr (CG) {
            s_ring[(j & 3) * C::CORE + ((a0 + k) * T3 + bcol) * N4 + i4b] = pcv;
            const int i2 = i2_0 + a0 + k;
            if (own_plane && col_ok && i2 < n2)
              a.pnew[(int64_t)j * plane + ((int64_t)i2 * n3 + i3_0 + bcol) * N4 + i4b] = pcv;
          }
        }
      }
      __syncthreads();
    }
    // ---- emit plane j-3 and rotate the accumulator ring ----
    const int c = j - kGramHalf;
    if (c >= c0) {
      float part = 0.f;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int i2 = i2_0 + a0 + k;
        if (col_ok && i2 < n2) {
          const float qv = acc[k][0];
          a.q[(int64_t)c * plane + ((int64_t)i2 * n3 + i3_0 + bcol) * N4 + i4b] = qv;
          if constexpr (CG) part = fmaf(qv, s_ring[(c & 3) * C::CORE + ((a0 + k) * T3 + bcol) * N4 + i4b], part);
        }
      }
      dot += (double)part;
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
      for (int e = 0; e < 6; ++e) acc[k][e] = acc[k][e + 1];
      acc[k][6] = 0.f;
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

template <int N4, int T2, int T3, int T3P, int NT, int STAGES, bool CG>
tca_status launch_fused(tca_plan_s* p, const FusedArgs& base, cudaStream_t s) {
  using C = Cfg<N4, T2, T3, T3P, NT, STAGES, CG>;
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
  a.chunk = (n1 + best_nc - 1) / best_nc;
  a.nchunks = (n1 + a.chunk - 1) / a.chunk;
  a.tiles3 = tiles3;
  const int grid = tiles * a.nchunks;
  if (grid > p->red.max_blocks) return TCA_ERR_UNSUPPORTED;
  kfn<<<grid, NT, C::BYTES, s>>>(a);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace

tca_status normal_fused_f32(tca_plan_s* p, const float* r, const float* p_old, float* p_new, float* q,
                            bool cg_mode, cudaStream_t s) {
  if (!p->fused_ok) return TCA_ERR_UNSUPPORTED;
  FusedArgs a{};
  a.r = r;
  a.pold = p_old;
  a.pnew = p_new;
  a.q = q;
  const int d = p->d;
  int64_t dims[4];
  for (int k = 0; k < 4; ++k) dims[k] = k < d ? p->n[k] : 1;
  for (int k = 0; k < d; ++k) {
    a.g[k] = p->mode[k].gram.band.w32;
    a.l[k] = p->mode[k].lap.w32;
  }
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
    return cg_mode ? launch_fused<8, 16, 16, 2, 256, 3, true>(p, a, s) : launch_fused<8, 16, 16, 2, 256, 3, false>(p, a, s);
  } else if (n4 == 4) {
    return cg_mode ? launch_fused<4, 16, 32, 4, 256, 3, true>(p, a, s) : launch_fused<4, 16, 32, 4, 256, 3, false>(p, a, s);
  } else if (n4 == 1) {
    return cg_mode ? launch_fused<1, 32, 64, 8, 256, 3, true>(p, a, s) : launch_fused<1, 32, 64, 8, 256, 3, false>(p, a, s);
  }
  return TCA_ERR_UNSUPPORTED;
}

}  // namespace tca
