// Learned initial guess / preconditioner: a 4-layer 3D convolutional network
// over modes 1..3 of a tensor (mode 4 is a batch index), trained on the GPU by
// the kernels in this file (forward, backpropagation, Adam).
//
//   h1 = relu(conv(u, W1) + b1)      1 -> 32 channels
//   h2 = relu(conv(h1, W2) + b2)     32 -> 32
//   h3 = relu(conv(h2, W3) + b3)     32 -> 32
//   y  = conv(h3, W4) + b4           32 -> 1
//
// conv is the 'same' 3x3x3 cross-correlation with zero padding; tap
// t = 9a + 3b + e (a, b, e in 0..2) reads the neighbour at offset
// (a-1, b-1, e-1) in modes 1..3.  Weights and the activations h1..h3 (and
// their gradients) are stored in bfloat16; every sum accumulates in FP32.
//
// Layouts.  A tensor of shape (D, H, W, B) is a C-order array, voxel
// v = ((z H + y) W + x) B + n.  A 32-channel activation is [V][32] bfloat16
// (64 bytes per voxel, channels fastest).  The master parameters are FP32 in
// the packed order of the public API: per layer W[c_out][c_in][3][3][3], b.
// After every update a preparation kernel writes the bfloat16-rounded copies
// in the layouts the convolution kernels read (forward and flipped/transposed
// for the input gradients: the adjoint of a correlation with W[o][c][t] is
// the correlation with W[o][c][26 - t] with the channel roles swapped).
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <type_traits>
#include <vector>

#include "tca_internal.cuh"
#include "../../include/tca_net.h"

namespace tca {
namespace net {

constexpr int C = 32;
constexpr int T = 27;
// Packed parameter offsets (floats).
constexpr int64_t kW1 = 0, kB1 = kW1 + C * T;
constexpr int64_t kW2 = kB1 + C, kB2 = kW2 + C * C * T;
constexpr int64_t kW3 = kB2 + C, kB3 = kW3 + C * C * T;
constexpr int64_t kW4 = kB3 + C, kB4 = kW4 + C * T;
constexpr int64_t kParams = kB4 + 1;

// Derived (bfloat16-rounded) weight layouts, FP32 or bf16 as noted.
struct Derived {
  __align__(16) float w1f[T * C];  // [t][co]                      layer 1 forward
  __align__(16) float w4b[T * C];  // [t][ci] = W4[0][ci][26 - t]  layer 4 input gradient (1 -> 32)
  __align__(16) float w4f[T * C];  // [t][ci]                      layer 4 forward (32 -> 1)
  __align__(16) float b1[C];
  __align__(16) float b2[C];
  __align__(16) float b3[C];
  __align__(16) float b4[4];
  __align__(16) __nv_bfloat16 w2f[T * C * C];  // [t][i][o] = W2[o][i][t]
  __align__(16) __nv_bfloat16 w3f[T * C * C];
  __align__(16) __nv_bfloat16 w2b[T * C * C];  // [t][o][i] = W2[o][i][26 - t]: input gradient of layer 2
  __align__(16) __nv_bfloat16 w3b[T * C * C];
  // The same four 32 -> 32 weight sets in the tensor-core operand layout
  // (canonical K-major, no swizzle): tap t, output channel o (N row),
  // input channel i (K) at byte t 2048 + (i / 8) 512 + o 16 + (i % 8) 2.
  __align__(16) __nv_bfloat16 w2f_tc[T * C * C];
  __align__(16) __nv_bfloat16 w3f_tc[T * C * C];
  __align__(16) __nv_bfloat16 w2b_tc[T * C * C];
  __align__(16) __nv_bfloat16 w3b_tc[T * C * C];
  // Layer 4 (32 -> 1) in the same layout with N padded to 16 rows (row 0 is
  // the output channel, rows 1..15 zero): byte t 1024 + (i / 8) 256 + o 16 + (i % 8) 2.
  __align__(16) __nv_bfloat16 w4f_tc[T * 16 * C];
};

// Address of a member of the device-resident Derived block.
#define DW(n, field) \
  (reinterpret_cast<const std::remove_reference_t<decltype(Derived::field[0])>*>( \
      reinterpret_cast<const char*>((n)->dw) + offsetof(Derived, field)))

struct Dims {
  int D, H, W, B;
  int64_t V;
};

__device__ __forceinline__ int64_t tap_offset(int t, const Dims& d) {
  const int a = t / 9 - 1, b = (t / 3) % 3 - 1, e = t % 3 - 1;
  return (((int64_t)a * d.H + b) * d.W + e) * d.B;
}

// Validity mask of the 27 taps for voxel (z, y, x): bit t set when the
// neighbour lies inside the volume.
__device__ __forceinline__ unsigned tap_mask(int z, int y, int x, const Dims& d) {
  unsigned m = 0;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int zz = z + t / 9 - 1, yy = y + (t / 3) % 3 - 1, xx = x + t % 3 - 1;
    if (zz >= 0 && zz < d.D && yy >= 0 && yy < d.H && xx >= 0 && xx < d.W) m |= 1u << t;
  }
  return m;
}

__device__ __forceinline__ void decode(int64_t v, const Dims& d, int& z, int& y, int& x) {
  int64_t r = v / d.B;
  x = (int)(r % d.W);
  r /= d.W;
  y = (int)(r % d.H);
  z = (int)(r / d.H);
}

__device__ __forceinline__ float bf(const __nv_bfloat16 h) { return __bfloat162float(h); }
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float round_bf(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// Store 32 FP32 values as 32 bfloat16 (64 bytes) at dst.
__device__ __forceinline__ void store32(__nv_bfloat16* dst, const float* acc) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 w;
    w.x = pack2(acc[8 * q + 0], acc[8 * q + 1]);
    w.y = pack2(acc[8 * q + 2], acc[8 * q + 3]);
    w.z = pack2(acc[8 * q + 4], acc[8 * q + 5]);
    w.w = pack2(acc[8 * q + 6], acc[8 * q + 7]);
    d4[q] = w;
  }
}
__device__ __forceinline__ void load32(const __nv_bfloat16* src, float* out) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 w = __ldg(s4 + q);
    out[8 * q + 0] = bf_lo(w.x); out[8 * q + 1] = bf_hi(w.x);
    out[8 * q + 2] = bf_lo(w.y); out[8 * q + 3] = bf_hi(w.y);
    out[8 * q + 4] = bf_lo(w.z); out[8 * q + 5] = bf_hi(w.z);
    out[8 * q + 6] = bf_lo(w.w); out[8 * q + 7] = bf_hi(w.w);
  }
}

constexpr int kThreads = 128;

// ---- 1 -> 32 channels ------------------------------------------------------
// Forward (layer 1): out = relu(sum_t w[t][co] * in[v + off t] * in_scale + b).
// Input gradient of layer 4 (MASK): out = (sum_t w4b[t][ci] g[v + off t]) * (h3 > 0).
// A job is 256 consecutive voxels of one row (z, y) of the volume (the
// flattened (x, n) index, L = W B voxels).  Its nine input rows
// (z + a - 1, y + b - 1) over those voxels and B voxels on each side (the x
// neighbours) are copied into shared memory by cp.async, zeros off the
// volume, one job ahead of the arithmetic (two buffers).  Thread t owns
// voxels (t >> 1) + 64 u (u = 0..3) of the job and the channels
// 16 (t & 1) .. + 15, so that for each u a warp's 16-byte stores cover
// contiguous voxels.  Per channel the taps accumulate in tap order (bias, then
// t = 0 .. 26; each input scaled as it is used), two channels per packed FMA.
constexpr int kRowVox = 256;  // voxels of a row per job

// Shared memory of the 1 -> 32 kernel for a 4th-mode extent B: two buffers of nine rows.
size_t conv1to32_smem(int B) { return sizeof(float) * 2 * 9 * (size_t)(kRowVox + 2 * B); }

__device__ __forceinline__ void cp_async4_zfill(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

template <bool MASK>
__global__ void __launch_bounds__(kThreads) conv1to32_kernel(const float* __restrict__ in,
                                                             const float* __restrict__ scale_dev,
                                                             const float* __restrict__ w, const float* __restrict__ bias,
                                                             const __nv_bfloat16* __restrict__ mask_src,
                                                             __nv_bfloat16* __restrict__ out, Dims d) {
  static_assert(kThreads * 2 == kRowVox, "two threads per voxel column, four voxels each");
  __shared__ __align__(16) float sw[T * C];
  __shared__ float sb[C];
  extern __shared__ float srow[];  // [2][9][kRowVox + 2 B]
  for (int i = threadIdx.x; i < T * C; i += blockDim.x) sw[i] = w[i];
  if (threadIdx.x < C) sb[threadIdx.x] = bias ? bias[threadIdx.x] : 0.f;
  const float inv = scale_dev ? 1.f / *scale_dev : 1.f;
  const int L = d.W * d.B;
  const int SW = kRowVox + 2 * d.B;
  const int chunks = (L + kRowVox - 1) / kRowVox;
  const int64_t jobs = (int64_t)d.D * d.H * chunks;
  const int half = threadIdx.x & 1;
  const int vl = threadIdx.x >> 1;
  // Copies of job `job`'s nine rows into buffer `buf` (one commit group).
  auto stage = [&](int64_t job, int buf) {
    if (job < jobs) {
      const int64_t row = job / chunks;
      const int rb = (int)(job - row * chunks) * kRowVox;
      const int z = (int)(row / d.H), y = (int)(row - (int64_t)z * d.H);
      float* dst = srow + (size_t)buf * 9 * SW;
      for (int ab = 0; ab < 9; ++ab) {
        const int zz = z + ab / 3 - 1, yy = y + ab % 3 - 1;
        const bool rok = zz >= 0 && zz < d.D && yy >= 0 && yy < d.H;
        const float* base = in + (rok ? ((int64_t)zz * d.H + yy) * L : 0);
        for (int k = threadIdx.x; k < SW; k += blockDim.x) {
          const int rs = rb - d.B + k;
          const bool ok = rok && (unsigned)rs < (unsigned)L;
          cp_async4_zfill(dst + ab * SW + k, ok ? base + rs : in, ok);
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int buf = 0;
  stage(blockIdx.x, 0);
  for (int64_t job = blockIdx.x; job < jobs; job += gridDim.x, buf ^= 1) {
    // The other buffer was last read by the previous job (every thread is past it).
    __syncthreads();
    stage(job + gridDim.x, buf ^ 1);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();  // this job's rows (and the weights) are in
    const int64_t row = job / chunks;
    const int rb = (int)(job - row * chunks) * kRowVox;
    float2 acc[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[u][c] = make_float2(sb[16 * half + 2 * c], sb[16 * half + 2 * c + 1]);
#pragma unroll 1
    for (int ab = 0; ab < 9; ++ab) {
      const float* sr = srow + ((size_t)buf * 9 + ab) * SW + vl;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int t = 3 * ab + e;
        float val[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) val[u] = sr[64 * u + e * d.B] * inv;
        const float4* w4 = reinterpret_cast<const float4*>(sw + t * C + 16 * half);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 ww = w4[q];
          const float2 w01 = make_float2(ww.x, ww.y), w23 = make_float2(ww.z, ww.w);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 v2 = make_float2(val[u], val[u]);
            acc[u][2 * q] = __ffma2_rn(w01, v2, acc[u][2 * q]);
            acc[u][2 * q + 1] = __ffma2_rn(w23, v2, acc[u][2 * q + 1]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = rb + vl + 64 * u;
      if (r >= L) continue;
      const int64_t v = row * L + r;
      float a[16];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        a[2 * c] = acc[u][c].x;
        a[2 * c + 1] = acc[u][c].y;
      }
      if constexpr (MASK) {
        const uint4* hs = reinterpret_cast<const uint4*>(mask_src + v * C + 16 * half);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint4 hw = __ldg(hs + q);
          const uint32_t hv[4] = {hw.x, hw.y, hw.z, hw.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (!(bf_lo(hv[k]) > 0.f)) a[8 * q + 2 * k] = 0.f;
            if (!(bf_hi(hv[k]) > 0.f)) a[8 * q + 2 * k + 1] = 0.f;
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) a[c] = fmaxf(a[c], 0.f);
      }
      uint4* dst = reinterpret_cast<uint4*>(out + v * C + 16 * half);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint4 o;
        o.x = pack2(a[8 * q + 0], a[8 * q + 1]);
        o.y = pack2(a[8 * q + 2], a[8 * q + 3]);
        o.z = pack2(a[8 * q + 4], a[8 * q + 5]);
        o.w = pack2(a[8 * q + 6], a[8 * q + 7]);
        dst[q] = o;
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---- 32 -> 1 channel (layer 4 forward) ---------------------------------------
// y = (sum_t sum_ci w4f[t][ci] h3[v + off t][ci] + b4) * out_scale
__global__ void __launch_bounds__(kThreads) conv32to1_kernel(const __nv_bfloat16* __restrict__ h,
                                                             const float* __restrict__ w, const float* __restrict__ bias,
                                                             const float* __restrict__ scale_dev,
                                                             float* __restrict__ out, Dims d) {
  __shared__ float sw[T * C];
  for (int i = threadIdx.x; i < T * C; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const float s = scale_dev ? *scale_dev : 1.f;
  const float b = bias[0];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += (int64_t)gridDim.x * blockDim.x) {
    int z, y, x;
    decode(v, d, z, y, x);
    const unsigned m = tap_mask(z, y, x, d);
    float acc = b;
    for (int t = 0; t < T; ++t) {
      if (!(m >> t & 1u)) continue;
      float hv[C];
      load32(h + (v + tap_offset(t, d)) * C, hv);
      const float* wt = sw + t * C;
#pragma unroll
      for (int c = 0; c < C; ++c) acc = fmaf(wt[c], hv[c], acc);
    }
    out[v] = acc * s;
  }
}

// ---- 32 -> 32 channels (layers 2, 3 and their input gradients) -----------------
// out[v][o] = act(sum_t sum_i w[t][i][o] in[v + off t][i] + b[o]); act = relu
// (forward) or the mask (h > 0) of the layer below (input gradient).
template <bool MASK>
__global__ void __launch_bounds__(kThreads) conv32to32_kernel(const __nv_bfloat16* __restrict__ in,
                                                              const __nv_bfloat16* __restrict__ w,
                                                              const float* __restrict__ bias,
                                                              const __nv_bfloat16* __restrict__ mask_src,
                                                              __nv_bfloat16* __restrict__ out, Dims d) {
  extern __shared__ __align__(16) unsigned char net_smem[];
  uint32_t* sw = reinterpret_cast<uint32_t*>(net_smem);  // [t][i][o/2] bf16 pairs
  for (int i = threadIdx.x; i < T * C * C / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(sw)[i] = reinterpret_cast<const uint4*>(w)[i];
  __shared__ float sb[C];
  if (threadIdx.x < C) sb[threadIdx.x] = bias ? bias[threadIdx.x] : 0.f;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += (int64_t)gridDim.x * blockDim.x) {
    int z, y, x;
    decode(v, d, z, y, x);
    const unsigned m = tap_mask(z, y, x, d);
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = sb[c];
    for (int t = 0; t < T; ++t) {
      if (!(m >> t & 1u)) continue;
      const uint4* src = reinterpret_cast<const uint4*>(in + (v + tap_offset(t, d)) * C);
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const uint4 iw = __ldg(src + q);
        const float xi[8] = {bf_lo(iw.x), bf_hi(iw.x), bf_lo(iw.y), bf_hi(iw.y),
                             bf_lo(iw.z), bf_hi(iw.z), bf_lo(iw.w), bf_hi(iw.w)};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint4* wr = reinterpret_cast<const uint4*>(sw + ((t * C + 8 * q + k) * C) / 2);
#pragma unroll
          for (int o8 = 0; o8 < 4; ++o8) {
            const uint4 ww = wr[o8];
            acc[8 * o8 + 0] = fmaf(bf_lo(ww.x), xi[k], acc[8 * o8 + 0]);
            acc[8 * o8 + 1] = fmaf(bf_hi(ww.x), xi[k], acc[8 * o8 + 1]);
            acc[8 * o8 + 2] = fmaf(bf_lo(ww.y), xi[k], acc[8 * o8 + 2]);
            acc[8 * o8 + 3] = fmaf(bf_hi(ww.y), xi[k], acc[8 * o8 + 3]);
            acc[8 * o8 + 4] = fmaf(bf_lo(ww.z), xi[k], acc[8 * o8 + 4]);
            acc[8 * o8 + 5] = fmaf(bf_hi(ww.z), xi[k], acc[8 * o8 + 5]);
            acc[8 * o8 + 6] = fmaf(bf_lo(ww.w), xi[k], acc[8 * o8 + 6]);
            acc[8 * o8 + 7] = fmaf(bf_hi(ww.w), xi[k], acc[8 * o8 + 7]);
          }
        }
      }
    }
    if constexpr (MASK) {
      float h[C];
      load32(mask_src + v * C, h);
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = h[c] > 0.f ? acc[c] : 0.f;
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fmaxf(acc[c], 0.f);
    }
    store32(out + v * C, acc);
  }
}

// ---- 32 -> 32 channels on the tensor cores -----------------------------------------
// The same convolution as an implicit GEMM on tcgen05 (BF16 operands, FP32
// accumulators in tensor memory).  A tile is 128 consecutive voxels of one
// row (z, y) of the volume (the flattened (x, n) index); per tap (a, b, e)
// the A operand is the input rows (z + a - 1, y + b - 1) shifted by (e - 1) B
// voxels, K = 32 input channels, N = 32 output channels:
//   D[r][o] += sum_i in[v_r + off t][i] W[t][o][i]      (27 taps x 2 MMAs of K = 16)
// A CTA walks columns of tiles along y for fixed (z, segment): input strips
// (128 + 2B voxels x 32 channels of one row (z', y')) stay in a 5-row ring in
// shared memory and each input row is loaded once per column.  Strip layout:
// [channel chunk c (4)][voxel s][16 bytes] - the canonical no-swizzle K-major
// layout (8 voxel rows x 16 bytes per core matrix), so a tap's shift is just
// a start address.  Warp roles, connected by mbarriers (every wait bounded):
//   warps 0-3  producer: cp.async of the three strips of the next row into a
//              free ring slot (zero fill at the volume's faces); completion
//              arrives on the slot's mbarrier (cp.async.mbarrier.arrive);
//   warp 4     MMA: an elected lane issues the 54 MMAs of a tile into one of two
//              TMEM accumulators, commits to the accumulator's mbarrier and,
//              for the row no later tile reads, to that ring slot's mbarrier;
//   warps 5-8  epilogue: TMEM -> registers, bias + ReLU (forward) or the ReLU
//              mask of the layer below (input gradient), bfloat16, 64 bytes per
//              voxel to HBM.
namespace tc {

constexpr int kTile = 128;
constexpr int kRing = 5;
constexpr int kProdWarps = 4, kEpiWarps = 4;
constexpr int kMmaWarp = kProdWarps;
constexpr int kThr = (kProdWarps + 1 + kEpiWarps) * 32;  // 288
constexpr long long kWaitLimit = 1ll << 26;
constexpr int kWBytes = T * C * C * 2;  // 55296: weight tile of a 32 -> 32 layer (N = 32)

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

struct Args {
  const __nv_bfloat16* in;
  __nv_bfloat16* out;         // 32-channel output (N = 32)
  float* out1;                // one-channel output (N = 16, row 0): (acc + bias[0]) * scale
  const float* scale;         // device scalar or null
  const __nv_bfloat16* w;     // tensor-core layout, 27 x 2048 bytes
  const float* bias;          // forward: bias + ReLU; null: mask mode
  const __nv_bfloat16* mask;  // mask mode: out = acc * (mask > 0)
  int D, H, W, B;
  int L, segs, S, ychunk, ychunks;
  int64_t items;
};

// barrier layout: full[kRing], empty[kRing], acc_full[2], acc_empty[2]
enum { B_FULL = 0, B_EMPTY = kRing, B_ACCF = 2 * kRing, B_ACCE = 2 * kRing + 2, NBAR = 2 * kRing + 4 };

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, int parity, volatile int* abort) {
  for (long long it = 0; it < kWaitLimit; ++it) {
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

// tcgen05.commit of all prior MMAs to an mbarrier, issued by one elected lane.
__device__ __forceinline__ void commit_elect(uint64_t* b) {
  asm volatile(
      "{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\t"
      "@p tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(su32(b)));
}

// Per-CTA walk over (item, row) in a fixed order shared by every role: item
// `it` covers tiles y0 .. y1 - 1 of column (z, seg) and input rows y0 - 1 .. y1.
struct Walk {
  int z, seg, y0, y1;
  __device__ __forceinline__ void set(const Args& g, int64_t item) {
    const int yc = (int)(item % g.ychunks);
    seg = (int)((item / g.ychunks) % g.segs);
    z = (int)(item / ((int64_t)g.ychunks * g.segs));
    y0 = yc * g.ychunk;
    y1 = min(g.H, y0 + g.ychunk);
  }
};

template <int NO>
__global__ void __launch_bounds__(kThr, 1) conv_tc_kernel(Args g, int* timeout_flag) {
  static_assert(NO == 32 || NO == 16, "output channels per MMA");
  constexpr int kW = T * NO * C * 2;  // weight bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  unsigned char* sw = base;                                          // weights
  unsigned char* ring = base + kWBytes;                              // kRing x 3 x 4 x S x 16 (same offset for N = 16)
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + (size_t)kRing * 3 * 4 * g.S * 16);
  unsigned* tslot = reinterpret_cast<unsigned*>(bars + NBAR);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  float* sbias = reinterpret_cast<float*>(tslot + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned strip_bytes = 4u * g.S * 16u;

  for (int k = tid; k < kW / 16; k += kThr)
    reinterpret_cast<uint4*>(sw)[k] = __ldg(reinterpret_cast<const uint4*>(g.w) + k);
  if (tid < C) sbias[tid] = g.bias ? g.bias[tid] : 0.f;
  if (tid == 0) {
    for (int i = 0; i < kRing; ++i) {
      bar_init(&bars[B_FULL + i], kProdWarps * 32);
      bar_init(&bars[B_EMPTY + i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      bar_init(&bars[B_ACCF + i], 1);
      bar_init(&bars[B_ACCE + i], kEpiWarps * 32);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(2 * NO));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // weights -> tensor-core reads
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = *tslot;

  if (warp < kProdWarps) {
    // ---------------- producer ----------------
    // The copy pattern of a row is the same for every row: per thread, up to
    // kMaxCp 16-byte pieces (strip dz, channel chunk c, voxel sv) with their
    // shared-memory offsets, precomputed once.
    constexpr int kMaxCp = (3 * 4 * 176 + kProdWarps * 32 - 1) / (kProdWarps * 32);  // S <= 176
    int cp_dst[kMaxCp], cp_sv[kMaxCp];
    uint64_t cp_dz = 0;  // 2 bits per piece
    const int n16 = 3 * 4 * g.S;
#pragma unroll
    for (int i = 0; i < kMaxCp; ++i) {
      const int idx = tid + i * kProdWarps * 32;
      cp_dst[i] = -1;
      cp_sv[i] = 0;
      if (idx < n16) {
        const int c = idx & 3;
        const int sv = (idx >> 2) % g.S;
        const int dz = idx / (4 * g.S);
        cp_dst[i] = (dz * 4 + c) * g.S * 16 + sv * 16;
        cp_sv[i] = sv * C + c * 8;  // element offset within the strip's voxels (before the row base)
        cp_dz |= (uint64_t)dz << (2 * i);
      }
    }
    int64_t n = 0;  // row sequence number of this CTA
    bool stop = false;
    for (int64_t item = blockIdx.x; item < g.items && !stop; item += gridDim.x) {
      Walk wk;
      wk.set(g, item);
      const int vl0 = wk.seg * kTile - g.B;  // voxel of strip position 0
      for (int yr = wk.y0 - 1; yr <= wk.y1; ++yr, ++n) {
        const int slot = (int)(n % kRing);
        if (n >= kRing && !bar_wait(&bars[B_EMPTY + slot], (int)((n / kRing - 1) & 1), abort)) {
          stop = true;
          break;
        }
        const unsigned sp = su32(ring) + (unsigned)slot * 3u * strip_bytes;
        // Element offset of strip position 0 in each strip's row (z - 1, z, z + 1)
        // (negative for the first segment's halo) and whether that row exists.
        // (Three named values, not an array: a runtime-indexed array would live in local memory.)
        const bool yok = yr >= 0 && yr < g.H;
        const bool ok0 = yok && wk.z >= 1, ok1 = yok, ok2 = yok && wk.z + 1 < g.D;
        const int64_t rowb = ((int64_t)wk.z * g.H + (yok ? yr : 0)) * g.L + vl0;  // strip dz = 1
        const int64_t zstep = (int64_t)g.H * g.L;
        const int64_t rb0 = (rowb - zstep) * C, rb1 = rowb * C, rb2 = (rowb + zstep) * C;
#pragma unroll
        for (int i = 0; i < kMaxCp; ++i) {
          if (cp_dst[i] < 0) continue;
          const int dz = (int)((cp_dz >> (2 * i)) & 3);
          const int vl = vl0 + cp_sv[i] / C;
          const bool rok = dz == 0 ? ok0 : (dz == 1 ? ok1 : ok2);
          const int64_t rb = dz == 0 ? rb0 : (dz == 1 ? rb1 : rb2);
          const bool ok = rok && vl >= 0 && vl < g.L;
          const __nv_bfloat16* src = ok ? g.in + rb + cp_sv[i] : g.in;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sp + (unsigned)cp_dst[i]), "l"(src),
                       "r"(ok ? 16 : 0)
                       : "memory");
        }
        // The slot's barrier completes once every producer thread's copies have landed.
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(&bars[B_FULL + slot]))
                     : "memory");
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == kMmaWarp) {
    // ---------------- MMA ----------------
    // The whole warp runs this loop so that the descriptors stay warp-uniform
    // (uniform registers); one elected lane issues each tcgen05 instruction.
    {
      const unsigned idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NO >> 3) << 17) | ((unsigned)(kTile >> 4) << 24);
      const unsigned sw_a = su32(sw), ring_a = su32(ring);
      const unsigned lbo_a = (unsigned)g.S * 16u;
      const uint64_t wd = desc(sw_a, NO * 16u, 128u);  // + (t 64 NO + ks 32 NO) / 16 per tap
      int64_t nbase = 0;  // row sequence number of row y0 - 1 of the current item
      int64_t k = 0;      // tile sequence number
      bool stop = false;
      for (int64_t item = blockIdx.x; item < g.items && !stop; item += gridDim.x) {
        Walk wk;
        wk.set(g, item);
        for (int y = wk.y0; y < wk.y1; ++y, ++k) {
          // rows y - 1, y, y + 1 have sequence numbers nbase + (y - y0) + {0, 1, 2}
          const int64_t nr = nbase + (y - wk.y0);
          bool ok = true;
          for (int d = 0; d < 3 && ok; ++d) {
            const int64_t m = nr + d;
            // wait only for the newest row (the older two were waited for by earlier tiles)
            if (d == 2 || y == wk.y0) ok = bar_wait(&bars[B_FULL + (int)(m % kRing)], (int)((m / kRing) & 1), abort);
          }
          const int as = (int)(k & 1);
          if (ok && k >= 2) ok = bar_wait(&bars[B_ACCE + as], (int)(((k - 2) >> 1) & 1), abort);
          if (!__all_sync(0xffffffffu, ok)) {
            *abort = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const unsigned dtm = tmem + (unsigned)(as * NO);
          // Descriptor of strip (row y - 1 + b, dz a); a tap adds its shift in
          // 16-byte units to the address field (addresses stay below 256 KB).
          uint64_t sd[3][3];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const unsigned slot = (unsigned)((nr + b) % kRing);
#pragma unroll
            for (int a = 0; a < 3; ++a) sd[b][a] = desc(ring_a + (slot * 3u + a) * strip_bytes, lbo_a, 128u);
          }
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const int a = t / 9, b = (t / 3) % 3, e = t % 3;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint64_t ad = sd[b][a] + (uint64_t)(2 * ks * g.S + e * g.B);
              const uint64_t bd = wd + (uint64_t)(t * 4 * NO + ks * 2 * NO);
              asm volatile(
                  "{\n\t.reg .pred p, q;\n\telect.sync _|p, 0xffffffff;\n\tsetp.ne.u32 q, %4, 0;\n\t"
                  "@p tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(dtm),
                  "l"(ad), "l"(bd), "r"(idesc), "r"((t | ks) ? 1u : 0u));
            }
          }
          commit_elect(&bars[B_ACCF + as]);
          // Rows whose last reader is this tile: y - 1, and at the column's end also y and y + 1.
          const int nfree = (y == wk.y1 - 1) ? 3 : 1;
          for (int d = 0; d < nfree; ++d) commit_elect(&bars[B_EMPTY + (int)((nr + d) % kRing)]);
        }
        nbase += (wk.y1 - wk.y0) + 2;
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int lq = warp & 3;  // TMEM lane quarter this warp may access
    const int row = 32 * lq + lane;
    const float oscale = (NO == 16 && g.scale) ? *g.scale : 1.f;
    int64_t k = 0;
    bool stop = false;
    for (int64_t item = blockIdx.x; item < g.items && !stop; item += gridDim.x) {
      Walk wk;
      wk.set(g, item);
      for (int y = wk.y0; y < wk.y1; ++y, ++k) {
        const int as = (int)(k & 1);
        const bool ok = __all_sync(0xffffffffu, bar_wait(&bars[B_ACCF + as], (int)((k >> 1) & 1), abort));
        if (!ok) {
          *abort = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const unsigned taddr = tmem + ((unsigned)(32 * lq) << 16) + (unsigned)(as * NO);
        if constexpr (NO == 16) {
          unsigned v0;
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v0) : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          asm volatile("tcgen05.fence::before_thread_sync;");
          bar_arrive(&bars[B_ACCE + as]);
          const int vl = wk.seg * kTile + row;
          if (vl < g.L) {
            const int64_t vox = ((int64_t)wk.z * g.H + y) * g.L + vl;
            g.out1[vox] = (__uint_as_float(v0) + sbias[0]) * oscale;
          }
          continue;
        }
        unsigned v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        bar_arrive(&bars[B_ACCE + as]);  // the accumulator is free for tile k + 2
        const int vl = wk.seg * kTile + row;
        if (vl < g.L) {
          const int64_t vox = ((int64_t)wk.z * g.H + y) * g.L + vl;
          float acc[C];
          if (g.mask) {
            float h[C];
            load32(g.mask + vox * C, h);
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = h[c] > 0.f ? __uint_as_float(v[c]) : 0.f;
          } else {
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = fmaxf(__uint_as_float(v[c]) + sbias[c], 0.f);
          }
          store32(g.out + vox * C, acc);
        }
      }
    }
  }
  __syncthreads();
  if (*abort && tid == 0 && timeout_flag) atomicExch(timeout_flag, 1);
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NO));
  }
}

size_t smem_bytes(int S) { return 128 + (size_t)kWBytes + (size_t)kRing * 3 * 4 * S * 16 + NBAR * 8 + 16 + C * 4; }

}  // namespace tc

// ---- loss ----------------------------------------------------------------------
// g = bf16(2 (y - t) / V);  loss += sum (y - t)^2 / V  (last block adds to *loss).
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                   float* __restrict__ g, Dims d, double* loss, Reduce red) {
  __shared__ double sh[8];
  double acc = 0.0;
  const float inv = 2.f / (float)d.V;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < d.V; v += (int64_t)gridDim.x * blockDim.x) {
    const float diff = y[v] - t[v];
    g[v] = round_bf(inv * diff);
    acc += (double)diff * (double)diff;
  }
  double tot;
  if (dev::grid_sum_last(acc, red, &tot, sh)) *loss += tot / (double)d.V;
}

// ---- weight gradients ------------------------------------------------------------
// dW[t][o][i] = sum_v G[v][o] X[v + off t][i] over one chunk of rows (z, y) of the
// volume, written as per-chunk partial sums.  CG / CX: channels of G / X (32 or 1);
// G and X are bfloat16 [V][32] when 32 channels, FP32 [V] when 1.  A thread owns a
// 4 (o) x 4 (i) block of one tap (1 x 4 / 4 x 1 for single-channel operands).
template <int CG, int CX>
__global__ void __launch_bounds__(192) wgrad_kernel(const void* __restrict__ Gp, const void* __restrict__ Xp,
                                                    float* __restrict__ partial, Dims d, int rows_per_chunk) {
  constexpr int NO = CG == 1 ? 1 : 4, NI = CX == 1 ? 1 : 4;
  constexpr int GO = CG / NO, GI = CX / NI;     // groups of o and i
  constexpr int COMBOS = T * GO * GI;
  const int combo = blockIdx.x * blockDim.x + threadIdx.x;
  if (combo >= COMBOS) return;
  const int t = combo / (GO * GI);
  const int og = (combo / GI) % GO, ig = combo % GI;
  const int a = t / 9 - 1, b = (t / 3) % 3 - 1, e = t % 3 - 1;
  const int64_t off = tap_offset(t, d);
  float acc[NO * NI];
#pragma unroll
  for (int k = 0; k < NO * NI; ++k) acc[k] = 0.f;
  const int rows = d.D * d.H;
  const int r0 = blockIdx.y * rows_per_chunk, r1 = min(rows, r0 + rows_per_chunk);
  const int x0 = max(0, -e), x1 = min(d.W, d.W - e);
  for (int r = r0; r < r1; ++r) {
    const int z = r / d.H, y = r % d.H;
    if (z + a < 0 || z + a >= d.D || y + b < 0 || y + b >= d.H) continue;
    const int64_t vb = ((int64_t)r * d.W) * d.B;
    for (int64_t v = vb + (int64_t)x0 * d.B; v < vb + (int64_t)x1 * d.B; ++v) {
      float gv[NO], xv[NI];
      if constexpr (CG == 1) {
        gv[0] = __ldg(reinterpret_cast<const float*>(Gp) + v);
      } else {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(Gp) + v * C + og * 4));
        gv[0] = bf_lo(w.x); gv[1] = bf_hi(w.x); gv[2] = bf_lo(w.y); gv[3] = bf_hi(w.y);
      }
      if constexpr (CX == 1) {
        xv[0] = __ldg(reinterpret_cast<const float*>(Xp) + v + off);
      } else {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(Xp) + (v + off) * C + ig * 4));
        xv[0] = bf_lo(w.x); xv[1] = bf_hi(w.x); xv[2] = bf_lo(w.y); xv[3] = bf_hi(w.y);
      }
#pragma unroll
      for (int o = 0; o < NO; ++o)
#pragma unroll
        for (int i = 0; i < NI; ++i) acc[o * NI + i] = fmaf(gv[o], xv[i], acc[o * NI + i]);
    }
  }
  // partial[chunk][t][o][i] over the full CG x CX block.
  float* dst = partial + (int64_t)blockIdx.y * T * CG * CX + (int64_t)t * CG * CX;
#pragma unroll
  for (int o = 0; o < NO; ++o)
#pragma unroll
    for (int i = 0; i < NI; ++i) dst[(og * NO + o) * CX + ig * NI + i] = acc[o * NI + i];
}

// Bias gradient partials: db[o] = sum_v G[v][o] per chunk of rows.
template <int CG>
__global__ void __launch_bounds__(256) bgrad_kernel(const void* __restrict__ Gp, float* __restrict__ partial, Dims d,
                                                    int rows_per_chunk) {
  __shared__ float sh[256];
  const int rows = d.D * d.H;
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(rows, r0 + rows_per_chunk);
  const int64_t v0 = (int64_t)r0 * d.W * d.B, v1 = (int64_t)r1 * d.W * d.B;
  // thread -> (channel, lane): CG == 32: 32 channels x 8 lanes; CG == 1: 256 lanes.
  const int ch = CG == 1 ? 0 : threadIdx.x % 32;
  const int lane = CG == 1 ? threadIdx.x : threadIdx.x / 32;
  const int lanes = CG == 1 ? 256 : 8;
  float acc = 0.f;
  for (int64_t v = v0 + lane; v < v1; v += lanes) {
    if constexpr (CG == 1) acc += __ldg(reinterpret_cast<const float*>(Gp) + v);
    else acc += bf(reinterpret_cast<const __nv_bfloat16*>(Gp)[v * C + ch]);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < (CG == 1 ? 1 : 32)) {
    float s = 0.f;
    for (int l = 0; l < lanes; ++l) s += sh[CG == 1 ? l : l * 32 + ch];
    partial[(int64_t)blockIdx.x * CG + ch] = s;
  }
}

// Sum the chunk partials (fixed order) and add into the packed gradient:
// weights from partial[chunk][t][o][i] to grad[w_off + (o CIN + i) 27 + t],
// biases from bpartial[chunk][o] to grad[b_off + o].
__global__ void reduce_grads_kernel(const float* __restrict__ partial, const float* __restrict__ bpartial,
                                    int chunks, int co, int ci, float* __restrict__ grad, int64_t w_off,
                                    int64_t b_off) {
  const int nw = T * co * ci;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nw) {
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += partial[(int64_t)c * nw + k];
    const int t = k / (co * ci), o = (k / ci) % co, i = k % ci;
    grad[w_off + ((int64_t)o * ci + i) * T + t] += s;
  } else if (k < nw + co) {
    const int o = k - nw;
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += bpartial[(int64_t)c * co + o];
    grad[b_off + o] += s;
  }
}

// ---- optimiser and weight preparation ---------------------------------------------
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            int64_t n, float lr, float beta1, float beta2, float eps, float bc1, float bc2,
                            float grad_scale) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float gk = g[k] * grad_scale;
    const float mk = beta1 * m[k] + (1.f - beta1) * gk;
    const float vk = beta2 * v[k] + (1.f - beta2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
    g[k] = 0.f;
  }
}

__global__ void prep_kernel(const float* __restrict__ p, Derived* __restrict__ dw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < T * C) {
    const int t = k / C, c = k % C;
    dw->w1f[k] = round_bf(p[kW1 + (int64_t)c * T + t]);
    dw->w4f[k] = round_bf(p[kW4 + (int64_t)c * T + t]);
    dw->w4b[k] = round_bf(p[kW4 + (int64_t)c * T + (T - 1 - t)]);
  }
  if (k < C) {
    dw->b1[k] = p[kB1 + k];
    dw->b2[k] = p[kB2 + k];
    dw->b3[k] = p[kB3 + k];
  }
  if (k == 0) dw->b4[0] = p[kB4];
  if (k < T * C * C) {
    const int t = k / (C * C), i = (k / C) % C, o = k % C;  // [t][i][o]
    dw->w2f[k] = __float2bfloat16_rn(p[kW2 + ((int64_t)o * C + i) * T + t]);
    dw->w3f[k] = __float2bfloat16_rn(p[kW3 + ((int64_t)o * C + i) * T + t]);
    // input gradient: input channel i' = o of the layer, output o' = i, flipped tap
    dw->w2b[k] = __float2bfloat16_rn(p[kW2 + ((int64_t)i * C + o) * T + (T - 1 - t)]);
    dw->w3b[k] = __float2bfloat16_rn(p[kW3 + ((int64_t)i * C + o) * T + (T - 1 - t)]);
    // tensor-core layout: element index of (t, N row o, K col i)
    const int tc = t * C * C + (i / 8) * (8 * C) + o * 8 + (i % 8);
    dw->w2f_tc[tc] = dw->w2f[k];
    dw->w3f_tc[tc] = dw->w3f[k];
    dw->w2b_tc[tc] = dw->w2b[k];
    dw->w3b_tc[tc] = dw->w3b[k];
  }
  if (k < T * 16 * C) {
    const int t = k / (16 * C), o = (k / C) % 16, i = k % C;
    const float v = o == 0 ? p[kW4 + (int64_t)i * T + t] : 0.f;
    dw->w4f_tc[t * 16 * C + (i / 8) * (8 * 16) + o * 8 + (i % 8)] = __float2bfloat16_rn(v);
  }
}

// RMS of a vector into *scale (FP32): sqrt(sum x^2 / n); 1 when it is zero.
__global__ void __launch_bounds__(256) rms_kernel(const float* __restrict__ x, int64_t n, float* scale, Reduce red) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)x[i] * (double)x[i];
  double tot;
  if (dev::grid_sum_last(acc, red, &tot, sh)) {
    const double r = sqrt(tot / (double)n);
    *scale = r > 0.0 ? (float)r : 1.f;
  }
}

}  // namespace net
}  // namespace tca

using namespace tca;
using namespace tca::net;

struct tca_net_s {
  float* params = nullptr;  // master FP32, packed
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  Derived* dw = nullptr;
  int64_t adam_t = 0;
  // activation buffers, sized for cap voxels
  int64_t cap = 0;
  __nv_bfloat16* h[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16* gbuf[2] = {nullptr, nullptr};
  float* y = nullptr;
  float* g = nullptr;
  float* partial = nullptr;   // weight-gradient chunk partials
  float* bpartial = nullptr;
  int chunks_cap = 0;
  double* loss = nullptr;     // device accumulator
  float* scale = nullptr;     // device scalar (RMS of the input)
  Reduce red;
  int num_sms = 0;
  bool force_cuda_cores = false;  // 32 -> 32 layers on the CUDA cores (tests of both paths)
};

namespace {

constexpr int kMaxChunks = 256;
constexpr size_t kConvSmem = (size_t)T * C * C * 2;  // bf16 weights of one 32 -> 32 layer

tca_status net_alloc(tca_net_s* n) {
  cudaError_t e = cudaMalloc((void**)&n->params, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->grads, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->adam_m, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->adam_v, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->dw, sizeof(Derived));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->partial, sizeof(float) * (size_t)kMaxChunks * T * C * C);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->bpartial, sizeof(float) * (size_t)kMaxChunks * C);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->scale, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->red.partials, sizeof(double) * 4096);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->red.ticket, sizeof(unsigned int) * 2);
  if (e == cudaSuccess) e = cudaMemset(n->red.ticket, 0, sizeof(unsigned int) * 2);
  if (e == cudaSuccess) e = cudaMemset(n->grads, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(n->loss, 0, sizeof(double));
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  n->red.max_blocks = 4096;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, dev);
  return TCA_OK;
}

tca_status ensure_act(tca_net_s* n, int64_t V) {
  if (V <= n->cap) return TCA_OK;
  for (auto*& p : n->h) { cudaFree(p); p = nullptr; }
  for (auto*& p : n->gbuf) { cudaFree(p); p = nullptr; }
  cudaFree(n->y);
  cudaFree(n->g);
  n->y = n->g = nullptr;
  n->cap = 0;
  cudaError_t e = cudaSuccess;
  for (auto*& p : n->h)
    if (e == cudaSuccess) e = cudaMalloc((void**)&p, sizeof(__nv_bfloat16) * C * (size_t)V);
  for (auto*& p : n->gbuf)
    if (e == cudaSuccess) e = cudaMalloc((void**)&p, sizeof(__nv_bfloat16) * C * (size_t)V);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->y, sizeof(float) * (size_t)V);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->g, sizeof(float) * (size_t)V);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return TCA_ERR_ALLOC;
  }
  n->cap = V;
  return TCA_OK;
}

tca_status get_dims(const int64_t* dims, Dims* d) {
  for (int k = 0; k < 4; ++k)
    if (dims[k] <= 0 || dims[k] > 65536) return TCA_ERR_INVALID_ARG;
  d->D = (int)dims[0];
  d->H = (int)dims[1];
  d->W = (int)dims[2];
  d->B = (int)dims[3];
  d->V = dims[0] * dims[1] * dims[2] * dims[3];
  if ((int64_t)d->D * d->H > (1 << 30) || d->V > ((int64_t)1 << 34)) return TCA_ERR_INVALID_ARG;
  return TCA_OK;
}

int grid_for(const tca_net_s* n, int64_t V, int per_sm) {
  const int64_t want = (V + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)n->num_sms * per_sm));
}

// Launch of the row-structured 1 -> 32 kernel: one job per 256 voxels of a row.
template <bool MASK>
tca_status launch_1to32(const tca_net_s* n, const float* in, const float* scale, const float* w, const float* bias,
                        const __nv_bfloat16* mask, __nv_bfloat16* out, const Dims& d, cudaStream_t s) {
  const size_t smem = conv1to32_smem(d.B);
  if (smem > 160 * 1024) {
    set_error_message("network: the fourth mode is too long for the first layer's row tiles");
    return TCA_ERR_UNSUPPORTED;
  }
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(conv1to32_kernel<MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return TCA_ERR_CUDA;
    }
  }
  const int64_t L = (int64_t)d.W * d.B;
  const int64_t jobs = (int64_t)d.D * d.H * ((L + kRowVox - 1) / kRowVox);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(jobs, (int64_t)n->num_sms * 8));
  conv1to32_kernel<MASK><<<grid, kThreads, smem, s>>>(in, scale, w, bias, mask, out, d);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

tca_status prep(tca_net_s* n, cudaStream_t s) {
  prep_kernel<<<(T * C * C + 255) / 256, 256, 0, s>>>(n->params, n->dw);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// Work split of the tensor-core convolution: columns (z, segment) of tiles,
// cut along y into chunks so that the persistent CTAs get balanced waves
// (each chunk also reloads three halo rows).
tc::Args tc_geometry(const tca_net_s* n, const Dims& d) {
  tc::Args g{};
  g.D = d.D;
  g.H = d.H;
  g.W = d.W;
  g.B = d.B;
  g.L = d.W * d.B;
  g.segs = (g.L + tc::kTile - 1) / tc::kTile;
  g.S = tc::kTile + 2 * d.B;
  const int64_t cols = (int64_t)d.D * g.segs;
  const int sms = std::max(1, n->num_sms);
  int best = d.H;
  double best_cost = 1e300;
  for (int nc = 1; nc <= d.H; ++nc) {
    const int ych = (d.H + nc - 1) / nc;
    const int64_t items = cols * ((d.H + ych - 1) / ych);
    const double cost = (double)((items + sms - 1) / sms) * (ych + 3);
    if (cost < best_cost) {
      best_cost = cost;
      best = ych;
    }
  }
  g.ychunk = best;
  g.ychunks = (d.H + best - 1) / best;
  g.items = cols * g.ychunks;
  return g;
}

bool tc_supported(const Dims& d) { return d.B <= 24; }

tca_status conv32(tca_net_s* n, const __nv_bfloat16* in, const __nv_bfloat16* w, const __nv_bfloat16* w_tc,
                  const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* out, const Dims& d, cudaStream_t s) {
  if (w_tc && tc_supported(d) && !n->force_cuda_cores) {
    tc::Args g = tc_geometry(n, d);
    g.in = in;
    g.out = out;
    g.w = w_tc;
    g.bias = mask ? nullptr : bias;
    g.mask = mask;
    const size_t smem = tc::smem_bytes(g.S);
    static bool tc_attr = false;
    if (!tc_attr) {
      cudaFuncSetAttribute(tc::conv_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      tc_attr = true;
    }
    const int grid = (int)std::min<int64_t>(g.items, (int64_t)std::max(1, n->num_sms));
    tc::conv_tc_kernel<32><<<grid, tc::kThr, smem, s>>>(g, wait_timeout_flag());
    TCA_LAUNCH_CHECK();
    return TCA_OK;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(conv32to32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
    cudaFuncSetAttribute(conv32to32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
    attr = true;
  }
  const int grid = grid_for(n, d.V, 3);
  if (mask) conv32to32_kernel<true><<<grid, kThreads, kConvSmem, s>>>(in, w, bias, mask, out, d);
  else conv32to32_kernel<false><<<grid, kThreads, kConvSmem, s>>>(in, w, bias, nullptr, out, d);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

// Forward pass into n->h[0..2] and y (y = s Net(u / s) when scaled).
tca_status forward(tca_net_s* n, const float* u, float* y, const Dims& d, bool scaled, cudaStream_t s) {
  const int grid = grid_for(n, d.V, 8);
  TCA_TRY(launch_1to32<false>(n, u, scaled ? n->scale : nullptr, DW(n, w1f), DW(n, b1), nullptr, n->h[0], d, s));
  TCA_TRY(conv32(n, n->h[0], DW(n, w2f), DW(n, w2f_tc), DW(n, b2), nullptr, n->h[1], d, s));
  TCA_TRY(conv32(n, n->h[1], DW(n, w3f), DW(n, w3f_tc), DW(n, b3), nullptr, n->h[2], d, s));
  if (tc_supported(d) && !n->force_cuda_cores) {
    // Layer 4 on the tensor cores with N padded to 16 (one real output channel).
    tc::Args g = tc_geometry(n, d);
    g.in = n->h[2];
    g.out1 = y;
    g.scale = scaled ? n->scale : nullptr;
    g.w = DW(n, w4f_tc);
    g.bias = DW(n, b4);
    static bool tc1_attr = false;
    if (!tc1_attr) {
      cudaFuncSetAttribute(tc::conv_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      tc1_attr = true;
    }
    const int tgrid = (int)std::min<int64_t>(g.items, (int64_t)std::max(1, n->num_sms));
    tc::conv_tc_kernel<16><<<tgrid, tc::kThr, tc::smem_bytes(g.S), s>>>(g, wait_timeout_flag());
  } else {
    conv32to1_kernel<<<grid, kThreads, 0, s>>>(n->h[2], DW(n, w4f), DW(n, b4), scaled ? n->scale : nullptr, y, d);
  }
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template <int CG, int CX>
tca_status wgrad(tca_net_s* n, const void* G, const void* X, const Dims& d, int co, int ci, int64_t w_off,
                 int64_t b_off, cudaStream_t s) {
  constexpr int combos = T * (CG == 1 ? 1 : CG / 4) * (CX == 1 ? 1 : CX / 4);
  const int bx = (combos + 191) / 192;
  const int rows = d.D * d.H;
  const int want = std::max(1, std::min({kMaxChunks, rows, (n->num_sms * 4) / bx}));
  const int rpc = (rows + want - 1) / want;
  const int chunks = (rows + rpc - 1) / rpc;
  dim3 grid(bx, chunks);
  wgrad_kernel<CG, CX><<<grid, 192, 0, s>>>(G, X, n->partial, d, rpc);
  TCA_LAUNCH_CHECK();
  bgrad_kernel<CG><<<chunks, 256, 0, s>>>(G, n->bpartial, d, rpc);
  TCA_LAUNCH_CHECK();
  const int nk = T * co * ci + co;
  reduce_grads_kernel<<<(nk + 255) / 256, 256, 0, s>>>(n->partial, n->bpartial, chunks, co, ci, n->grads, w_off,
                                                       b_off);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

}  // namespace

extern "C" int64_t tca_net_param_count(void) { return kParams; }

extern "C" tca_status tca_net_use_tensor_cores(tca_net_t n, int enable) {
  if (!n) return TCA_ERR_INVALID_ARG;
  n->force_cuda_cores = enable == 0;
  return TCA_OK;
}

extern "C" tca_status tca_net_create(tca_net_t* out, const float* params, cudaStream_t s) {
  if (!out || !params) return TCA_ERR_INVALID_ARG;
  *out = nullptr;
  (void)wait_timeout_flag();
  tca_net_s* n = new tca_net_s();
  tca_status st = net_alloc(n);
  if (st == TCA_OK) st = tca_net_set_params(n, params, s);
  if (st != TCA_OK) {
    tca_net_destroy(n);
    return st;
  }
  *out = n;
  return TCA_OK;
}

extern "C" void tca_net_destroy(tca_net_t n) {
  if (!n) return;
  cudaFree(n->params);
  cudaFree(n->grads);
  cudaFree(n->adam_m);
  cudaFree(n->adam_v);
  cudaFree(n->dw);
  for (auto* p : n->h) cudaFree(p);
  for (auto* p : n->gbuf) cudaFree(p);
  cudaFree(n->y);
  cudaFree(n->g);
  cudaFree(n->partial);
  cudaFree(n->bpartial);
  cudaFree(n->loss);
  cudaFree(n->scale);
  cudaFree(n->red.partials);
  cudaFree(n->red.ticket);
  delete n;
}

extern "C" tca_status tca_net_set_params(tca_net_t n, const float* params, cudaStream_t s) {
  if (!n || !params) return TCA_ERR_INVALID_ARG;
  TCA_CUDA_TRY(cudaMemcpyAsync(n->params, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, s));
  TCA_CUDA_TRY(cudaMemsetAsync(n->adam_m, 0, sizeof(float) * kParams, s));
  TCA_CUDA_TRY(cudaMemsetAsync(n->adam_v, 0, sizeof(float) * kParams, s));
  TCA_CUDA_TRY(cudaMemsetAsync(n->grads, 0, sizeof(float) * kParams, s));
  n->adam_t = 0;
  TCA_TRY(prep(n, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  return TCA_OK;
}

extern "C" tca_status tca_net_get_params(tca_net_t n, float* params, cudaStream_t s) {
  if (!n || !params) return TCA_ERR_INVALID_ARG;
  TCA_CUDA_TRY(cudaMemcpyAsync(params, n->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  return TCA_OK;
}

extern "C" tca_status tca_net_get_grads(tca_net_t n, float* grads, cudaStream_t s) {
  if (!n || !grads) return TCA_ERR_INVALID_ARG;
  TCA_CUDA_TRY(cudaMemcpyAsync(grads, n->grads, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  return TCA_OK;
}

extern "C" tca_status tca_net_forward(tca_net_t n, const int64_t* dims, const float* u, float* y, cudaStream_t s) {
  if (!n || !dims || !u || !y) return TCA_ERR_INVALID_ARG;
  Dims d;
  TCA_TRY(get_dims(dims, &d));
  if (!is_device_ptr(u) || !is_device_ptr(y)) return TCA_ERR_UNSUPPORTED;
  TCA_TRY(ensure_act(n, d.V));
  return forward(n, u, y, d, false, s);
}

extern "C" tca_status tca_net_accumulate(tca_net_t n, const int64_t* dims, const float* u, const float* t,
                                         cudaStream_t s) {
  if (!n || !dims || !u || !t) return TCA_ERR_INVALID_ARG;
  Dims d;
  TCA_TRY(get_dims(dims, &d));
  if (!is_device_ptr(u) || !is_device_ptr(t)) return TCA_ERR_UNSUPPORTED;
  TCA_TRY(ensure_act(n, d.V));
  TCA_TRY(forward(n, u, n->y, d, false, s));
  loss_kernel<<<std::min<int64_t>((d.V + 255) / 256, 1024), 256, 0, s>>>(n->y, t, n->g, d, n->loss, n->red);
  TCA_LAUNCH_CHECK();
  // Layer 4: dW4 from g and h3; input gradient dh3 = conv(g, W4 flipped) masked by h3 > 0.
  TCA_TRY((wgrad<1, C>(n, n->g, n->h[2], d, 1, C, kW4, kB4, s)));
  TCA_TRY(launch_1to32<true>(n, n->g, nullptr, DW(n, w4b), nullptr, n->h[2], n->gbuf[0], d, s));
  // Layer 3: dW3 from dz3 = gbuf[0] and h2; dh2 = conv(dz3, W3^T flipped) masked by h2 > 0.
  TCA_TRY((wgrad<C, C>(n, n->gbuf[0], n->h[1], d, C, C, kW3, kB3, s)));
  TCA_TRY(conv32(n, n->gbuf[0], DW(n, w3b), DW(n, w3b_tc), nullptr, n->h[1], n->gbuf[1], d, s));
  // Layer 2: dW2 from dz2 = gbuf[1] and h1; dh1 masked by h1 > 0.
  TCA_TRY((wgrad<C, C>(n, n->gbuf[1], n->h[0], d, C, C, kW2, kB2, s)));
  TCA_TRY(conv32(n, n->gbuf[1], DW(n, w2b), DW(n, w2b_tc), nullptr, n->h[0], n->gbuf[0], d, s));
  // Layer 1: dW1 from dz1 = gbuf[0] and u.
  TCA_TRY((wgrad<C, 1>(n, n->gbuf[0], u, d, C, 1, kW1, kB1, s)));
  return TCA_OK;
}

extern "C" tca_status tca_net_take_loss(tca_net_t n, double* loss, cudaStream_t s) {
  if (!n || !loss) return TCA_ERR_INVALID_ARG;
  TCA_CUDA_TRY(cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  TCA_CUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(double), s));
  TCA_CUDA_TRY(cudaStreamSynchronize(s));
  return TCA_OK;
}

extern "C" tca_status tca_net_adam(tca_net_t n, float lr, float beta1, float beta2, float eps, float grad_scale,
                                   cudaStream_t s) {
  if (!n || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return TCA_ERR_INVALID_ARG;
  n->adam_t += 1;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)n->adam_t));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)n->adam_t));
  adam_kernel<<<(int)((kParams + 255) / 256), 256, 0, s>>>(n->params, n->grads, n->adam_m, n->adam_v, kParams, lr,
                                                          beta1, beta2, eps, bc1, bc2, grad_scale);
  TCA_LAUNCH_CHECK();
  return prep(n, s);
}

// x0 = s Net(A^T b / s), s = RMS(A^T b), then CG from x0 (tca_solve with x0_given).
namespace {

__global__ void add_kernel(float* __restrict__ x, const float* __restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

// kx <- rhs - kx
__global__ void residual_kernel(const float* __restrict__ rhs, float* __restrict__ kx, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    kx[i] = rhs[i] - kx[i];
}

// d = s Net(v / s), s = RMS(v), into out (device, V floats).
tca_status net_correction(tca_net_s* n, const float* v, float* out, const Dims& d, cudaStream_t s) {
  rms_kernel<<<std::min<int64_t>((d.V + 255) / 256, 1024), 256, 0, s>>>(v, d.V, n->scale, n->red);
  TCA_LAUNCH_CHECK();
  return forward(n, v, out, d, true, s);
}

}  // namespace

extern "C" tca_status tca_solve_net(tca_plan_t plan, tca_net_t n, const void* b, void* x, const tca_solve_opts* opts,
                                    int net_every, tca_solve_info* info, cudaStream_t s) {
  if (!plan || !n || !b || !x || net_every < 0) return TCA_ERR_INVALID_ARG;
  if (plan->prec == TCA_F64) return TCA_ERR_UNSUPPORTED;
  if (plan->d != 4 && plan->d != 3) return TCA_ERR_UNSUPPORTED;
  if (!is_device_ptr(b) || !is_device_ptr(x)) return TCA_ERR_UNSUPPORTED;
  int64_t dims[4] = {plan->n[0], plan->n[1], plan->n[2], plan->d == 4 ? plan->n[3] : 1};
  Dims d;
  TCA_TRY(get_dims(dims, &d));
  TCA_TRY(ensure_act(n, d.V));
  const auto t0 = std::chrono::steady_clock::now();
  // x0 = s Net(A^T b / s): A^T b (FP32) into the net's output buffer, then the network.
  TCA_TRY(tca_apply_T(plan, b, n->y, s));
  TCA_TRY(net_correction(n, n->y, (float*)x, d, s));
  tca_solve_opts o = opts ? *opts : tca_solve_opts{};
  if (!opts) {
    o.rtol = 1e-6;
    o.max_iter = 10000;
  }
  const int max_iter = o.max_iter > 0 ? o.max_iter : 10000;
  o.x0_given = 1;
  tca_solve_info acc{}, step{};
  int corrections = 0;
  tca_status st = TCA_OK;
  for (;;) {
    o.max_iter = net_every > 0 ? std::min(net_every, max_iter - acc.iters) : max_iter - acc.iters;
    st = tca_solve(plan, b, x, &o, &step, s);
    acc.iters += step.iters;
    acc.refinements += step.refinements;
    acc.rel_res_true = step.rel_res_true;
    acc.rel_res_recursive = step.rel_res_recursive;
    acc.sweep_ms += step.sweep_ms;
    acc.sweep_launches += step.sweep_launches;
    if (st != TCA_ERR_NOT_CONVERGED || net_every == 0 || acc.iters >= max_iter) break;
    // Preconditioner step: x += s Net(r / s) on the residual r = A^T b - K x
    // (A^T b in FP32 is still in the net's output buffer), then CG restarts from x.
    const int vg = (int)std::min<int64_t>((d.V + 255) / 256, (int64_t)n->num_sms * 8);
    TCA_TRY(tca_apply_normal(plan, x, n->g, s));
    residual_kernel<<<vg, 256, 0, s>>>(n->y, n->g, d.V);
    TCA_LAUNCH_CHECK();
    TCA_TRY(net_correction(n, n->g, n->g, d, s));
    add_kernel<<<vg, 256, 0, s>>>((float*)x, n->g, d.V);
    TCA_LAUNCH_CHECK();
    ++corrections;
  }
  if (info) {
    *info = acc;
    info->refinements = corrections;  // preconditioner steps taken inside the solve
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return st;
}
