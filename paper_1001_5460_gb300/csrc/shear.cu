// One-dimensional shear transforms (Table 1: rotation as a product of 1D shear
// transforms).  A shear along mode a driven by mode b resamples every line
// along mode a at positions moved by slope * (i_b - center):
//
//   Y[.., i_a, .., i_b, ..] = sum_j h(i_a - slope (i_b - center) - j) X[.., j, .., i_b, ..]
//
// with j over the line's points and h the linear (hat) kernel or cubic
// convolution with a = -1/2.  Unlike the factors of Eq. separable_transf the
// transformation differs from line to line (it carries the index of mode b),
// so it is its own kernel rather than a plan factor.  Three such shears with
// slopes tan(t/2), -sin(t), tan(t/2) rotate a plane by t.
//
// Layout: the grid's y dimension is i_b; each block forms the shift of its
// lines once (FP64 position, its integer part and the tap weights from the
// fraction) and then streams the elements with that i_b in storage order
// (32-bit index arithmetic below 2^31 elements), 16-byte vectors along the
// fastest mode where it is neither of the two.  HBM-bound: each element is
// read up to four times from nearby addresses (L1/L2) and written once.
#include <algorithm>
#include <cmath>

#include "tca_internal.cuh"

namespace tca {
namespace {

constexpr int kShearThreads = 256;

// Weights of the taps j0 - 1 .. j0 + 2 at fraction f of the position p = j0 + f.
__device__ __forceinline__ double shear_h(double u, int kind) {
  u = fabs(u);
  if (kind == 1) return u < 1.0 ? 1.0 - u : 0.0;
  const double a = -0.5;
  if (u <= 1.0) return ((a + 2.0) * u - (a + 3.0)) * u * u + 1.0;
  if (u < 2.0) return ((a * u - 5.0 * a) * u + 8.0 * a) * u - 4.0 * a;
  return 0.0;
}

template <typename I>
struct ShearGeom {
  I n_a, stride_a;  // mode a: length and stride (elements)
  I inner_b;        // product of the sizes after mode b (its stride)
  I n_b;
  I per_b;          // elements with one value of i_b: N / n_b
};

// 16-byte vectors along the fastest mode (float4 / double2).
template <typename T> struct ShearVec;
template <> struct ShearVec<float> { using t = float4; static constexpr int n = 4; };
template <> struct ShearVec<double> { using t = double2; static constexpr int n = 2; };

// VEC: neither mode a nor mode b is the fastest mode, whose length is a
// multiple of the vector width, and x, y are 16-byte aligned: the VN
// consecutive outputs along the fastest mode share i_a, i_b and the taps, so
// one thread forms them from VN-wide loads of the same taps.
template <typename T, typename I, bool VEC>
__global__ void __launch_bounds__(kShearThreads) shear_kernel(const T* __restrict__ x, T* __restrict__ y,
                                                              ShearGeom<I> g, double slope, double center, int kind) {
  __shared__ int s_k0;
  __shared__ T s_w[4];
  const I ib = (I)blockIdx.y;
  if (threadIdx.x == 0) {
    // The source position of output i_a is i_a + q, q = -slope (i_b - center): taps
    // i_a + floor(q) - 1 .. i_a + floor(q) + 2.  A shift beyond n_a + 4 reads nothing
    // either way, so floor(q) is clamped to [-(n_a + 4), n_a + 4].
    const double q = -slope * ((double)ib - center);
    const double fq = floor(q);
    const double f = q - fq;
    const double lim = (double)g.n_a + 4.0;
    s_k0 = (int)fmin(fmax(fq, -lim), lim);
    for (int m = 0; m < 4; ++m) s_w[m] = (T)shear_h(f - (double)(m - 1), kind);
  }
  __syncthreads();
  const long long k0 = s_k0;
  T w[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) w[m] = s_w[m];
  constexpr int VN = VEC ? ShearVec<T>::n : 1;
  using VT = typename ShearVec<T>::t;
  const I groups = g.per_b / (I)VN;
  for (I e4 = (I)(blockIdx.x * blockDim.x + threadIdx.x); e4 < groups; e4 += (I)(gridDim.x * blockDim.x)) {
    const I e = e4 * (I)VN;
    const I outer = e / g.inner_b, r = e - outer * g.inner_b;
    const I gi = (outer * g.n_b + ib) * g.inner_b + r;
    const I ia = (gi / g.stride_a) % g.n_a;
    const I base = gi - ia * g.stride_a;
    if constexpr (VEC) {
      VT acc;
      T* as = reinterpret_cast<T*>(&acc);
#pragma unroll
      for (int c = 0; c < VN; ++c) as[c] = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const long long j = (long long)ia + k0 + (m - 1);
        if (w[m] != T(0) && j >= 0 && j < (long long)g.n_a) {
          const VT v = reinterpret_cast<const VT*>(x)[(base + (I)j * g.stride_a) / (I)VN];
          const T* vs = reinterpret_cast<const T*>(&v);
#pragma unroll
          for (int c = 0; c < VN; ++c) as[c] += w[m] * vs[c];
        }
      }
      reinterpret_cast<VT*>(y)[gi / (I)VN] = acc;
    } else {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const long long j = (long long)ia + k0 + (m - 1);
        if (w[m] != T(0) && j >= 0 && j < (long long)g.n_a) acc += w[m] * x[base + (I)j * g.stride_a];
      }
      y[gi] = acc;
    }
  }
}

template <typename T, typename I>
tca_status launch_shear_as(const int64_t* dims, int order, int mode_a, int mode_b, double slope, double center,
                           int kind, const T* x, T* y, cudaStream_t s) {
  ShearGeom<I> g{};
  int64_t N = 1, stride_a = 1, inner_b = 1;
  for (int k = 0; k < order; ++k) N *= dims[k];
  for (int k = mode_a + 1; k < order; ++k) stride_a *= dims[k];
  for (int k = mode_b + 1; k < order; ++k) inner_b *= dims[k];
  g.n_a = (I)dims[mode_a];
  g.stride_a = (I)stride_a;
  g.inner_b = (I)inner_b;
  g.n_b = (I)dims[mode_b];
  g.per_b = (I)(N / dims[mode_b]);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // About eight resident blocks per SM over all lines, at least one per line.
  const int last = order - 1;
  constexpr int VW = ShearVec<T>::n;
  const bool vec = mode_a != last && mode_b != last && dims[last] % VW == 0 && (uintptr_t)x % 16 == 0 &&
                   (uintptr_t)y % 16 == 0;
  const int64_t per_thread = vec ? VW : 1;
  const int64_t want_x = (N / dims[mode_b] / per_thread + kShearThreads - 1) / kShearThreads;
  const int64_t cap_x = std::max<int64_t>(1, (int64_t)sms * 8 / dims[mode_b] + 1);
  const dim3 grid((unsigned)std::min(want_x, cap_x), (unsigned)dims[mode_b]);
  if (vec) shear_kernel<T, I, true><<<grid, kShearThreads, 0, s>>>(x, y, g, slope, center, kind);
  else shear_kernel<T, I, false><<<grid, kShearThreads, 0, s>>>(x, y, g, slope, center, kind);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

template <typename T>
tca_status launch_shear(int order, const int64_t* dims, int mode_a, int mode_b, double slope, double center,
                        int kind, const T* x, T* y, cudaStream_t s) {
  int64_t N = 1;
  for (int k = 0; k < order; ++k) N *= dims[k];
  if (dims[mode_b] > 65535 || dims[mode_a] >= (int64_t)1 << 30) return TCA_ERR_UNSUPPORTED;  // grid y; tap range
  if (N < ((int64_t)1 << 31))
    return launch_shear_as<T, uint32_t>(dims, order, mode_a, mode_b, slope, center, kind, x, y, s);
  return launch_shear_as<T, int64_t>(dims, order, mode_a, mode_b, slope, center, kind, x, y, s);
}

}  // namespace
}  // namespace tca

using namespace tca;

extern "C" tca_status tca_apply_shear(int order, const int64_t* dims, int mode_a, int mode_b, double slope,
                                      double center, int kind, tca_precision prec, const void* x, void* y,
                                      cudaStream_t stream) {
  if (!dims || !x || !y || x == y) return TCA_ERR_INVALID_ARG;
  if (order < 2 || order > kMaxModes) return TCA_ERR_INVALID_ARG;
  if (mode_a < 0 || mode_a >= order || mode_b < 0 || mode_b >= order || mode_a == mode_b) return TCA_ERR_INVALID_ARG;
  if (kind != TCA_SHEAR_LINEAR && kind != TCA_SHEAR_CUBIC) return TCA_ERR_INVALID_ARG;
  if (!std::isfinite(slope) || !std::isfinite(center)) return TCA_ERR_INVALID_ARG;
  if (prec != TCA_F32 && prec != TCA_F64) return TCA_ERR_INVALID_ARG;
  int64_t N = 1;
  for (int k = 0; k < order; ++k) {
    if (dims[k] <= 0) return TCA_ERR_SHAPE;
    if (dims[k] > ((int64_t)1 << 40) / N) return TCA_ERR_UNSUPPORTED;  // more than 2^40 elements
    N *= dims[k];
  }
  if (!is_device_ptr(x) || !is_device_ptr(y)) {
    set_error_message("tca_apply_shear takes device buffers");
    return TCA_ERR_INVALID_ARG;
  }
  if (prec == TCA_F64)
    return launch_shear<double>(order, dims, mode_a, mode_b, slope, center, kind, (const double*)x, (double*)y,
                                stream);
  return launch_shear<float>(order, dims, mode_a, mode_b, slope, center, kind, (const float*)x, (float*)y, stream);
}
