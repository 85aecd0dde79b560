// Vector steps of a CG iteration on caller-owned float vectors, for solvers
// that drive the iteration themselves (the slab-partitioned solve, where each
// rank owns a contiguous run of mode-1 planes and the ranks combine their
// inner products with an all-reduce).  These are the vector operations of
// Fig. 2 (Sec. 4.1): C := C + alpha P, R := R - alpha Q, P := R + beta P and
// the inner products <P, Q>, <R, R>.
#include <algorithm>

#include "tca_internal.cuh"

namespace {

constexpr int kThreads = 256;

// y = a x + b y
__global__ void __launch_bounds__(kThreads) axpby_kernel(float* __restrict__ y, const float* __restrict__ x, float a,
                                                         float b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], b * y[i]);
}

// *out += sum_i a[i] b[i]: FP32 products summed in FP64 per thread, per block,
// then one FP64 atomic per block (the caller's stream zeroes *out first).
__global__ void __launch_bounds__(kThreads) dot_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                                       int64_t n, double* out) {
  __shared__ double sh[kThreads / 32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  const double t = tca::dev::block_sum(acc, sh);
  if (threadIdx.x == 0) atomicAdd(out, t);
}

int grid_for(int64_t n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int64_t want = (n + kThreads * 4 - 1) / (kThreads * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
}

}  // namespace

extern "C" tca_status tca_vec_axpby(float* y, const float* x, double a, double b, int64_t n, cudaStream_t stream) {
  if (n < 0 || (n > 0 && (!y || !x))) return TCA_ERR_INVALID_ARG;
  if (n == 0) return TCA_OK;
  if (!tca::is_device_ptr(y) || !tca::is_device_ptr(x)) return TCA_ERR_UNSUPPORTED;
  axpby_kernel<<<grid_for(n), kThreads, 0, stream>>>(y, x, (float)a, (float)b, n);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}

extern "C" tca_status tca_vec_dot(const float* a, const float* b, int64_t n, double* out, cudaStream_t stream) {
  if (!out || n < 0 || (n > 0 && (!a || !b))) return TCA_ERR_INVALID_ARG;
  if (!tca::is_device_ptr(out) || (n > 0 && (!tca::is_device_ptr(a) || !tca::is_device_ptr(b))))
    return TCA_ERR_UNSUPPORTED;
  TCA_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), stream));
  if (n == 0) return TCA_OK;
  dot_kernel<<<grid_for(n), kThreads, 0, stream>>>(a, b, n, out);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}
