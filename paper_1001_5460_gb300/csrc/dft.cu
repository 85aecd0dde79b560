// Discrete Fourier transform over several modes (Table 1: F = E G H C with
// one-dimensional DFT transforms), on complex data held as two real tensors.
//
// Along each selected mode k the complex tensor z = re + i im is multiplied by
// F_k = C_k + i S_k with C_k[j][i] = cos(2 pi j i / n_k) and S_k[j][i] =
// -sin(2 pi j i / n_k) (inverse: +sin, both divided by n_k):
//   re' = re x_k C_k - im x_k S_k,   im' = re x_k S_k + im x_k C_k
// four real dense mode products and two combinations per mode, the products
// on the library's dense mode-product kernels (tcgen05 3xTF32 for FP32 data
// where the operand tiles fit, CUDA cores otherwise; FP64 natively).  This is
// the separable definition, O(n_k) work per output and mode, not an FFT.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tca_internal.cuh"

namespace tca {
namespace {

constexpr int kDftThreads = 256;
constexpr double kPi = 3.14159265358979323846;

// out = a + sb * b (out may be a).
template <typename T>
__global__ void __launch_bounds__(kDftThreads) dft_combine_kernel(const T* a, const T* __restrict__ b, T* out,
                                                                  int64_t n, T sb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] + sb * b[i];
}

// One plan per real factor family: factor k = C_k (or S_k) on the selected
// modes (dense), an ELL-4 identity elsewhere (never applied).
tca_status dft_plan(int order, const int64_t* dims, uint32_t mask, bool sine, bool inverse, tca_precision prec,
                    cudaStream_t s, tca_plan_s** out) {
  std::vector<std::vector<double>> vals(order);
  std::vector<std::vector<int32_t>> col0(order);
  tca_factor f[kMaxModes] = {};
  for (int k = 0; k < order; ++k) {
    const int64_t n = dims[k];
    if (!((mask >> k) & 1)) {
      vals[k].assign((size_t)n * 4, 0.0);
      col0[k].resize((size_t)n);
      for (int64_t i = 0; i < n; ++i) {
        col0[k][i] = (int32_t)i;
        vals[k][i * 4] = 1.0;
      }
      f[k].kind = TCA_FACTOR_ELL4;
      f[k].m = n;
      f[k].n = n;
      f[k].values = vals[k].data();
      f[k].col0 = col0[k].data();
      continue;
    }
    vals[k].assign((size_t)(n * n), 0.0);
    {
      const double scale = inverse ? 1.0 / (double)n : 1.0;
      for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
          // The angle from the exact integer product j i mod n.
          const double th = 2.0 * kPi * (double)((j * i) % n) / (double)n;
          vals[k][j * n + i] = sine ? (inverse ? std::sin(th) : -std::sin(th)) * scale : std::cos(th) * scale;
        }
    }
    f[k].kind = TCA_FACTOR_DENSE;
    f[k].m = n;
    f[k].n = n;
    f[k].values = vals[k].data();
  }
  const tca_reg none = {0.0, 0u, 0u};
  return tca_plan(out, order, dims, f, &none, prec, s);
}

template <typename T>
tca_status run_dft(int order, const int64_t* dims, uint32_t mask, bool inverse, tca_precision prec, const T* re_in,
                   const T* im_in, T* re_out, T* im_out, cudaStream_t s) {
  int64_t N = 1;
  for (int k = 0; k < order; ++k) N *= dims[k];
  tca_plan_s* pc = nullptr;
  tca_plan_s* ps = nullptr;
  T* work[3] = {nullptr, nullptr, nullptr};  // re and im of the intermediate, a product's scratch
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    for (T* w : work) cudaFree(w);
    if (pc) tca_destroy(pc);
    if (ps) tca_destroy(ps);
  };
  tca_status st = dft_plan(order, dims, mask, false, inverse, prec, s, &pc);
  if (st == TCA_OK) st = dft_plan(order, dims, mask, true, inverse, prec, s, &ps);
  for (int w = 0; w < 3 && st == TCA_OK; ++w) {
    const cudaError_t e = cudaMalloc((void**)&work[w], sizeof(T) * (size_t)N);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      st = TCA_ERR_ALLOC;
    }
  }
  if (st != TCA_OK) {
    cleanup();
    return st;
  }
  int ks[kMaxModes], nk = 0;
  for (int k = 0; k < order; ++k)
    if ((mask >> k) & 1) ks[nk++] = k;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 1023) / 1024, 4096));
  const T* cre = re_in;
  const T* cim = im_in;
  for (int step = 0; step < nk && st == TCA_OK; ++step) {
    const int k = ks[step];
    // The last mode writes the outputs; earlier ones alternate so that a step
    // never writes what it reads.
    const bool to_out = ((nk - 1 - step) % 2) == 0;
    T* nre = to_out ? re_out : work[0];
    T* nim = to_out ? im_out : work[1];
    int64_t O = 1, I = 1;
    for (int a = 0; a < k; ++a) O *= dims[a];
    for (int a = k + 1; a < order; ++a) I *= dims[a];
    const ModeOp& c = pc->mode[k].fwd;
    const ModeOp& sn = ps->mode[k].fwd;
    st = launch_mode_op<T, T, T>(c, cre, nre, O, I, s);  // re' = re C ...
    if (st == TCA_OK && cim) {
      st = launch_mode_op<T, T, T>(sn, cim, work[2], O, I, s);  // ... - im S
      if (st == TCA_OK) {
        dft_combine_kernel<T><<<grid, kDftThreads, 0, s>>>(nre, work[2], nre, N, T(-1));
        const cudaError_t e = cudaGetLastError();
        note_launches(1);
        if (e != cudaSuccess) {
          set_cuda_error(e);
          st = TCA_ERR_CUDA;
        }
      }
    }
    if (st == TCA_OK) st = launch_mode_op<T, T, T>(sn, cre, nim, O, I, s);  // im' = re S ...
    if (st == TCA_OK && cim) {
      st = launch_mode_op<T, T, T>(c, cim, work[2], O, I, s);  // ... + im C
      if (st == TCA_OK) {
        dft_combine_kernel<T><<<grid, kDftThreads, 0, s>>>(nim, work[2], nim, N, T(1));
        const cudaError_t e = cudaGetLastError();
        note_launches(1);
        if (e != cudaSuccess) {
          set_cuda_error(e);
          st = TCA_ERR_CUDA;
        }
      }
    }
    cre = nre;
    cim = nim;
  }
  cleanup();
  return st;
}

}  // namespace
}  // namespace tca

using namespace tca;

extern "C" tca_status tca_apply_dft(int order, const int64_t* dims, uint32_t mode_mask, int inverse,
                                    tca_precision prec, const void* re_in, const void* im_in, void* re_out,
                                    void* im_out, cudaStream_t stream) {
  if (!dims || !re_in || !re_out || !im_out) return TCA_ERR_INVALID_ARG;
  if (order < 1 || order > kMaxModes) return TCA_ERR_INVALID_ARG;
  if (mode_mask == 0 || (mode_mask >> order) != 0) return TCA_ERR_INVALID_ARG;
  if (prec != TCA_F32 && prec != TCA_F64) return TCA_ERR_INVALID_ARG;
  const void* outs[2] = {re_out, im_out};
  const void* ins[2] = {re_in, im_in};
  if (re_out == im_out) return TCA_ERR_INVALID_ARG;
  for (const void* o : outs)
    for (const void* i : ins)
      if (o == i) return TCA_ERR_INVALID_ARG;
  // Plans take three or four modes: lower orders get trailing modes of length 1.
  int64_t d[kMaxModes];
  int64_t N = 1;
  for (int k = 0; k < order; ++k) {
    if (dims[k] <= 0) return TCA_ERR_SHAPE;
    if (((mode_mask >> k) & 1) && dims[k] > 256) return TCA_ERR_UNSUPPORTED;  // dense factors up to 256 x 256
    if (dims[k] > ((int64_t)1 << 24)) return TCA_ERR_UNSUPPORTED;
    if (dims[k] > ((int64_t)1 << 40) / N) return TCA_ERR_UNSUPPORTED;
    N *= dims[k];
    d[k] = dims[k];
  }
  const int ord = std::max(order, 3);
  for (int k = order; k < ord; ++k) d[k] = 1;
  if (!is_device_ptr(re_in) || (im_in && !is_device_ptr(im_in)) || !is_device_ptr(re_out) || !is_device_ptr(im_out)) {
    set_error_message("tca_apply_dft takes device buffers");
    return TCA_ERR_INVALID_ARG;
  }
  if (prec == TCA_F64)
    return run_dft<double>(ord, d, mode_mask, inverse != 0, prec, (const double*)re_in, (const double*)im_in,
                           (double*)re_out, (double*)im_out, stream);
  return run_dft<float>(ord, d, mode_mask, inverse != 0, prec, (const float*)re_in, (const float*)im_in,
                        (float*)re_out, (float*)im_out, stream);
}
