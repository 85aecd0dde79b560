// Relative residual norm without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want to
// check a solution: code that must not call cudaMalloc after start-up (a
// real-time loop with a fixed memory budget, a process whose device memory is
// owned by another allocator, or a library hook that runs while the caller
// holds its allocator lock).  tca_rel_residual_noalloc serves them: it is the
// two-norm reduction the solver uses for its true residual, but its per-block
// partial sums live in one fixed, file-scope device array instead of a
// plan's workspace, so the call allocates nothing.
//
// The array below is a static device variable: every GPU that loads this
// library holds it (256 KiB) until the process exits.  Host code may not use
// its name as an address; the device address is looked up with
// cudaGetSymbolAddress during the first call on a device (set-up), and again
// on the first call after that device's context changed (a cudaDeviceReset
// unloads the module, so an address cached from before would be stale).  Every call
// shares the array and it keeps the last call's contents, so the call clears
// the counter it needs at zero before launching, and calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// the array and give undefined results.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "tca_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaChunk = 8192;                      // elements reduced by one block
constexpr int kNaMaxBlocks = 16384;                 // partial-sum slots per norm
constexpr int64_t kNaMaxN = (int64_t)kNaChunk * kNaMaxBlocks;  // 134,217,728 elements
constexpr int kNaDoubles = 2 * kNaMaxBlocks + 1;    // two partial arrays + counter word

// Layout: [0, kNaMaxBlocks) partials of ||rhs - kx||^2, [kNaMaxBlocks, 2 kNaMaxBlocks)
// partials of ||rhs||^2, last slot: arrival counter (as unsigned int).
static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};  // context the cached address belongs to

// Current driver context (the runtime's primary context of the current
// device), through the runtime's driver entry point; null if unavailable.
void* current_context() {
  using GetCurrent = CUresult (*)(CUcontext*);
  static GetCurrent fn = []() -> GetCurrent {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<GetCurrent>(f);
    return nullptr;
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

__device__ __forceinline__ double na_block_sum(double v, double* sh) {
  v = tca::dev::warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = lane < (kNaThreads / 32) ? sh[lane] : 0.0;
  if (wid == 0) t = tca::dev::warp_sum(t);
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kNaThreads) rel_residual_noalloc_kernel(const double* __restrict__ rhs,
                                                                          const double* __restrict__ kx, int64_t n,
                                                                          double* __restrict__ out,
                                                                          double* __restrict__ scratch) {
  __shared__ double sh[kNaThreads / 32];
  __shared__ bool last;
  double* part_rr = scratch;
  double* part_bb = scratch + kNaMaxBlocks;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + 2 * kNaMaxBlocks);
  const int64_t lo = (int64_t)blockIdx.x * kNaChunk;
  const int64_t hi = lo + kNaChunk < n ? lo + kNaChunk : n;
  double rr = 0.0, bb = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kNaThreads) {
    const double b = rhs[i];
    const double r = b - kx[i];
    rr += r * r;
    bb += b * b;
  }
  rr = na_block_sum(rr, sh);
  bb = na_block_sum(bb, sh);
  if (threadIdx.x == 0) {
    part_rr[blockIdx.x] = rr;
    part_bb[blockIdx.x] = bb;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double srr = 0.0, sbb = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kNaThreads) {
    srr += ((volatile double*)part_rr)[i];
    sbb += ((volatile double*)part_bb)[i];
  }
  srr = na_block_sum(srr, sh);
  sbb = na_block_sum(sbb, sh);
  if (threadIdx.x == 0) {
    *out = sbb > 0.0 ? sqrt(srr) / sqrt(sbb) : sqrt(srr);
    *counter = 0u;
  }
}

// Device address of the scratch array on the current device: looked up on
// the first call on that device and again whenever the device's context is
// not the one the cached address was taken in.
tca_status scratch_for_current_device(double** addr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    tca::set_cuda_error(e);
    return TCA_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TCA_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  void* ctx = current_context();
  if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      tca::set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
      return TCA_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
    // cudaGetSymbolAddress made the primary context current if it was not yet.
    g_scratch_ctx[dev] = ctx ? ctx : current_context();
  }
  *addr = g_scratch_addr[dev];
  return TCA_OK;
}

}  // namespace

extern "C" tca_status tca_rel_residual_noalloc(const double* rhs, const double* kx, int64_t n, double* out,
                                               cudaStream_t stream) {
  if (!out || n < 0 || (n > 0 && (!rhs || !kx))) return TCA_ERR_INVALID_ARG;
  if (n > kNaMaxN) {
    tca::set_error_message("tca_rel_residual_noalloc: n exceeds the fixed scratch limit of 134217728 elements");
    return TCA_ERR_UNSUPPORTED;
  }
  double* scratch = nullptr;
  TCA_TRY(scratch_for_current_device(&scratch));
  // The arrival counter must start at zero; a previous call leaves it at zero
  // unless that call was interrupted, so clear it on every call.
  TCA_CUDA_TRY(cudaMemsetAsync(scratch + 2 * kNaMaxBlocks, 0, sizeof(double), stream));
  const int blocks = n == 0 ? 1 : (int)((n + kNaChunk - 1) / kNaChunk);
  rel_residual_noalloc_kernel<<<blocks, kNaThreads, 0, stream>>>(rhs, kx, n, out, scratch);
  TCA_LAUNCH_CHECK();
  return TCA_OK;
}
