// Internal declarations of the tca library: plan layout, error plumbing and
// small device helpers shared by the kernels.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <vector>

#include "../../include/tca.h"

namespace tca {

constexpr int kMaxModes = 4;
constexpr int kGramHalf = 3;  // G_k = A_k^T A_k of a 4-wide band is 7-banded
constexpr int kLapHalf = 2;   // D2^T D2 is 5-banded
constexpr int kMaxBandW = 16; // widest transposed ELL4 band accepted
constexpr int kMaxProfiledIters = 64;  // iterations per graph replay when sweeps are timed
constexpr int kDirBufs = 4;            // CG direction buffers; x is updated once per kDirBufs iterations

// y[o] = sum_{e < W} w[o*W + e] * x[start[o] + e]; indices outside [0, n_in)
// carry weight 0 in w and are skipped by the kernels.
struct Band {
  int64_t n_out = 0, n_in = 0;
  int W = 0;
  int32_t* start = nullptr;  // device, n_out
  float* w32 = nullptr;      // device, n_out * W
  double* w64 = nullptr;     // device, n_out * W
  float2* wff = nullptr;     // device, n_out * W: w64 split into (hi, lo) floats
  int rows32 = 0;            // input rows spanned by any 32 consecutive outputs (TMA tile height)
  bool unit = false;         // start[j] = start[0] + j (Gram and regulariser bands)
  std::vector<int32_t> start_host;  // host copy of start (transposed-factor bands)
};

// Row-major n_out x n_in matrix.
struct Dense {
  int64_t n_out = 0, n_in = 0;
  float* a32 = nullptr;
  double* a64 = nullptr;
  float2* aff = nullptr;          // a64 split into (hi, lo) floats
  int32_t* zero_start = nullptr;  // n_out zeros: the matrix viewed as a full-width band
};

enum OpKind { OP_BAND = 0, OP_DENSE = 1 };

struct ModeOp {
  int kind = OP_BAND;
  Band band;
  Dense dense;
  int tc_split = 0;  // dense FP32 products on tensor cores: 0 off, 1 TF32, 2 3xTF32
  int sm_cap = 0;    // SMs its persistent kernels may fill (0: the whole GPU; set by batched solves)
  const struct Scalars* stop = nullptr;  // preconditioner factors: the tensor-core product returns at
                                         // entry once these CG stop flags are set
  int64_t n_out() const { return kind == OP_BAND ? band.n_out : dense.n_out; }
  int64_t n_in() const { return kind == OP_BAND ? band.n_in : dense.n_in; }
};

struct Mode {
  int64_t n = 0, m = 0;
  int factor_kind = TCA_FACTOR_DENSE;
  ModeOp fwd;   // A_k   (m x n)
  ModeOp bwd;   // A_k^T (n x m)
  ModeOp gram;  // G_k = A_k^T A_k (n x n): 7-band (W=7, start=i-3) or dense
  bool reg = false;
  Band lap;     // lambda * D2^T D2 as a 5-band (W=5, start=i-2); zeros if !reg
};

// CG scalars, resident on the device (FP64, Fig. 2 names).
struct Scalars {
  double rho;       // <R, R>
  double rho_new;   // rho1
  double pq;        // <P, Q>
  double alpha;
  double beta;      // rho1 / rho for the next direction update
  double bnorm;     // ||rhs||
  double rtol;      // stopping threshold on sqrt(rho) / bnorm
  double aux;       // spare reduction slot (true residual norm^2, dots)
  int32_t converged;
  int32_t breakdown;
  int32_t iters;     // CG iterations completed on the device
  int32_t max_iter;  // kernels of an iteration skip their work once iters reaches it
  int32_t restarts;  // device-side restarts from the true residual (batched solve)
  int32_t pad;
  // Grouped solution update: alpha of the first npend positions of the
  // current group of kDirBufs iterations, whose x += alpha p is still pending.
  double alpha_hist[kDirBufs - 1];
  int32_t npend;
  int32_t pad2;
};

// True once the iteration loop must stop doing work (converged, broken down or
// out of iterations); every CG kernel tests it on entry.
__host__ __device__ inline bool cg_done(const Scalars* s) {
  return s->converged | s->breakdown | (s->iters >= s->max_iter);
}

// Reduction scratch for the last-block-finishes pattern.
struct Reduce {
  double* partials = nullptr;  // one slot per block
  unsigned int* ticket = nullptr;
  int max_blocks = 0;
};

// Alternative coefficients for the fused sweep: the same kernel applies any
// operator of the form (B_1 kron .. kron B_d) + sum_k (I .. C_k .. I) with
// 7-band B_k and 5-band C_k (the banded separable preconditioner: B_k the
// truncated inverses, C_k zero).
struct FusedBands {
  const float* g[kMaxModes] = {};
  const float* l[kMaxModes] = {};
  float g4[8 * 7] = {};  // n4 = 8 plans: B_4 and C_4 by [i4][tap] (kernel parameters)
  float l4[8 * 5] = {};
};

// State of a TCA_BF16_IR plan's inner CG (normal_bf16.cu): the inner axis
// c = (i3, i4) of length nc split into tiles of 128, each with its W = G_3 kron
// G_4 and R = lambda (L_3 kron I + I kron L_4) operand tiles (bfloat16,
// KC chunks of 8 inputs x 128 outputs x 16 bytes, W then R per tile), the
// bfloat16 CG vectors and their TMA views.
struct Bf16State {
  int64_t nc = 0;
  int H = 0, KC = 0, ctiles = 0;
  int nchunks = 0;                  // tile extent along mode 1 chosen by tca_autotune (0: wave model)
  int model_nchunks = 0;            // chunk count the last sweep launched with
  int rpt = 4;                      // core rows per worker thread (4: 16 worker warps, 8: 8), autotuned
  void* wt = nullptr;               // device operand tiles
  __nv_bfloat16* r = nullptr;       // inner residual
  __nv_bfloat16* q = nullptr;       // K p
  __nv_bfloat16* x = nullptr;       // staging of a plain sweep's input
  __nv_bfloat16* p[kDirBufs] = {};  // rotating directions
  bool tma = false;                 // halo tiles by TMA (else cp.async pieces)
  CUtensorMap tm_r, tm_x, tm_p[kDirBufs];
};

struct TmgState;  // tensor multigrid preconditioner (tmg.cu)

}  // namespace tca

struct tca_plan_s {
  int d = 0;
  int prec = TCA_F32;
  int64_t n[tca::kMaxModes] = {1, 1, 1, 1};
  int64_t m[tca::kMaxModes] = {1, 1, 1, 1};
  int64_t N = 0, M = 0;
  double lambda = 0.0;
  tca::Mode mode[tca::kMaxModes];
  int order_fwd[tca::kMaxModes];  // mode order for apply (shrinking first, expanding last)
  int order_bwd[tca::kMaxModes];  // mode order for apply_T
  bool all_band = true;
  bool fused_ok = false;          // fused normal-operator sweep applies to this shape
  int fused_nchunks = 0;          // autotuned chunk count along mode 1 (0: wave model)
  int fused_model_nchunks = 0;    // chunk count the last fused launch used
  float ws_g4[8 * 7] = {};        // n4 = 8 plans: G_4 and lambda L_4 bands (host copies, [i4][tap])
  float ws_l4[8 * 5] = {};

  int64_t ws_elems = 0;           // capacity of each ping-pong buffer (elements)
  void* ws[2] = {nullptr, nullptr};
  double* ws64[2] = {nullptr, nullptr};  // FP64 ping-pong for the true residual
  int64_t ws64_elems = 0;

  // Solver vectors (element type of the plan), allocated on first solve.
  void* rhs = nullptr;
  void* r = nullptr;
  void* p[tca::kDirBufs] = {};
  void* q = nullptr;
  double* rhs64 = nullptr;
  double* res64 = nullptr;
  float* dbuf = nullptr;    // refinement correction d (mixed-precision plans)
  // Separable-inverse preconditioner: per-mode dense (G_k + s lambda L_k)^-1,
  // built for shift pc_shift (0: not built); z = M^-1 r.
  tca::ModeOp pc[tca::kMaxModes];
  double pc_shift = 0.0;
  uint64_t pc_generation = 0;  // bumped whenever the factors are rebuilt (graph cache keys)
  void* z = nullptr;
  bool pc_on = false;       // the iteration being built or run is preconditioned
  int pc_kind = 0;          // TCA_PRECOND_SEPARABLE(_BANDED) or TCA_PRECOND_JACOBI while pc_on
  // Banded separable preconditioner: 7-band truncations of (G_k + s lambda L_k)^-1,
  // for shift pcb_shift (0: not built); applied by the fused sweep (pcb_fused) or
  // as band mode products (pcb).
  tca::ModeOp pcb[tca::kMaxModes];
  tca::FusedBands pcb_fused;
  float* pcb_zero = nullptr;  // zero 5-bands
  double pcb_shift = 0.0;
  double pc_model_shift = 0.0;  // corner-model shift of the separable preconditioners (0: not yet formed)
  void* pc_dinv = nullptr;  // Jacobi: 1 / diag(K), n-shaped, element type of the plan (built on first use)
  tca::TmgState* tmg = nullptr;  // tensor multigrid cycle: transfers, vectors, smoother interval
  void* stage_x = nullptr;  // host-pointer staging (n-shaped)
  void* stage_b = nullptr;  // host-pointer staging (m-shaped)
  cudaStream_t copy_stream = nullptr;  // host-pointer solves: b uploaded under A^T b, x copied back
  cudaEvent_t copy_ev = nullptr;       // under the true residual
  cudaEvent_t chunk_ev[8] = {};

  tca::Bf16State bf;             // TCA_BF16_IR plans
  // Scattered samples (tca_plan_scattered): sample rows grouped by the tile
  // of the unknown grid that holds their window's anchor cell; M = sc_m.
  bool scattered = false;
  int64_t sc_m = 0;
  int32_t* sc_col0 = nullptr;        // [k][s]
  double* sc_w = nullptr;            // [k][s][4] (every scattered plan: FP64 operators and true residual)
  float* sc_w32 = nullptr;           // [k][s][4] (TCA_F32 plans)
  int32_t* sc_perm = nullptr;        // grouped position -> caller's sample index
  int32_t* sc_tile_start = nullptr;  // [tiles + 1]: first grouped sample of each tile
  double* sc_tmp = nullptr;          // sample-space vector of the normal operator (m doubles)
  int sc_ts[tca::kMaxModes] = {};    // tile extent per mode (anchor cells)
  int sc_nt[tca::kMaxModes] = {};    // tiles per mode
  int64_t sc_tiles = 0;
  int64_t sc_region = 0;             // largest shared-memory region of a tile (elements)
  tca::Scalars* scal = nullptr;  // device
  tca::Scalars* scal_host = nullptr;  // pinned mirror
  tca::Reduce red;

  // Cached CUDA graph of `graph_iters` CG iterations for one x buffer.
  cudaGraphExec_t graph_exec = nullptr;
  const void* graph_x = nullptr;
  int graph_iters = 0;
  bool graph_profiled = false;
  int graph_pc = 0;  // preconditioner kind the cached graph was built with (0: none)
  uint64_t graph_launches = 0;       // kernels per pass of the iteration graph
  uint64_t graph_head_launches = 0;  // kernels before its loop (unprofiled graphs)
  cudaEvent_t sweep_ev[2 * tca::kMaxProfiledIters] = {};  // start/end per iteration of a profiled graph

  int num_sms = 0;
  uint64_t generation = 0;  // unique per plan created in this process (cache keys)
};

namespace tca {

// ---- error plumbing -------------------------------------------------------
void set_cuda_error(cudaError_t e);
void set_error_message(const char* msg);
void note_launches(uint64_t count);

#define TCA_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) {                                 \
      ::tca::set_cuda_error(_e);                             \
      return TCA_ERR_CUDA;                                   \
    }                                                        \
  } while (0)

#define TCA_TRY(expr)                                        \
  do {                                                       \
    tca_status _s = (expr);                                  \
    if (_s != TCA_OK) return _s;                             \
  } while (0)

#define TCA_LAUNCH_CHECK()                                   \
  do {                                                       \
    ::tca::note_launches(1);                                 \
    cudaError_t _e = cudaGetLastError();                     \
    if (_e != cudaSuccess) {                                 \
      ::tca::set_cuda_error(_e);                             \
      return TCA_ERR_CUDA;                                   \
    }                                                        \
  } while (0)

inline size_t elem_size(const tca_plan_s* p) { return p->prec == TCA_F64 ? 8 : 4; }

// ---- launchers implemented in the .cu files --------------------------------
// Mode product y = x x_k op over a tensor viewed as (O, n_in, I) -> (O, n_out, I).
template <typename Tin, typename Tout, typename Tc>
tca_status launch_mode_op(const ModeOp& op, const Tin* x, Tout* y, int64_t O, int64_t I,
                          cudaStream_t s);

// y (+)= lambda * sum_k (x x_k L_k) over the 4D view dims[4]; accumulate adds into y.
template <typename Tin, typename Tout>
tca_status launch_reg_add(const tca_plan_s* p, const Tin* x, Tout* y, const int64_t* dims,
                          cudaStream_t s);

// Reduction target of a fused <x, Kx> -> alpha (CG sweep through the generic sequence).
struct RegDot {
  Scalars* sc;
  Reduce red;
};

// Separable-inverse preconditioner for shift s: build (or keep) the per-mode
// factors and the z buffer; apply_precond writes z = M^-1 r (element type T).
tca_status ensure_precond(tca_plan_s* p, double shift);
// The separable preconditioners' default shift: the corner model of the
// spectrum of M^-1 K (formed on the host once per plan).
tca_status precond_model_shift(tca_plan_s* p, double* shift);
// Point-Jacobi preconditioner: build (once) 1 / diag(K) and the z buffer.
tca_status ensure_jacobi(tca_plan_s* p);
// Banded separable preconditioner for shift s: build (or keep) the 7-band
// truncated inverses and the z buffer.
tca_status ensure_precond_banded(tca_plan_s* p, double shift);
template <typename T>
tca_status apply_precond(tca_plan_s* p, const T* r, T* z, cudaStream_t s);
// The banded separable preconditioner and rho1 = <r, z> with the PCG scalars in
// one fused sweep (init: a fresh start); TCA_ERR_UNSUPPORTED where the fused
// sweep cannot do both (the caller applies M^-1 and forms the dot apart).
tca_status apply_precond_dot(tca_plan_s* p, const float* r, float* z, bool init, cudaStream_t s);
// Largest 3xTF32 / TF32 split the tensor-core dense kernel takes for an
// n_out x n_in factor (2, 1, or 0 when it takes none).
int dense_tc_max_split(int64_t n_in, int64_t n_out);

// Normal operator through the generic (unfused) sequence, element type T; with
// dot, <x, y> and alpha = rho / <x, y> are formed in the same pass.
template <typename T>
tca_status normal_generic(tca_plan_s* p, const T* x, T* y, cudaStream_t s, const RegDot* dot = nullptr);

// FP64 normal operator applied to a float or double x (true residual).
template <typename Tin>
tca_status normal_fp64(tca_plan_s* p, const Tin* x, double* y, cudaStream_t s);

// Chained apply / apply_T with device pointers.
template <typename Tin, typename Tout, typename Tc>
tca_status apply_chain(tca_plan_s* p, bool transpose, const Tin* x, Tout* y, void* const* ws,
                       int64_t ws_elems, cudaStream_t s);

// Fused FP32 sweep (fused_ok): optionally p_new = r + beta p_old, q = K p_new,
// <p_new, q> reduced to alpha.  pdot (plain sweep, n4 = 8 only): also
// rho1 = <p_old, q> and the PCG scalars (1: a fresh start, 2: an update), the
// sweep then being the preconditioner z = M^-1 r.  Returns
// TCA_ERR_UNSUPPORTED if not applicable.
tca_status normal_fused_f32(tca_plan_s* p, const float* r, const float* p_old, float* p_new,
                            float* q, bool cg_mode, cudaStream_t s, const FusedBands* bands = nullptr,
                            const Scalars* stop = nullptr, int pdot = 0);

// Blocks used by grid-stride vector kernels.
int vector_grid(const tca_plan_s* p, int64_t n);

// Double-float (FP32 pair) arithmetic for FP64-accurate products (residual_ff.cu).
tca_status split_ff(const double* a, float2* b, int64_t n, cudaStream_t s);
tca_status chain_ff(tca_plan_s* p, bool transpose, bool gram, const float* x, float2* y, float* y32,
                    float2* const* ws, int64_t ws_elems, cudaStream_t s);
tca_status chain_ff_rhs_from_host(tca_plan_s* p, const float* b_host, float* b_stage, float2* y, float* y32,
                                  float2* const* ws, int64_t ws_elems, cudaStream_t s, cudaStream_t cs,
                                  cudaEvent_t* ev, int chunks);
tca_status residual_ff(tca_plan_s* p, const float* x, const float2* rhs_ff, float2* kx_ff, float* r_out,
                       Reduce red, Reduce red2, cudaStream_t s);

// TMA-staged / register-fibre banded mode products (mode_tma.cu); UNSUPPORTED
// when the shape or alignment does not fit, so callers fall back.
tca_status launch_band_fast(const Band& band, const float* x, float* y, int64_t O, int64_t I, cudaStream_t s,
                            int sm_cap = 0);
int rows_per_chunk(const int32_t* start_host, int64_t n_out, int W);
// Dense mode product on tcgen05 tensor cores (dense_tc.cu); split 1 = TF32, 2 = 3xTF32.
tca_status launch_dense_tc(const Dense& d, const float* x, float* y, int64_t O, int64_t I, int split,
                           cudaStream_t s, int sm_cap = 0, const Scalars* stop = nullptr);
// Device address of the wait-timeout flag (for kernels in other translation units).
int* wait_timeout_flag();
// Synchronise s; TCA_ERR_TIMEOUT (and clear the flag) if a bounded wait gave up.
tca_status check_wait_timeout(cudaStream_t s);
// Tiled FP32 tensor map (no swizzle, zero fill out of bounds): dims innermost
// first, strides in bytes for dims 1 .. rank-1.  False if the driver rejects it
// (alignment) or the encoder is unavailable.
bool encode_tmap_f32(CUtensorMap* map, const void* base, int rank, const uint64_t* dims, const uint64_t* strides,
                     const uint32_t* box);

// Tiled tensor map of any element type (no swizzle, zero fill out of bounds).
bool encode_tmap(CUtensorMap* map, CUtensorMapDataType dtype, const void* base, int rank, const uint64_t* dims,
                 const uint64_t* strides, const uint32_t* box);

// bfloat16 tensor-core normal operator and inner-CG kernels (normal_bf16.cu).
bool bf16_shape_ok(const tca_plan_s* p);
tca_status bf16_prepare(tca_plan_s* p);
void bf16_release(tca_plan_s* p);
tca_status bf16_sweep(tca_plan_s* p, int pold_idx, __nv_bfloat16* pnew, __nv_bfloat16* q, cudaStream_t s);
tca_status normal_bf16(tca_plan_s* p, const float* x, float* y, cudaStream_t s);
tca_status bf16_start(tca_plan_s* p, const float* src, Reduce red, cudaStream_t s);
tca_status bf16_update(tca_plan_s* p, float* d, int pos, Reduce red, cudaStream_t s);
tca_status bf16_flush(tca_plan_s* p, float* d, Reduce red, cudaStream_t s);

// Solver buffers and scalars set so that a CG-mode sweep runs in full outside
// a solve (the autotuner times the sweep that solves run).
tca_status prepare_sweep_timing(tca_plan_s* p, cudaStream_t s);

// Scattered samples (scattered.cu): y = A x (gather) and x = A^T y (scatter-add,
// x zeroed first); perm: y in the caller's sample order.  T = double on every
// scattered plan, T = float on TCA_F32 plans.
template <typename T>
tca_status scattered_gather(const tca_plan_s* p, const T* x, T* y, bool perm, cudaStream_t s);
template <typename T>
tca_status scattered_scatter(const tca_plan_s* p, const T* y, T* x, bool perm, cudaStream_t s);
void scattered_release(tca_plan_s* p);

// Tensor multigrid preconditioner (tmg.cu): set up (or keep) the cycle for the
// options' tmg_* fields; z = V r (returns at once when the CG stop flags of
// p->scal are set and skip_if_done); free the state with the plan.
tca_status tmg_setup(tca_plan_s* p, const tca_solve_opts* o, cudaStream_t s);
template <typename T>
tca_status tmg_cycle(tca_plan_s* p, const T* r, T* z, bool skip_if_done, cudaStream_t s);
void tmg_reset_count(tca_plan_s* p);
void tmg_release(tca_plan_s* p);

bool is_device_ptr(const void* ptr);
tca_status ensure_stage(tca_plan_s* p);
tca_status ensure_ws64_public(tca_plan_s* p);

}  // namespace tca

// ---- device helpers --------------------------------------------------------
namespace tca {
namespace dev {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide FP64 sum; result valid in thread 0.  `sh` needs blockDim/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Last-block-finishes grid reduction.  Every block calls it with its partial;
// the block that arrives last sums all partials in a fixed order and returns
// true in thread 0 with the total in *total.  Deterministic for a fixed grid.
// am_last: one int of shared memory for the block's verdict.
__device__ __forceinline__ bool grid_sum_last_at(double v, Reduce red, double* total, double* sh,
                                                 volatile int* am_last_flag) {
  volatile int& am_last = *am_last_flag;
  const double bs = block_sum(v, sh);
  if (threadIdx.x == 0) {
    red.partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned int t = atomicAdd(red.ticket, 1u);
    am_last = (t == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += ((volatile double*)red.partials)[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    *total = s;
    *red.ticket = 0u;
  }
  return threadIdx.x == 0;
}

__device__ __forceinline__ bool grid_sum_last(double v, Reduce red, double* total, double* sh) {
  __shared__ int am_last;
  return grid_sum_last_at(v, red, total, sh, &am_last);
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<double>(double v) { return (float)v; }

}  // namespace dev
}  // namespace tca
