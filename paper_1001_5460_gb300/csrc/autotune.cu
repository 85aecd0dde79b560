// Autotuner for the normal-operator sweep that CG solves run (the CG form:
// p = r + beta p_old, q = K p, <p, q>).  It times candidates on the device and
// keeps the fastest in the plan:
//   - FP32 fused sweep: the tile extent along mode 1 (how many chunks of planes
//     the CTAs split mode 1 into), around the wave/halo cost model's choice;
//   - bfloat16 tensor-core sweep (TCA_BF16_IR): the same chunk count and the
//     worker layout (4 core rows per thread with 16 worker warps, or 8 rows
//     with 8 warps).
// This is the plan-time choice of evaluation by cost (Sec. 2.1, Sec. 4
// expression analysis), made by measurement on this GPU.  Results are cached
// per (precision, n1, n2, n3, n4) for the life of the process.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tca_internal.cuh"

namespace tca {
namespace {

struct Choice {
  int nchunks = 0;
  int rpt = 0;
};

std::mutex g_tune_mutex;
std::map<std::tuple<int, int64_t, int64_t, int64_t, int64_t>, Choice> g_tune_cache;

// Mean device time of `reps` launches of fn (after one warm-up), or a negative
// value if a launch failed.
template <typename F>
float time_launches(F fn, int reps, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t s, tca_status* st) {
  *st = fn();
  if (*st != TCA_OK) return -1.f;
  if (cudaEventRecord(e0, s) != cudaSuccess) return -1.f;
  for (int r = 0; r < reps && *st == TCA_OK; ++r) *st = fn();
  if (*st != TCA_OK) return -1.f;
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / reps;
}

std::vector<int> chunk_candidates(int model, int64_t n1) {
  std::vector<int> cand = {model, model / 2, model * 2, (model * 3) / 2, (model * 2) / 3, model * 3, model + 1,
                           model - 1, 1, 2, 4};
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  cand.erase(std::remove_if(cand.begin(), cand.end(), [&](int c) { return c < 1 || c > n1; }), cand.end());
  return cand;
}

}  // namespace
}  // namespace tca

using namespace tca;

extern "C" tca_status tca_autotune(tca_plan_t plan, cudaStream_t s) {
  if (!plan) return TCA_ERR_INVALID_ARG;
  tca_plan_s* p = plan;
  const bool bf = p->prec == TCA_BF16_IR;
  if (p->prec == TCA_F64 || (!bf && !p->fused_ok)) return TCA_OK;  // nothing to tune
  const auto key = std::make_tuple(p->prec, p->n[0], p->n[1], p->n[2], p->d == 4 ? p->n[3] : (int64_t)1);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      if (bf) {
        p->bf.nchunks = it->second.nchunks;
        p->bf.rpt = it->second.rpt;
      } else {
        p->fused_nchunks = it->second.nchunks;
      }
      return TCA_OK;
    }
  }
  TCA_TRY(prepare_sweep_timing(p, s));
  cudaEvent_t e0, e1;
  TCA_CUDA_TRY(cudaEventCreate(&e0));
  TCA_CUDA_TRY(cudaEventCreate(&e1));
  Choice best;
  float best_ms = 1e30f;
  tca_status st = TCA_OK;
  if (bf) {
    for (int rpt : {4, 8}) {
      p->bf.rpt = rpt;
      p->bf.nchunks = 0;
      st = bf16_sweep(p, 0, p->bf.p[1], p->bf.q, s);
      if (st != TCA_OK) break;
      for (int nc : chunk_candidates(std::max(1, p->bf.model_nchunks), p->n[0])) {
        p->bf.nchunks = nc;
        const float ms = time_launches([&] { return bf16_sweep(p, 0, p->bf.p[1], p->bf.q, s); }, 5, e0, e1, s, &st);
        if (st != TCA_OK) break;
        if (ms >= 0.f && ms < best_ms) {
          best_ms = ms;
          best.nchunks = nc;
          best.rpt = rpt;
        }
      }
      if (st != TCA_OK) break;
    }
    if (best.rpt) {
      p->bf.nchunks = best.nchunks;
      p->bf.rpt = best.rpt;
    }
  } else {
    float* r = (float*)p->r;
    p->fused_nchunks = 0;
    st = normal_fused_f32(p, r, (const float*)p->p[0], (float*)p->p[1], (float*)p->q, true, s);
    if (st == TCA_OK) {
      for (int nc : chunk_candidates(std::max(1, p->fused_model_nchunks), p->n[0])) {
        p->fused_nchunks = nc;
        const float ms = time_launches(
            [&] { return normal_fused_f32(p, r, (const float*)p->p[0], (float*)p->p[1], (float*)p->q, true, s); }, 5,
            e0, e1, s, &st);
        if (st != TCA_OK) break;
        if (ms >= 0.f && ms < best_ms) {
          best_ms = ms;
          best.nchunks = nc;
        }
      }
    }
    p->fused_nchunks = best.nchunks;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // The sweeps above wrote the solver's directions and scalars; every solve
  // starts from its own set-up, and the iteration graph is rebuilt so that
  // its launches use the new choice.
  if (p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  if (st != TCA_OK) return st;
  TCA_TRY(check_wait_timeout(s));
  // A breakdown flag would mean the timed sweeps returned at entry: keep no choice.
  Scalars hs;
  TCA_CUDA_TRY(cudaMemcpy(&hs, p->scal, sizeof(Scalars), cudaMemcpyDeviceToHost));
  if (hs.breakdown || hs.converged) {
    p->fused_nchunks = 0;
    p->bf.nchunks = 0;
    set_error_message("tca_autotune: the timed sweeps did no work");
    return TCA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = best;
  return TCA_OK;
}

extern "C" int tca_autotuned_chunks(tca_plan_t plan) {
  if (!plan) return 0;
  return plan->prec == TCA_BF16_IR ? plan->bf.nchunks : plan->fused_nchunks;
}

extern "C" int tca_autotuned_rows(tca_plan_t plan) {
  return (plan && plan->prec == TCA_BF16_IR && plan->bf.nchunks > 0) ? plan->bf.rpt : 0;
}
