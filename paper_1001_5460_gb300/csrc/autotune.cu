// Autotuner for the fused normal-operator sweep: picks the tile extent along
// mode 1 (how many chunks of planes the CTAs split mode 1 into) by timing
// candidates on the device, around the choice of the wave/halo cost model.
// Results are cached per (n1, n2, n3, n4) for the life of the process.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tca_internal.cuh"

namespace tca {
namespace {

std::mutex g_tune_mutex;
std::map<std::tuple<int64_t, int64_t, int64_t, int64_t>, int> g_tune_cache;

}  // namespace
}  // namespace tca

using namespace tca;

extern "C" tca_status tca_autotune(tca_plan_t plan, cudaStream_t s) {
  if (!plan) return TCA_ERR_INVALID_ARG;
  tca_plan_s* p = plan;
  if (!p->fused_ok || p->prec == TCA_F64) return TCA_OK;  // nothing to tune
  const auto key = std::make_tuple(p->n[0], p->n[1], p->n[2], p->d == 4 ? p->n[3] : (int64_t)1);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      p->fused_nchunks = it->second;
      return TCA_OK;
    }
  }
  float* x = (float*)p->ws[0];
  float* y = (float*)p->ws[1];
  TCA_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)p->N, s));
  p->fused_nchunks = 0;
  TCA_TRY(normal_fused_f32(p, nullptr, x, nullptr, y, false, s));
  const int model = std::max(1, p->fused_model_nchunks);
  std::vector<int> cand = {model, model / 2, model * 2, (model * 3) / 2, model * 3, 1, 2, 4};
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  cudaEvent_t e0, e1;
  TCA_CUDA_TRY(cudaEventCreate(&e0));
  TCA_CUDA_TRY(cudaEventCreate(&e1));
  int best = model;
  float best_ms = 1e30f;
  tca_status st = TCA_OK;
  for (int nc : cand) {
    if (nc < 1 || nc > p->n[0]) continue;
    p->fused_nchunks = nc;
    st = normal_fused_f32(p, nullptr, x, nullptr, y, false, s);  // warm-up (and validity of the shape)
    if (st != TCA_OK) break;
    if (cudaEventRecord(e0, s) != cudaSuccess) break;
    for (int r = 0; r < 5 && st == TCA_OK; ++r) st = normal_fused_f32(p, nullptr, x, nullptr, y, false, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = nc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->fused_nchunks = best;
  if (st != TCA_OK) return st;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = best;
  return TCA_OK;
}

extern "C" int tca_autotuned_chunks(tca_plan_t plan) { return plan ? plan->fused_nchunks : 0; }
