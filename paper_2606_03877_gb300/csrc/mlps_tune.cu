// mlps_tune.cu -- autotuner of the batched render: picks the screen-tile edge of the binning and
// intersection stages (16 or 8 pixels) and the samples per CTA of the forward tensor-core MLP
// (2 to 5 chunks of 128 sample rows in flight, 6 with E4M3) by timing every candidate on the caller's own
// batch with CUDA events. Decisions are cached per batch shape (MLP shape, precision, samples,
// and every item's primitive count and resolution) for the life of the process.
//
// The tuner synchronises the stream it times on, so it must run outside stream capture; the
// tuned configuration is then used for the captured calls.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mlps.h"

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;  // key -> (tile, mlp_groups)

std::string tune_key(const mlps_config* c, const mlps_batch_item* items, int n, int do_backward) {
  std::string k;
  const int32_t head[] = {c->xyz_freqs, c->dir_freqs, c->hidden_width, c->hidden_layers, c->feat_dim,
                          c->samples, c->precision, c->max_hits_per_ray, c->contact, c->slot_dim, c->tile_sort,
                          do_backward};
  k.append(reinterpret_cast<const char*>(head), sizeof(head));
  for (int i = 0; i < n; ++i) {
    const int32_t it[] = {items[i].prim_count, items[i].cam.width, items[i].cam.height};
    k.append(reinterpret_cast<const char*>(it), sizeof(it));
  }
  return k;
}

struct Args {
  const mlps_scene* scene;
  const mlps_batch_item* items;
  int n, do_backward;
  const float* d_rgb;
  float *rgb, *trans, *feat;
  void* saved;
  size_t saved_bytes;
  void* scratch;
  size_t scratch_bytes;
  float *d_weights, *d_centers, *d_scales, *d_quats;
  void* stream;
};

mlps_status run_once(const mlps_config* c, const Args& a) {
  mlps_status s = mlps_render_batch_forward(c, a.scene, a.items, a.n, a.rgb, a.trans, a.feat, a.saved,
                                            a.saved_bytes, a.scratch, a.scratch_bytes, a.stream);
  if (s != MLPS_OK || !a.do_backward) return s;
  return mlps_render_batch_backward(c, a.scene, a.items, a.n, a.d_rgb, nullptr, nullptr, a.saved,
                                    a.saved_bytes, a.d_weights, a.d_centers, a.d_scales, a.d_quats,
                                    a.scratch, a.scratch_bytes, a.stream);
}

// Mean milliseconds per forward(+backward) of candidate `c`, or a negative value if the candidate
// does not run (unsupported, workspace too small, or a device error).
float time_candidate(const mlps_config* c, const Args& a, int reps) {
  size_t sb = 0, tb = 0;
  if (mlps_batch_workspace_size(c, a.scene->K, a.items, a.n, &sb, &tb) != MLPS_OK) return -1.f;
  if (sb > a.saved_bytes || tb > a.scratch_bytes) return -2.f;
  cudaStream_t st = static_cast<cudaStream_t>(a.stream);
  if (run_once(c, a) != MLPS_OK) return -1.f;  // warm-up (kernel attributes, caches)
  if (mlps_read_status(a.saved, a.stream) != MLPS_OK) return -3.f;
  if (a.do_backward && mlps_read_status(a.scratch, a.stream) != MLPS_OK) return -3.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -4.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -4.f;
  }
  float ms = -4.f;
  bool ok = cudaEventRecord(e0, st) == cudaSuccess;
  for (int r = 0; r < reps && ok; ++r) ok = run_once(c, a) == MLPS_OK;
  ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
  if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms /= (float)reps;
  else ms = -4.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace

extern "C" mlps_status mlps_autotune_batch(
    const mlps_config* cfg, const mlps_scene* scene, const mlps_batch_item* items, int32_t n_items,
    int32_t do_backward, const float* d_rgb, float* rgb, float* trans, float* feat, void* saved,
    size_t saved_bytes, void* scratch, size_t scratch_bytes, float* d_weights, float* d_centers,
    float* d_scales, float* d_quats, int32_t reps, mlps_config* tuned, float* best_ms,
    int32_t* n_candidates, int32_t* cand_tile, int32_t* cand_groups, float* cand_ms, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (!scene || !items || n_items < 1 || !tuned || reps < 1 || (do_backward && !d_rgb))
    return MLPS_ERR_INVALID_ARGUMENT;
  const std::string key = tune_key(cfg, items, n_items, do_backward);
  if (n_candidates) *n_candidates = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *tuned = *cfg;
      tuned->tile = it->second.first;
      tuned->mlp_groups = it->second.second;
      if (best_ms) *best_ms = 0.f;  // cached decision: nothing timed
      return MLPS_OK;
    }
  }
  const Args a{scene, items, n_items, do_backward, d_rgb, rgb, trans, feat, saved, saved_bytes,
               scratch, scratch_bytes, d_weights, d_centers, d_scales, d_quats, stream};
  const bool tc = cfg->precision == MLPS_BF16 || cfg->precision == MLPS_FP8_E4M3;
  std::vector<int> groups = {0};
  if (tc && cfg->hidden_width == 64 && cfg->feat_dim == 0)
    groups = cfg->precision == MLPS_FP8_E4M3 ? std::vector<int>{6, 5, 4, 3, 2} : std::vector<int>{5, 4, 3, 2};
  float best = -1.f;
  int best_tile = cfg->tile, best_groups = cfg->mlp_groups, nc = 0;
  // with the tile-centre order the tile edge is part of the result, not a schedule: keep it
  const std::vector<int> tiles = cfg->tile_sort ? std::vector<int>{cfg->tile} : std::vector<int>{16, 8};
  for (int tile : tiles) {
    for (int g : groups) {
      mlps_config c = *cfg;
      c.tile = tile;
      c.mlp_groups = g;
      if (mlps_check_config(&c) != MLPS_OK) continue;
      const float ms = time_candidate(&c, a, reps);
      if (nc < 16) {
        if (cand_tile) cand_tile[nc] = tile;
        if (cand_groups) cand_groups[nc] = g;
        if (cand_ms) cand_ms[nc] = ms;
      }
      ++nc;
      if (ms > 0.f && (best < 0.f || ms < best)) {
        best = ms;
        best_tile = tile;
        best_groups = g;
      }
    }
  }
  if (n_candidates) *n_candidates = nc < 16 ? nc : 16;
  if (best < 0.f) return MLPS_ERR_UNSUPPORTED;  // no candidate ran
  *tuned = *cfg;
  tuned->tile = best_tile;
  tuned->mlp_groups = best_groups;
  if (best_ms) *best_ms = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best_tile, best_groups};
  return MLPS_OK;
}

extern "C" void mlps_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}
