// mlps_api.cu -- the C ABI of include/mlps.h: validation, workspace carving and the stage
// sequence of the forward and backward passes.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

using namespace mlps;

namespace {

// ------------------------------------------------------------------------------------------
// Profiler (host-side, optional)

struct ProfRec {
  int stage;
  cudaEvent_t a, b;
};
const char* kStageNames[] = {"setup", "tile_lists", "intersect", "prim_scan", "scatter",
                             "mlp_fwd", "composite_fwd", "composite_bwd", "mlp_bwd", "pose_bwd",
                             "pack", "slots_fwd", "slots_bwd", "loss", "adam"};
constexpr int kNumStages = sizeof(kStageNames) / sizeof(kStageNames[0]);
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_prof_pool;
float g_prof_ms[kNumStages];
int g_prof_cnt[kNumStages];

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// A stage: an NVTX range for external profilers (a no-op without one attached) and, when the
// library's profiler is on, a pair of CUDA events on the stream.
struct StageTimer {
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageTimer(int s, cudaStream_t stream) : stage(s), st(stream) {
    nvtxRangePushA(kStageNames[s]);
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    a = prof_event();
    cudaEventRecord(a, st);
  }
  ~StageTimer() {
    nvtxRangePop();
    if (!a) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t b = prof_event();
    cudaEventRecord(b, st);
    g_prof_pending.push_back({stage, a, b});
  }
};

std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

enum { ST_SETUP, ST_TILES, ST_INTERSECT, ST_SCAN, ST_SCATTER, ST_MLP_FWD, ST_COMP_FWD,
       ST_COMP_BWD, ST_MLP_BWD, ST_POSE_BWD, ST_PACK, ST_SLOTS_FWD, ST_SLOTS_BWD, ST_LOSS, ST_ADAM };

// ------------------------------------------------------------------------------------------
// Model and packing layouts

bool finite_f(float x) { return std::isfinite(x); }

// Bytes of a packed blob that the MLP kernels read (the slot embeddings follow them).
size_t mlp_bytes(const Model& m, const Packed& pk) {
  return (size_t)(m.C > 0 ? pk.slot_byte : pk.stride);
}

mlps_status check_cfg(const mlps_config* c) {
  if (!c) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->xyz_freqs < 0 || c->xyz_freqs > 16 || c->dir_freqs < 0 || c->dir_freqs > 16)
    return MLPS_ERR_INVALID_ARGUMENT;
  if (c->hidden_layers < 1 || c->hidden_layers > kMaxLayers - 1) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->feat_dim < 0 || c->feat_dim > kMaxFeat) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->samples < 1 || c->samples > 128) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->max_hits_per_ray < 1 || c->max_hits_per_ray > kMaxHits) return MLPS_ERR_INVALID_ARGUMENT;
  if (!finite_f(c->hit_capacity_per_ray) || !(c->hit_capacity_per_ray > 0.f))
    return MLPS_ERR_INVALID_ARGUMENT;
  if (!finite_f(c->t_eps) || c->t_eps < 0.f || c->t_eps >= 1.f) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->early_stop_wave < 0 || c->early_stop_wave > c->max_hits_per_ray) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->early_stop_wave > 0 && c->slot_dim > 0) return MLPS_ERR_UNSUPPORTED;
  if (c->tile_sort != 0 && c->tile_sort != 1) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->contact != 0 && (c->contact != 1 || c->samples != 1)) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->slot_dim < 0 || c->slot_dim > kMaxSlotDim) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->slot_dim % 4 != 0) return MLPS_ERR_UNSUPPORTED;  // float4 channel groups
  if (c->mlp_groups != 0 && (c->mlp_groups < 2 || c->mlp_groups > 6)) return MLPS_ERR_INVALID_ARGUMENT;
  if (c->hidden_width != 32 && c->hidden_width != 64 && c->hidden_width != 128)
    return MLPS_ERR_UNSUPPORTED;
  if (c->tile != 16 && c->tile != 8) return MLPS_ERR_UNSUPPORTED;
  if (c->precision != MLPS_FP32 && c->precision != MLPS_BF16 && c->precision != MLPS_FP8_E4M3)
    return MLPS_ERR_INVALID_ARGUMENT;
  if (model_input_dim(c->xyz_freqs, c->dir_freqs) > 128) return MLPS_ERR_UNSUPPORTED;
  return MLPS_OK;
}

// The tensor-core kernels are built for hidden widths 64 and 128. A 32-wide model (the paper's
// 72-32-32-4) runs on them with its hidden layers zero-padded to 64 units: the extra units have
// zero weights and bias, so their ReLU output is 0 and they change no result. The packer reads
// the canonical (32-wide) weights and writes the padded tiles; the kernels see the padded shape.
}  // namespace

Model mlps::tc_model(const Model& m) {
  if (m.width != 32) return m;
  Model t = m;
  t.width = 64;
  for (int l = 0; l < m.nl; ++l) {
    t.din[l] = l == 0 ? m.nin : 64;
    t.dout[l] = l == m.nl - 1 ? m.nout : 64;
  }
  return t;
}

namespace {

Model make_model(const mlps_config* c) {
  Model m;
  std::memset(&m, 0, sizeof(m));
  m.nin = model_input_dim(c->xyz_freqs, c->dir_freqs);
  m.nout = 4 + c->feat_dim;
  m.width = c->hidden_width;
  m.nl = c->hidden_layers + 1;
  m.S = c->samples;
  m.F = c->feat_dim;
  m.xyzL = c->xyz_freqs;
  m.dirL = c->dir_freqs;
  m.contact = c->contact;
  m.C = c->slot_dim;
  int off = 0;
  for (int l = 0; l < m.nl; ++l) {
    m.din[l] = l == 0 ? m.nin : m.width;
    m.dout[l] = l == m.nl - 1 ? m.nout : m.width;
    m.woff[l] = off;
    off += m.din[l] * m.dout[l];
    m.boff[l] = off;
    off += m.dout[l];
  }
  m.P = off;
  m.Prow = off + 4 * m.C;
  return m;
}

int r4(int x) { return (x + 3) & ~3; }
long long r256(long long x) { return (x + 255) & ~255LL; }

Packed make_packed(const mlps_config* c, const Model& m) {
  Packed pk;
  std::memset(&pk, 0, sizeof(pk));
  pk.precision = c->precision;
  if (c->precision == MLPS_BF16 || c->precision == MLPS_FP8_E4M3) {
    TcPlan P;
    long long stride = 0;
    if (tc_plan(tc_model(m), &P, &stride, c->precision == MLPS_FP8_E4M3)) {
      pk.stride = stride;
      pk.slot_byte = P.slot_byte;
    }
    return pk;
  }
  int off = 0;
  for (int l = 0; l < m.nl; ++l) {
    pk.woff[l] = off;
    off = r4(off + m.din[l] * m.dout[l]);
    pk.boff[l] = off;
    off = r4(off + m.dout[l]);
  }
  pk.slot_byte = (long long)off * 4;  // FP32 slot embeddings [4][C] after the layers
  off += 4 * m.C;
  pk.stride = r256((long long)off * 4);
  return pk;
}

// ------------------------------------------------------------------------------------------
// Workspace layout

struct Carve {
  size_t off = 256;  // header first
  template <typename T>
  size_t take(size_t count) {
    size_t o = off;
    off += (count * sizeof(T) + 255) & ~size_t(255);
    return o;
  }
};

// One view of a call: its camera and the primitives it renders (a single-scene call gives every
// view the whole scene; a batch gives each item its own range, at its own resolution).
struct ViewSpec {
  mlps_camera cam;
  int prim_base, prim_n;
};

struct Layout {
  // saved
  size_t hit_prim, hit_ray, hit_tmid, hit_r0, hit_r1, hit_p, hit_out, hit_feat, ray_start,
      ray_count, prim_count, prim_start, chunk_start, prim_list, rec, slot_of, views, geo, pview,
      saved_total;
  // scratch
  size_t prim_cursor, tile_count, tile_list, hit_grad, hit_gfeat, dgeo, slot_ga, slot_gu, dwb, live_slot,
      live_bcount, live_prim_count, live_prim_start, live_chunk_start, ray_alive, scratch_total;
  long long hit_cap;
  long long n_rays, n_pairs, n_tiles_all, n_cand;
  int max_view_tiles;
  int H0, W0, ntx0, nty0;  // view 0
};

bool make_layout(const mlps_config* c, int K, const ViewSpec* vs, int V, Layout* L) {
  const int F = c->feat_dim;
  L->n_rays = L->n_pairs = L->n_tiles_all = L->n_cand = 0;
  L->max_view_tiles = 0;
  for (int v = 0; v < V; ++v) {
    const long long ntx = (vs[v].cam.width + c->tile - 1) / c->tile;
    const long long nty = (vs[v].cam.height + c->tile - 1) / c->tile;
    L->n_rays += (long long)vs[v].cam.width * vs[v].cam.height;
    L->n_pairs += vs[v].prim_n;
    L->n_tiles_all += ntx * nty;
    L->n_cand += ntx * nty * vs[v].prim_n;
    L->max_view_tiles = std::max(L->max_view_tiles, (int)(ntx * nty));
  }
  L->W0 = vs[0].cam.width;
  L->H0 = vs[0].cam.height;
  L->ntx0 = (L->W0 + c->tile - 1) / c->tile;
  L->nty0 = (L->H0 + c->tile - 1) / c->tile;
  if (L->n_rays > 0x7fffffffLL || L->n_pairs > 0x7fffffffLL) return false;
  double cap = std::ceil((double)L->n_rays * (double)c->hit_capacity_per_ray);
  if (cap < 1) cap = 1;
  if (cap > 0x7fff0000) return false;
  L->hit_cap = (long long)cap;
  const size_t hc = (size_t)L->hit_cap, nr = (size_t)L->n_rays;
  Carve s;
  L->hit_prim = s.take<int>(hc);
  L->hit_ray = s.take<int>(hc);
  L->hit_tmid = s.take<float>(hc);
  L->hit_r0 = s.take<float>(hc);
  L->hit_r1 = s.take<float>(hc);
  L->hit_p = s.take<float>(3 * hc);
  L->hit_out = s.take<float4>(hc);
  L->hit_feat = s.take<float>(hc * (size_t)(F > 0 ? F : 1));
  L->ray_start = s.take<int>(nr ? nr : 1);
  L->ray_count = s.take<int>(nr ? nr : 1);
  L->prim_count = s.take<int>((size_t)K + 1);
  L->prim_start = s.take<int>((size_t)K + 1);
  L->chunk_start = s.take<int>((size_t)K + 1);
  L->prim_list = s.take<int>(hc);
  L->rec = s.take<IntervalRec>(hc);
  L->slot_of = s.take<int>(hc);
  L->views = s.take<ViewData>((size_t)V);
  L->geo = s.take<PrimGeo>((size_t)K + 1);
  L->pview = s.take<PrimView>((size_t)L->n_pairs + 1);
  L->saved_total = s.off;
  Carve t;
  L->prim_cursor = t.take<int>((size_t)K + 1);
  L->tile_count = t.take<int>((size_t)L->n_tiles_all + 1);
  L->tile_list = t.take<int>((size_t)L->n_cand + 1);
  L->hit_grad = t.take<float4>(hc);
  L->hit_gfeat = t.take<float>(hc * (size_t)(F > 0 ? F : 1));
  L->dgeo = t.take<float>((size_t)K * 12 + 1);
  L->slot_ga = t.take<float>(c->slot_dim > 0 ? hc : 1);
  L->slot_gu = t.take<float4>(c->slot_dim > 0 ? hc : 1);
  {  // the wide backward's block-private weight gradients: one FP32 copy per SM
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
    const Model mm = make_model(c);
    L->dwb = t.take<float>(c->hidden_width == 128 ? (size_t)n_sm * mm.P : 1);
  }
  // the MLP backward's interval lists (live intervals only)
  L->live_slot = t.take<int>(hc);
  L->live_bcount = t.take<int>(hc / kLiveBlock + 2);
  L->live_prim_count = t.take<int>((size_t)K + 1);
  L->live_prim_start = t.take<int>((size_t)K + 1);
  L->live_chunk_start = t.take<int>((size_t)K + 1);
  L->ray_alive = t.take<unsigned char>(c->early_stop_wave > 0 ? nr + 1 : 1);
  L->scratch_total = t.off;
  return true;
}

Work make_work(const mlps_config* c, const Layout& L, int K, int V, void* saved, void* scratch) {
  Work w;
  std::memset(&w, 0, sizeof(w));
  char* sv = static_cast<char*>(saved);
  char* sc = static_cast<char*>(scratch);
  w.saved_hdr = reinterpret_cast<int*>(sv);
  w.hit_prim = reinterpret_cast<int*>(sv + L.hit_prim);
  w.hit_ray = reinterpret_cast<int*>(sv + L.hit_ray);
  w.hit_tmid = reinterpret_cast<float*>(sv + L.hit_tmid);
  w.hit_r0 = reinterpret_cast<float*>(sv + L.hit_r0);
  w.hit_r1 = reinterpret_cast<float*>(sv + L.hit_r1);
  w.hit_p = reinterpret_cast<float*>(sv + L.hit_p);
  w.hit_out = reinterpret_cast<float4*>(sv + L.hit_out);
  w.hit_feat = reinterpret_cast<float*>(sv + L.hit_feat);
  w.ray_start = reinterpret_cast<int*>(sv + L.ray_start);
  w.ray_count = reinterpret_cast<int*>(sv + L.ray_count);
  w.prim_count = reinterpret_cast<int*>(sv + L.prim_count);
  w.prim_start = reinterpret_cast<int*>(sv + L.prim_start);
  w.chunk_start = reinterpret_cast<int*>(sv + L.chunk_start);
  w.prim_list = reinterpret_cast<int*>(sv + L.prim_list);
  w.rec = reinterpret_cast<IntervalRec*>(sv + L.rec);
  w.slot_of = reinterpret_cast<int*>(sv + L.slot_of);
  w.views = reinterpret_cast<ViewData*>(sv + L.views);
  w.geo = reinterpret_cast<PrimGeo*>(sv + L.geo);
  w.pview = reinterpret_cast<PrimView*>(sv + L.pview);
  if (sc) {
    w.scr_hdr = reinterpret_cast<int*>(sc);
    w.prim_cursor = reinterpret_cast<int*>(sc + L.prim_cursor);
    w.tile_count = reinterpret_cast<int*>(sc + L.tile_count);
    w.tile_list = reinterpret_cast<int*>(sc + L.tile_list);
    w.hit_grad = reinterpret_cast<float4*>(sc + L.hit_grad);
    w.hit_gfeat = reinterpret_cast<float*>(sc + L.hit_gfeat);
    w.dgeo = reinterpret_cast<float*>(sc + L.dgeo);
    if (c->slot_dim > 0) {
      w.slot_ga = reinterpret_cast<float*>(sc + L.slot_ga);
      w.slot_gu = reinterpret_cast<float4*>(sc + L.slot_gu);
    }
    if (c->hidden_width == 128) w.dwb = reinterpret_cast<float*>(sc + L.dwb);
    w.live_slot = reinterpret_cast<int*>(sc + L.live_slot);
    w.live_bcount = reinterpret_cast<int*>(sc + L.live_bcount);
    w.live_prim_count = reinterpret_cast<int*>(sc + L.live_prim_count);
    w.live_prim_start = reinterpret_cast<int*>(sc + L.live_prim_start);
    w.live_chunk_start = reinterpret_cast<int*>(sc + L.live_chunk_start);
    w.ray_alive = reinterpret_cast<unsigned char*>(sc + L.ray_alive);
    // w.bslot stays null: only the MLP backward's copy of the Work points at the live lists
  }
  w.K = K;
  w.V = V;
  w.H = L.H0;
  w.W = L.W0;
  w.ntx = L.ntx0;
  w.nty = L.nty0;
  w.n_tiles = L.ntx0 * L.nty0;
  w.tile = c->tile;
  w.tile_sort = c->tile_sort;
  w.n_pairs = (int)L.n_pairs;
  w.max_view_tiles = L.max_view_tiles;
  w.n_tiles_all = (int)L.n_tiles_all;
  w.n_rays = (int)L.n_rays;
  w.hit_cap = (int)L.hit_cap;
  w.max_hits = c->max_hits_per_ray;
  w.ipc = (c->samples <= 128) ? 128 / c->samples : 1;
  w.S = c->samples;
  w.t_eps = c->t_eps;
  return w;
}

mlps_status check_cam(const mlps_camera& c) {
  if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return MLPS_ERR_INVALID_ARGUMENT;
  const float vals[5] = {c.fx, c.fy, c.cx, c.cy, c.near_t};
  for (float x : vals)
    if (!finite_f(x)) return MLPS_ERR_INVALID_ARGUMENT;
  for (float x : c.world_to_cam)
    if (!finite_f(x)) return MLPS_ERR_INVALID_ARGUMENT;
  if (c.fx == 0.f || c.fy == 0.f || c.near_t < 0.f) return MLPS_ERR_INVALID_ARGUMENT;
  return MLPS_OK;
}

// Single-scene call: every view renders all K primitives; all views share one resolution (the
// output arrays are [V, H, W, ...]).
mlps_status specs_from_cams(const mlps_camera* cams, int V, int K, std::vector<ViewSpec>* out) {
  if (!cams || V < 1 || V > kMaxViews || K < 0) return MLPS_ERR_INVALID_ARGUMENT;
  out->resize(V);
  for (int v = 0; v < V; ++v) {
    mlps_status s = check_cam(cams[v]);
    if (s != MLPS_OK) return s;
    if (cams[v].width != cams[0].width || cams[v].height != cams[0].height) return MLPS_ERR_UNSUPPORTED;
    (*out)[v] = ViewSpec{cams[v], 0, K};
  }
  return MLPS_OK;
}

// Batch: item i renders primitives [prim_offset, prim_offset + prim_count) of the scene arrays.
mlps_status specs_from_items(const mlps_batch_item* items, int n, int K, std::vector<ViewSpec>* out) {
  if (!items || n < 1 || n > kMaxViews || K < 0) return MLPS_ERR_INVALID_ARGUMENT;
  out->resize(n);
  for (int i = 0; i < n; ++i) {
    mlps_status s = check_cam(items[i].cam);
    if (s != MLPS_OK) return s;
    const long long b = items[i].prim_offset, c = items[i].prim_count;
    if (b < 0 || c < 0 || b + c > K) return MLPS_ERR_INVALID_ARGUMENT;
    (*out)[i] = ViewSpec{items[i].cam, (int)b, (int)c};
  }
  return MLPS_OK;
}

// Device item table of the *_dev batch calls: the layout is sized from the caps (every item at
// max_width x max_height with max_prim_count primitives); k_views_from_items reads the items.
struct DevTable {
  const mlps_batch_item* items;
  mlps_batch_caps caps;
};

mlps_status specs_from_caps(int n, const mlps_batch_caps* caps, int K, std::vector<ViewSpec>* out) {
  if (!caps || n < 1 || n > kMaxViews || K < 0) return MLPS_ERR_INVALID_ARGUMENT;
  if (caps->max_width < 1 || caps->max_height < 1 || caps->max_width > 16384 || caps->max_height > 16384 ||
      caps->max_prim_count < 0)
    return MLPS_ERR_INVALID_ARGUMENT;
  mlps_camera c;
  std::memset(&c, 0, sizeof(c));
  c.width = caps->max_width;
  c.height = caps->max_height;
  out->assign(n, ViewSpec{c, 0, std::min(caps->max_prim_count, K)});
  return MLPS_OK;
}

ViewArray make_views(const ViewSpec* vs, int V, int tile) {
  ViewArray va;
  std::memset(&va, 0, sizeof(va));
  int ray_base = 0, pv_base = 0, tile_base = 0;
  long long cand_base = 0;
  for (int v = 0; v < V; ++v) {
    const mlps_camera& c = vs[v].cam;
    ViewData& d = va.v[v];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) d.R[i * 3 + j] = c.world_to_cam[i * 4 + j];
      d.t[i] = c.world_to_cam[i * 4 + 3];
    }
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    d.near_t = c.near_t;
    d.width = c.width;
    d.height = c.height;
    d.ray_base = ray_base;
    d.prim_base = vs[v].prim_base;
    d.prim_n = vs[v].prim_n;
    d.pv_base = pv_base;
    d.ntx = (c.width + tile - 1) / tile;
    d.nty = (c.height + tile - 1) / tile;
    d.tile_base = tile_base;
    d.cand_base = cand_base;
    ray_base += c.width * c.height;
    pv_base += vs[v].prim_n;
    tile_base += d.ntx * d.nty;
    cand_base += (long long)d.ntx * d.nty * vs[v].prim_n;
    // (the ray origin is formed on the device: k_store_views)
  }
  return va;
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  return n;
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

mlps_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MLPS_OK : MLPS_ERR_CUDA; }

mlps_status workspace_impl(const mlps_config* cfg, int K, const std::vector<ViewSpec>& vs,
                           size_t* saved_bytes, size_t* scratch_bytes) {
  Layout L;
  if (!make_layout(cfg, K, vs.data(), (int)vs.size(), &L)) return MLPS_ERR_UNSUPPORTED;
  *saved_bytes = L.saved_total;
  *scratch_bytes = L.scratch_total;
  return MLPS_OK;
}

// Forward over views `vs` (validated cameras and primitive ranges).
mlps_status forward_impl(const mlps_config* cfg, const mlps_scene* scene, const std::vector<ViewSpec>& vs,
                         float* rgb, float* trans, float* feat, void* saved, size_t saved_bytes,
                         void* scratch, size_t scratch_bytes, void* stream, const DevTable* dev = nullptr) {
  if (!scene || scene->K < 0 || !rgb || !trans || !saved || !scratch)
    return MLPS_ERR_INVALID_ARGUMENT;
  if (cfg->feat_dim + cfg->slot_dim > 0 && !feat) return MLPS_ERR_INVALID_ARGUMENT;
  const int K = scene->K;
  if (K > 0 && (!scene->centers || !scene->scales || !scene->quats || !scene->weights))
    return MLPS_ERR_INVALID_ARGUMENT;
  if (!aligned256(saved) || !aligned256(scratch) || (K > 0 && !aligned256(scene->weights)))
    return MLPS_ERR_INVALID_ARGUMENT;
  const int n_views = (int)vs.size();
  Layout L;
  if (!make_layout(cfg, K, vs.data(), n_views, &L)) return MLPS_ERR_UNSUPPORTED;
  if (saved_bytes < L.saved_total || scratch_bytes < L.scratch_total)
    return MLPS_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Work w = make_work(cfg, L, K, n_views, saved, scratch);
  Model m = make_model(cfg);
  const bool tc_fwd = cfg->precision == MLPS_BF16 || cfg->precision == MLPS_FP8_E4M3;
  MlpArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = tc_fwd ? tc_model(m) : m;
  a.pk = make_packed(cfg, m);
  a.weights = static_cast<const unsigned char*>(scene->weights);
  a.rows = 128;
  a.groups = cfg->mlp_groups;
  a.resident = (mlp_bytes(m, a.pk) + 2 * 128 * 4 * (size_t)std::max(std::max(m.nin, m.width), m.nout) +
                16 * 1024) <= 200 * 1024;
  const int n_sm = num_sms();
  {
    StageTimer tm(ST_SETUP, st);
    cudaMemsetAsync(w.saved_hdr, 0, 256, st);
    cudaMemsetAsync(w.scr_hdr, 0, 256, st);  // both regions' status words start clear
    cudaMemsetAsync(w.prim_count, 0, sizeof(int) * ((size_t)K + 1), st);
    if (dev)
      launch_views_from_items(w, dev->items, dev->caps.max_width, dev->caps.max_height,
                              dev->caps.max_prim_count, st);
    else
      launch_store_views(w, make_views(vs.data(), n_views, cfg->tile), st);
    count_launch(1 + launch_prim_setup(w, scene->centers, scene->scales, scene->quats, st));
  }
  {
    StageTimer tm(ST_TILES, st);
    launch_tile_lists(w, st);
    count_launch(1);
  }
  {
    StageTimer tm(ST_INTERSECT, st);
    if (!launch_intersect(w, st)) return MLPS_ERR_UNSUPPORTED;
    count_launch(1);
  }
  {
    StageTimer tm(ST_SCAN, st);
    if (K > 0) { launch_prim_scan(w, st); count_launch(1); }
  }
  {
    StageTimer tm(ST_SCATTER, st);
    if (K > 0) { launch_scatter(w, n_sm, st); count_launch(1); }
  }
  if (K > 0) {
    StageTimer tm(ST_MLP_FWD, st);
    TcPlan P;
    const bool tc = cfg->precision == MLPS_BF16 || cfg->precision == MLPS_FP8_E4M3;
    if (tc) {
      long long stride;
      tc_plan(a.m, &P, &stride, cfg->precision == MLPS_FP8_E4M3);
    }
    auto mlp = [&](const Work& wk) -> mlps_status {
      const cudaError_t e = tc ? launch_mlp_fwd_tc(wk, a, P, n_sm, st) : launch_mlp_fwd_simt(wk, a, n_sm, st);
      if (e == cudaErrorNotSupported) return MLPS_ERR_UNSUPPORTED;
      if (e != cudaSuccess) return MLPS_ERR_CUDA;
      count_launch(1);
      return MLPS_OK;
    };
    const int k1 = cfg->early_stop_wave;
    if (k1 == 0) {
      const mlps_status ms = mlp(w);
      if (ms != MLPS_OK) return ms;
    } else {
      // depth waves (App. B.2): each ray's first k1 hits; then the later hits of the rays whose
      // composite does not stop within them. The intervals behind a termination point are not
      // evaluated; the composite below never reaches them.
      Work wv = w;
      wv.prim_count = w.live_prim_count;
      wv.prim_start = w.live_prim_start;
      wv.chunk_start = w.live_chunk_start;
      wv.bslot = w.live_slot;
      launch_live_lists(w, 0, 1, k1, st);
      count_launch(4);
      mlps_status ms = mlp(wv);
      if (ms != MLPS_OK) return ms;
      launch_wave_alive(w, k1, st);
      launch_live_lists(w, 0, 2, k1, st);
      count_launch(w.n_rays > 0 ? 5 : 4);
      ms = mlp(wv);
      if (ms != MLPS_OK) return ms;
    }
  }
  {
    StageTimer tm(ST_COMP_FWD, st);
    launch_composite_fwd(w, cfg->feat_dim, cfg->feat_dim + cfg->slot_dim, rgb, trans, feat, st);
    count_launch(w.n_rays > 0 ? 1 : 0);
  }
  if (m.C > 0) {
    StageTimer tm(ST_SLOTS_FWD, st);
    launch_slots_fwd(w, m, a.pk, a.weights, feat + cfg->feat_dim, cfg->feat_dim + m.C, st);
    count_launch(w.n_rays > 0 ? 1 : 0);
  }
  return cuda_status(cudaGetLastError());
}


// Backward over views `vs` (the same views as the forward call that filled `saved`).
mlps_status backward_impl(const mlps_config* cfg, const mlps_scene* scene, const std::vector<ViewSpec>& vs,
                          const float* d_rgb, const float* d_trans, const float* d_feat, const void* saved,
                          size_t saved_bytes, float* d_weights, float* d_centers, float* d_scales,
                          float* d_quats, void* scratch, size_t scratch_bytes, void* stream) {
  if (!scene || scene->K < 0 || !d_rgb || !saved || !scratch) return MLPS_ERR_INVALID_ARGUMENT;
  const int K = scene->K;
  if (K > 0 && (!scene->weights || !d_weights || !d_centers || !d_scales || !d_quats))
    return MLPS_ERR_INVALID_ARGUMENT;
  if (!aligned256(saved) || !aligned256(scratch)) return MLPS_ERR_INVALID_ARGUMENT;
  const int n_views = (int)vs.size();
  Layout L;
  if (!make_layout(cfg, K, vs.data(), n_views, &L)) return MLPS_ERR_UNSUPPORTED;
  if (saved_bytes < L.saved_total || scratch_bytes < L.scratch_total)
    return MLPS_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Work w = make_work(cfg, L, K, n_views, const_cast<void*>(saved), scratch);
  Model m = make_model(cfg);
  MlpArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = m;
  a.pk = make_packed(cfg, m);
  a.weights = static_cast<const unsigned char*>(scene->weights);
  a.d_weights = d_weights;
  a.rows = 128;
  a.resident = (mlp_bytes(m, a.pk) <= 64 * 1024);
  TcPlan P;
  long long tc_stride = 0;
  // FP8 precision: the backward recomputes the MLP in BF16 from the BF16 tiles of the same blob
  const bool tc = cfg->precision == MLPS_BF16 || cfg->precision == MLPS_FP8_E4M3;
  // width 128: the BF16 tensor-core wide backward (BF16 / E4M3 precisions), or the FP32 wide
  // backward reading the FP32 blob or the BF16 tiles
  const bool wide = m.width == 128;
  if (wide) {
    if (tc && !tc_plan(m, &P, &tc_stride, cfg->precision == MLPS_FP8_E4M3)) return MLPS_ERR_UNSUPPORTED;
    if (!simt_bwd_wide_supported(a) || !w.dwb) return MLPS_ERR_UNSUPPORTED;
  } else if (tc) {
    // the tensor-core backward: 64-wide models (32-wide ones padded to 64) with the midpoint
    // samples, or the paper's contact-point model
    const Model tm = tc_model(m);
    if (!tc_plan(tm, &P, &tc_stride, cfg->precision == MLPS_FP8_E4M3) || !tc_bwd_supported(tm, P))
      return MLPS_ERR_UNSUPPORTED;
  } else if (cfg->precision != MLPS_FP32 || !simt_bwd_supported(a)) {
    return MLPS_ERR_UNSUPPORTED;
  }
  const int n_sm = num_sms();
  {
    StageTimer tm(ST_COMP_BWD, st);
    cudaMemsetAsync(w.scr_hdr, 0, 256, st);
    if (K > 0) {
      cudaMemsetAsync(w.dgeo, 0, sizeof(float) * 12 * (size_t)K, st);
      cudaMemsetAsync(d_weights, 0, sizeof(float) * (size_t)m.Prow * K, st);
      if (wide) cudaMemsetAsync(w.dwb, 0, sizeof(float) * (size_t)m.P * n_sm, st);
    }
  }
  const int FT = cfg->feat_dim + m.C;  // feature row: the MLP's outputs, then the slot channels
  const bool slot_grad = m.C > 0 && d_feat != nullptr;
  if (slot_grad) {
    // the slot features' gradient on each interval's optical depth (read by the composite
    // reverse) and on u (read by the per-primitive pass after the MLP backward)
    StageTimer tm(ST_SLOTS_BWD, st);
    launch_slots_bwd_ray(w, m, a.pk, a.weights, d_feat + cfg->feat_dim, FT, st);
    count_launch(w.n_rays > 0 ? 1 : 0);
  }
  {
    StageTimer tm(ST_COMP_BWD, st);
    launch_composite_bwd(w, cfg->feat_dim, FT, d_rgb, d_trans, cfg->feat_dim > 0 ? d_feat : nullptr,
                         slot_grad ? w.slot_ga : nullptr, st);
    count_launch(w.n_rays > 0 ? 1 : 0);
  }
  // the MLP backward walks its own lists: the intervals with a nonzero gradient only
  Work wb = w;
  if (K > 0) {
    StageTimer tm(ST_COMP_BWD, st);
    launch_live_lists(w, cfg->feat_dim, 0, 0, st);
    count_launch(4);
    wb.prim_count = w.live_prim_count;
    wb.prim_start = w.live_prim_start;
    wb.chunk_start = w.live_chunk_start;
    wb.bslot = w.live_slot;
  }
  if (K > 0) {
    StageTimer tm(ST_MLP_BWD, st);
    // width 128: the tensor-core kernel for the tensor-core precisions where it applies, else
    // the wide FP32 kernel
    const bool wide_tc = wide && tc && tc_bwd_wide_supported(m, P);
    cudaError_t e = wide_tc ? launch_mlp_bwd_tc_wide(wb, a, P, n_sm, st)
                    : wide  ? launch_mlp_bwd_simt_wide(wb, a, tc ? &P : nullptr, n_sm, st)
                    : tc    ? launch_mlp_bwd_tc(wb, a, P, n_sm, st)
                            : launch_mlp_bwd_simt(wb, a, n_sm, st);
    if (e == cudaErrorNotSupported) return MLPS_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return MLPS_ERR_CUDA;
    count_launch(1);
  }
  if (slot_grad && K > 0) {
    StageTimer tm(ST_SLOTS_BWD, st);
    launch_slots_bwd_prim(w, m, a.pk, a.weights, d_feat + cfg->feat_dim, FT, d_weights, n_sm, st);
    count_launch(1);
  }
  {
    StageTimer tm(ST_POSE_BWD, st);
    launch_pose_bwd(w, d_centers, d_scales, d_quats, st);
    count_launch(K > 0 ? 1 : 0);
  }
  return cuda_status(cudaGetLastError());
}


}  // namespace

// ============================================================================================
extern "C" {

int32_t mlps_abi_version(void) { return MLPS_ABI_VERSION; }

const char* mlps_status_string(mlps_status s) {
  switch (s) {
    case MLPS_OK: return "ok";
    case MLPS_ERR_INVALID_ARGUMENT: return "invalid argument";
    case MLPS_ERR_UNSUPPORTED: return "unsupported configuration";
    case MLPS_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case MLPS_ERR_CAPACITY_OVERFLOW: return "hit capacity overflow";
    case MLPS_ERR_TIMEOUT: return "bounded wait timed out";
    case MLPS_ERR_NONFINITE: return "non-finite value";
    case MLPS_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

mlps_status mlps_config_default(mlps_config* cfg, int32_t xyz_freqs, int32_t dir_freqs,
                                int32_t hidden_width, int32_t hidden_layers, int32_t feat_dim) {
  if (!cfg) return MLPS_ERR_INVALID_ARGUMENT;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->xyz_freqs = xyz_freqs;
  cfg->dir_freqs = dir_freqs;
  cfg->hidden_width = hidden_width;
  cfg->hidden_layers = hidden_layers;
  cfg->feat_dim = feat_dim;
  cfg->samples = 32;
  cfg->precision = MLPS_FP32;
  cfg->max_hits_per_ray = 64;
  cfg->hit_capacity_per_ray = 8.0f;
  cfg->t_eps = 1e-6f;
  cfg->tile = 16;
  return MLPS_OK;
}

int32_t mlps_input_dim(const mlps_config* cfg) {
  if (!cfg) return 0;
  return model_input_dim(cfg->xyz_freqs, cfg->dir_freqs);
}

int64_t mlps_param_count(const mlps_config* cfg) {
  if (check_cfg(cfg) != MLPS_OK) return 0;
  return make_model(cfg).Prow;
}

int64_t mlps_weight_stride(const mlps_config* cfg) {
  if (check_cfg(cfg) != MLPS_OK) return 0;
  Model m = make_model(cfg);
  Packed pk = make_packed(cfg, m);
  return pk.stride;
}

mlps_status mlps_check_config(const mlps_config* cfg) {
  mlps_status s = check_cfg(cfg);
  if (s != MLPS_OK) return s;
  if (cfg->precision == MLPS_BF16 || cfg->precision == MLPS_FP8_E4M3) {
    TcPlan P;
    long long stride;
    const Model m = tc_model(make_model(cfg));
    if (!tc_plan(m, &P, &stride, cfg->precision == MLPS_FP8_E4M3)) return MLPS_ERR_UNSUPPORTED;
    if (tc_fwd_groups(m.width, m.F, cfg->mlp_groups, cfg->precision == MLPS_FP8_E4M3) == 0)
      return MLPS_ERR_UNSUPPORTED;
    if (tc_smem_bytes(P, cfg->feat_dim, cfg->mlp_groups, cfg->samples) > 227 * 1024) return MLPS_ERR_UNSUPPORTED;
    return MLPS_OK;
  }
  if (cfg->precision != MLPS_FP32) return MLPS_ERR_UNSUPPORTED;
  return MLPS_OK;
}

mlps_status mlps_pack_weights(const mlps_config* cfg, int32_t K, const float* weights_fp32,
                              void* packed, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (K < 0 || (K > 0 && (!weights_fp32 || !packed)) || (packed && !aligned256(packed)))
    return MLPS_ERR_INVALID_ARGUMENT;
  Model m = make_model(cfg);
  Packed pk = make_packed(cfg, m);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  StageTimer tm(ST_PACK, st);
  if (cfg->precision == MLPS_BF16 || cfg->precision == MLPS_FP8_E4M3) {
    TcPlan P;
    long long stride;
    tc_plan(tc_model(m), &P, &stride, cfg->precision == MLPS_FP8_E4M3);
    launch_pack_bf16(m, P, stride, K, weights_fp32, packed, st);  // canonical shape in, padded tiles out
    count_launch(K > 0 ? (cfg->precision == MLPS_FP8_E4M3 ? 2 : 1) : 0);
  } else {
    launch_pack_fp32(m, pk, K, weights_fp32, packed, st);
    count_launch(K > 0 ? 1 : 0);
  }
  return cuda_status(cudaGetLastError());
}

mlps_status mlps_workspace_size(const mlps_config* cfg, int32_t K, const mlps_camera* cams,
                                int32_t n_views, size_t* saved_bytes, size_t* scratch_bytes) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (K < 0 || !saved_bytes || !scratch_bytes) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_cams(cams, n_views, K, &vs);
  if (s != MLPS_OK) return s;
  return workspace_impl(cfg, K, vs, saved_bytes, scratch_bytes);
}

mlps_status mlps_batch_workspace_size(const mlps_config* cfg, int32_t K, const mlps_batch_item* items,
                                      int32_t n_items, size_t* saved_bytes, size_t* scratch_bytes) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (K < 0 || !saved_bytes || !scratch_bytes) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_items(items, n_items, K, &vs);
  if (s != MLPS_OK) return s;
  return workspace_impl(cfg, K, vs, saved_bytes, scratch_bytes);
}

mlps_status mlps_render_forward(const mlps_config* cfg, const mlps_scene* scene,
                                const mlps_camera* cams, int32_t n_views, float* rgb,
                                float* trans, float* feat, void* saved, size_t saved_bytes,
                                void* scratch, size_t scratch_bytes, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (!scene || scene->K < 0) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_cams(cams, n_views, scene->K, &vs);
  if (s != MLPS_OK) return s;
  return forward_impl(cfg, scene, vs, rgb, trans, feat, saved, saved_bytes, scratch, scratch_bytes, stream);
}

mlps_status mlps_render_batch_forward(const mlps_config* cfg, const mlps_scene* scene,
                                      const mlps_batch_item* items, int32_t n_items, float* rgb,
                                      float* trans, float* feat, void* saved, size_t saved_bytes,
                                      void* scratch, size_t scratch_bytes, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (!scene || scene->K < 0) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_items(items, n_items, scene->K, &vs);
  if (s != MLPS_OK) return s;
  return forward_impl(cfg, scene, vs, rgb, trans, feat, saved, saved_bytes, scratch, scratch_bytes, stream);
}

mlps_status mlps_render_backward(const mlps_config* cfg, const mlps_scene* scene,
                                 const mlps_camera* cams, int32_t n_views, const float* d_rgb,
                                 const float* d_trans, const float* d_feat, const void* saved,
                                 size_t saved_bytes, float* d_weights, float* d_centers,
                                 float* d_scales, float* d_quats, void* scratch,
                                 size_t scratch_bytes, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (!scene || scene->K < 0) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_cams(cams, n_views, scene->K, &vs);
  if (s != MLPS_OK) return s;
  return backward_impl(cfg, scene, vs, d_rgb, d_trans, d_feat, saved, saved_bytes, d_weights, d_centers,
                       d_scales, d_quats, scratch, scratch_bytes, stream);
}

mlps_status mlps_render_batch_backward(const mlps_config* cfg, const mlps_scene* scene,
                                       const mlps_batch_item* items, int32_t n_items, const float* d_rgb,
                                       const float* d_trans, const float* d_feat, const void* saved,
                                       size_t saved_bytes, float* d_weights, float* d_centers,
                                       float* d_scales, float* d_quats, void* scratch,
                                       size_t scratch_bytes, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (!scene || scene->K < 0) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_items(items, n_items, scene->K, &vs);
  if (s != MLPS_OK) return s;
  return backward_impl(cfg, scene, vs, d_rgb, d_trans, d_feat, saved, saved_bytes, d_weights, d_centers,
                       d_scales, d_quats, scratch, scratch_bytes, stream);
}

mlps_status mlps_batch_workspace_size_dev(const mlps_config* cfg, int32_t K, int32_t n_items,
                                          const mlps_batch_caps* caps, size_t* saved_bytes,
                                          size_t* scratch_bytes) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (K < 0 || !saved_bytes || !scratch_bytes) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_caps(n_items, caps, K, &vs);
  if (s != MLPS_OK) return s;
  return workspace_impl(cfg, K, vs, saved_bytes, scratch_bytes);
}

mlps_status mlps_render_batch_forward_dev(const mlps_config* cfg, const mlps_scene* scene,
                                          const mlps_batch_item* dev_items, int32_t n_items,
                                          const mlps_batch_caps* caps, float* rgb, float* trans,
                                          float* feat, void* saved, size_t saved_bytes, void* scratch,
                                          size_t scratch_bytes, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (!scene || scene->K < 0 || !dev_items) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_caps(n_items, caps, scene->K, &vs);
  if (s != MLPS_OK) return s;
  const DevTable dev{dev_items, *caps};
  return forward_impl(cfg, scene, vs, rgb, trans, feat, saved, saved_bytes, scratch, scratch_bytes, stream,
                      &dev);
}

mlps_status mlps_render_batch_backward_dev(const mlps_config* cfg, const mlps_scene* scene,
                                           const mlps_batch_item* dev_items, int32_t n_items,
                                           const mlps_batch_caps* caps, const float* d_rgb,
                                           const float* d_trans, const float* d_feat, const void* saved,
                                           size_t saved_bytes, float* d_weights, float* d_centers,
                                           float* d_scales, float* d_quats, void* scratch,
                                           size_t scratch_bytes, void* stream) {
  mlps_status s = mlps_check_config(cfg);
  if (s != MLPS_OK) return s;
  if (!scene || scene->K < 0 || !dev_items) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_caps(n_items, caps, scene->K, &vs);
  if (s != MLPS_OK) return s;
  // (the views the forward call stored in `saved` are reused)
  return backward_impl(cfg, scene, vs, d_rgb, d_trans, d_feat, saved, saved_bytes, d_weights, d_centers,
                       d_scales, d_quats, scratch, scratch_bytes, stream);
}

mlps_status mlps_read_status(const void* region, void* stream) {
  if (!region) return MLPS_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  if (cudaMemcpyAsync(&h, region, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MLPS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MLPS_ERR_CUDA;
  if (h != 0) {
    const int zero = 0;
    cudaMemcpyAsync(const_cast<void*>(region), &zero, sizeof(int), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  }
  return h;
}

mlps_status mlps_backward_chunk_counts(const void* saved, const void* scratch, int64_t* chunks,
                                       int64_t* live, void* stream) {
  if (!saved || !scratch || !chunks || !live) return MLPS_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h[3] = {0, 0, 0}, t[3] = {0, 0, 0};
  if (cudaMemcpyAsync(h, saved, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(t, scratch, sizeof(t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MLPS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MLPS_ERR_CUDA;
  *chunks = h[2];
  *live = t[1];
  return MLPS_OK;
}

mlps_status mlps_forward_wave_counts(const void* saved, const void* scratch, int64_t* intervals,
                                     int64_t* evaluated, void* stream) {
  if (!saved || !scratch || !intervals || !evaluated) return MLPS_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h[2] = {0, 0}, t[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(h, saved, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(t, scratch, sizeof(t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MLPS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MLPS_ERR_CUDA;
  *intervals = h[1];
  *evaluated = t[3];
  return MLPS_OK;
}

mlps_status mlps_saved_hit_count(const void* saved, int64_t* n_hits, void* stream) {
  if (!saved || !n_hits) return MLPS_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h[2] = {0, 0};
  if (cudaMemcpyAsync(h, saved, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MLPS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MLPS_ERR_CUDA;
  *n_hits = h[1];
  return MLPS_OK;
}

mlps_status mlps_export_hits(const mlps_config* cfg, const mlps_camera* cams, int32_t n_views,
                             const void* saved, int32_t max_out, int32_t* count, int32_t* prim,
                             float* t0, float* t1, float* tmid, void* stream) {
  mlps_status s = check_cfg(cfg);
  if (s != MLPS_OK) return s;
  if (!saved || max_out < 1 || !count || !prim || !t0 || !t1 || !tmid)
    return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  // K only shifts arrays after the ray arrays; the hit/ray arrays do not depend on it.
  s = specs_from_cams(cams, n_views, 0, &vs);
  if (s != MLPS_OK) return s;
  Layout L;
  if (!make_layout(cfg, 0, vs.data(), n_views, &L)) return MLPS_ERR_UNSUPPORTED;
  Work w = make_work(cfg, L, 0, n_views, const_cast<void*>(saved), nullptr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (w.n_rays > 0) launch_export_hits(w, max_out, count, prim, t0, t1, tmid, st);
  return cuda_status(cudaGetLastError());
}

mlps_status mlps_export_tiles(const mlps_config* cfg, int32_t K, const mlps_camera* cams,
                              int32_t n_views, const void* scratch, int32_t* count,
                              int32_t* list, void* stream) {
  mlps_status s = check_cfg(cfg);
  if (s != MLPS_OK) return s;
  if (!scratch || !count || !list || K < 1) return MLPS_ERR_INVALID_ARGUMENT;
  std::vector<ViewSpec> vs;
  s = specs_from_cams(cams, n_views, K, &vs);
  if (s != MLPS_OK) return s;
  Layout L;
  if (!make_layout(cfg, K, vs.data(), n_views, &L)) return MLPS_ERR_UNSUPPORTED;
  static char dummy_saved[256];
  Work w = make_work(cfg, L, K, n_views, dummy_saved, const_cast<void*>(scratch));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  launch_export_tiles(w, count, list, st);
  return cuda_status(cudaGetLastError());
}

int64_t mlps_kernel_launches(int32_t reset) {
  long long v = reset ? g_launches.exchange(0) : g_launches.load();
  return (int64_t)v;
}

void mlps_profiler_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
}

int32_t mlps_profiler_read(const char** names, float* ms, int32_t* counts, int32_t max,
                           int32_t reset) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (const ProfRec& r : g_prof_pending) {
    float t = 0.f;
    cudaEventSynchronize(r.b);
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      g_prof_ms[r.stage] += t;
      g_prof_cnt[r.stage] += 1;
    }
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_pending.clear();
  for (int i = 0; i < kNumStages && i < max; ++i) {
    if (names) names[i] = kStageNames[i];
    if (ms) ms[i] = g_prof_ms[i];
    if (counts) counts[i] = g_prof_cnt[i];
  }
  if (reset) {
    for (int i = 0; i < kNumStages; ++i) { g_prof_ms[i] = 0.f; g_prof_cnt[i] = 0; }
  }
  return kNumStages;
}


// ------------------------------------------------------------------------------------------
// Training objective and optimizer (Sec. 3.5, App. A.4)

static bool loss_desc_ok(const mlps_loss_desc* d) {
  return d && d->n_views >= 1 && d->height >= 1 && d->width >= 1 && d->height <= 16384 &&
         d->width <= 16384 && d->tile >= 1 && d->feat_dim >= 0 && std::isfinite(d->lambda_ssim) &&
         d->lambda_ssim >= 0.f && d->lambda_ssim <= 1.f;
}

size_t mlps_loss_workspace_size(const mlps_loss_desc* d) {
  if (!loss_desc_ok(d)) return 0;
  const size_t pix = (size_t)d->n_views * d->height * d->width;
  return 256 + ((9 * pix * sizeof(float) + 255) & ~size_t(255));
}

mlps_status mlps_loss(const mlps_loss_desc* d, const float* rgb, const float* rgb_target, const float* feat,
                      const float* feat_target, float* d_rgb, float* d_feat, float* loss_out, void* workspace,
                      size_t workspace_bytes, void* stream) {
  if (!loss_desc_ok(d) || !rgb || !rgb_target || !d_rgb || !loss_out || !workspace)
    return MLPS_ERR_INVALID_ARGUMENT;
  if (d->feat_dim > 0 && (!feat || !feat_target)) return MLPS_ERR_INVALID_ARGUMENT;
  if (!aligned256(workspace)) return MLPS_ERR_INVALID_ARGUMENT;
  if (workspace_bytes < mlps_loss_workspace_size(d)) return MLPS_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  StageTimer tm(ST_LOSS, st);
  launch_loss(d->n_views, d->height, d->width, rgb, rgb_target, d->tile_mask, d->tile, d->lambda_ssim,
              d->feat_dim, feat, feat_target, d_rgb, d_feat, reinterpret_cast<float*>(ws + 256),
              reinterpret_cast<double*>(ws), loss_out, st);
  count_launch(3 + (d->feat_dim > 0 ? 1 : 0));
  return cuda_status(cudaGetLastError());
}

mlps_status mlps_adam_step(const mlps_adam_group* groups, int32_t n_groups, float beta1, float beta2, float eps,
                           int32_t step, void* stream) {
  if (!groups || n_groups < 1 || n_groups > MLPS_MAX_ADAM_GROUPS || step < 1) return MLPS_ERR_INVALID_ARGUMENT;
  if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return MLPS_ERR_INVALID_ARGUMENT;
  AdamGroupDev g[MLPS_MAX_ADAM_GROUPS];
  for (int k = 0; k < n_groups; ++k) {
    const mlps_adam_group& a = groups[k];
    if (a.n < 0 || (a.n > 0 && (!a.param || !a.grad || !a.m || !a.v)) || (a.kind != 0 && a.kind != 1) ||
        (a.kind == 1 && a.n > 0 && !a.aux) || !std::isfinite(a.lr))
      return MLPS_ERR_INVALID_ARGUMENT;
    g[k] = {a.param, a.grad, a.m, a.v, a.aux, (long long)a.n, a.lr, a.kind};
  }
  StageTimer tm(ST_ADAM, static_cast<cudaStream_t>(stream));
  launch_adam(g, n_groups, beta1, beta2, eps, step, num_sms(), static_cast<cudaStream_t>(stream));
  count_launch(1);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
