// mlps_common.cuh -- device-side types and helpers shared by the MLP-Splatting kernels.
//
// Double-float ("double-word") arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, giving ~44 significant bits from FP32 instructions only.
// The algorithms are the published error-free transformations: TwoSum (Knuth, TAOCP vol. 2),
// Fast2Sum (Dekker 1971), TwoProd through one FMA, and the double-word operations of Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44(2), 2017 (AccurateDWPlusDW, DWTimesFP3, DWTimesDW3, DWDivDW2) and
// the one-Newton-step square root of the same paper's Sec. 7 (SQRTDWtoDW). Every step uses an
// explicitly rounded intrinsic so that the compiler cannot contract or reassociate it.
//
// The ray-ellipsoid hit test runs in this arithmetic: its decision (m^2 < 1) and the contact
// point must agree with an FP64 evaluation on every ray not within ~1e-6 of tangency, which
// plain FP32 cannot do (the normalised offset o' reaches |o'| ~ 60 at these scenes, so one FP32
// rounding moves m^2 by ~1e-5).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mlps.h"

#define MLPS_DEV __device__ __forceinline__
#define MLPS_HD __host__ __device__ __forceinline__

namespace mlps {

constexpr int kMaxHits = 64;       // per-ray sorted-hit capacity limit
constexpr int kMaxLayers = 8;      // hidden_layers + 1
constexpr int kMaxFeat = 32;
constexpr int kMaxSlotDim = 2048;  // feature-slot channels (Sec. 3.4)
constexpr int kMaxViews = MLPS_MAX_VIEWS;
constexpr int kLiveBlock = 1024;  // chunks per block of the live-chunk compaction

// ------------------------------------------------------------------------------------------
// Device status word: first error wins.
MLPS_DEV void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// ------------------------------------------------------------------------------------------
// Double-float arithmetic
struct dfl {
  float hi, lo;
};

MLPS_DEV dfl df_make(float a) { return {a, 0.0f}; }

MLPS_DEV dfl two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

MLPS_DEV dfl fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

MLPS_DEV dfl two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

MLPS_DEV dfl df_add(dfl x, dfl y) {  // AccurateDWPlusDW
  dfl s = two_sum(x.hi, y.hi);
  dfl t = two_sum(x.lo, y.lo);
  float c = __fadd_rn(s.lo, t.hi);
  dfl v = fast_two_sum(s.hi, c);
  float w = __fadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}

MLPS_DEV dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
MLPS_DEV dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }

MLPS_DEV dfl df_mulf(dfl x, float y) {  // DWTimesFP3
  dfl c = two_prod(x.hi, y);
  float cl3 = __fmaf_rn(x.lo, y, c.lo);
  return fast_two_sum(c.hi, cl3);
}

MLPS_DEV dfl df_mul(dfl x, dfl y) {  // DWTimesDW3
  dfl c = two_prod(x.hi, y.hi);
  float tl0 = __fmul_rn(x.lo, y.lo);
  float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  float cl3 = __fadd_rn(c.lo, cl2);
  return fast_two_sum(c.hi, cl3);
}

MLPS_DEV dfl df_div(dfl x, dfl y) {  // DWDivDW2
  float th = __fdiv_rn(x.hi, y.hi);
  dfl r = df_mulf(y, th);
  dfl pi = two_sum(x.hi, -r.hi);
  float dl = __fsub_rn(x.lo, r.lo);
  float d = __fadd_rn(pi.lo, dl);
  float tl = __fdiv_rn(__fadd_rn(pi.hi, d), y.hi);
  return fast_two_sum(th, tl);
}

MLPS_DEV dfl df_sqrt(dfl x) {  // one Newton step on the FP32 square root
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  float s = __fsqrt_rn(x.hi);
  dfl p = two_prod(s, s);
  float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
  float c = __fdiv_rn(r, __fmul_rn(2.0f, s));
  return fast_two_sum(s, c);
}

MLPS_DEV float df_to_f(dfl x) { return __fadd_rn(x.hi, x.lo); }

MLPS_DEV dfl df_dot3(const dfl* a, const dfl* b) {
  return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}

// ------------------------------------------------------------------------------------------
// Per-view and per-primitive data computed once per call

// Camera of one view (host-computed; the origin is split into hi + lo of its FP64 value).
// One view of a render call. In a batch every view (item) renders its own primitive range of
// the scene arrays at its own resolution; a single-scene call has prim_base 0 and prim_n K.
struct ViewData {
  float R[9];       // world -> camera rotation block, row-major
  float t[3];
  float fx, fy, cx, cy;
  float near_t;
  float o_hi[3], o_lo[3];  // ray origin -R^T t
  int width, height;
  int ray_base;            // first global ray (pixel) of this view
  int prim_base, prim_n;   // the view's primitives [prim_base, prim_base + prim_n)
  int pv_base;             // first (view, primitive) record of this view in pview
  int ntx, nty;            // its screen tiles
  int tile_base;           // first tile of this view in tile_count
  int pad;
  long long cand_base;     // first candidate slot of this view in tile_list (tiles x prim_n)
};

struct ViewArray {
  ViewData v[kMaxViews];
};

// View-independent primitive geometry. M = S^-1 R(q/|q|)^T in double-float.
struct PrimGeo {
  float Mhi[9], Mlo[9];
  float R[9];       // R(qn), FP32 (backward)
  float qn[4];
  float qlen;
  float mu[3];
  float s[3];
  int valid;        // finite, s > 0, |q| > 0
};

// Per (view, primitive): o' = M (o - mu) in double-float and the conservative tile rectangle.
struct PrimView {
  float op_hi[3], op_lo[3];
  int tx0, ty0, tx1, ty1;  // inclusive tile range; tx0 > tx1 = empty
};

// Unit ray direction of pixel (x, y) in double-float (the hit test's precision).
// Unit direction of the ray through the image point (u, v) (pixel x spans [x, x + 1)).
MLPS_DEV void ray_dir_df_uv(const ViewData& V, float u, float v, dfl d[3]) {
  float nx = __fsub_rn(u, V.cx);
  float ny = __fsub_rn(v, V.cy);
  dfl dc0 = df_div(df_make(nx), df_make(V.fx));
  dfl dc1 = df_div(df_make(ny), df_make(V.fy));
  // R^T dc: component i = R[0][i] dc0 + R[1][i] dc1 + R[2][i] * 1
  dfl n2 = {0.f, 0.f};
  for (int i = 0; i < 3; ++i) {
    dfl a = df_add(df_mulf(dc0, V.R[i]), df_mulf(dc1, V.R[3 + i]));
    d[i] = df_add(a, df_make(V.R[6 + i]));
    n2 = df_add(n2, df_mul(d[i], d[i]));
  }
  dfl n = df_sqrt(n2);
  for (int i = 0; i < 3; ++i) d[i] = df_div(d[i], n);
}

MLPS_DEV void ray_dir_df(const ViewData& V, int x, int y, dfl d[3]) {
  // x + 0.5 is exact in FP32 (half-integers, |.| < 2^22)
  ray_dir_df_uv(V, __fadd_rn((float)x, 0.5f), __fadd_rn((float)y, 0.5f), d);
}

// Unit ray direction in plain FP32 (inputs of the MLP; smooth, so FP32 suffices).
MLPS_DEV void ray_dir_f(const ViewData& V, int x, int y, float d[3]) {
  float dc0 = ((float)x + 0.5f - V.cx) / V.fx;
  float dc1 = ((float)y + 0.5f - V.cy) / V.fy;
  float n2 = 0.f;
  for (int i = 0; i < 3; ++i) {
    d[i] = V.R[i] * dc0 + V.R[3 + i] * dc1 + V.R[6 + i];
    n2 += d[i] * d[i];
  }
  float inv = rsqrtf(n2);
  for (int i = 0; i < 3; ++i) d[i] *= inv;
}

// One hit interval as the MLP stage consumes it (64 bytes, written in primitive order by the
// gather stage so that a chunk's intervals are one contiguous block).
struct IntervalRec {
  int h;            // hit record index
  float p[3];       // closest point o' + t_mid d' (normalised frame)
  float r0, r1;     // t0 - t_mid, t1 - t_mid
  float dt;         // sample step Delta = (t1 - t0) / S (world units)
  float tmid;       // t_mid
  float dp[3];      // d' = M d
  float d[3];       // unit world ray direction
  float pad[2];
};
static_assert(sizeof(IntervalRec) == 64, "interval record is 64 bytes");

// ------------------------------------------------------------------------------------------
// Model shape (derived from mlps_config)
struct Model {
  int nin;          // encoded input width
  int nout;         // 4 + F
  int width;        // hidden width
  int nl;           // layers = hidden_layers + 1
  int S;            // samples per interval
  int F;            // feature outputs
  int xyzL, dirL;   // encoding frequencies
  int contact;      // 1: contact-point input gamma([d; delta]), S = 1 (Sec. 3.2)
  int C;            // slot-embedding dimension (Sec. 3.4); 0 = no feature slots
  int P;            // canonical MLP params per primitive
  int Prow;         // canonical params per primitive: the MLP's, then 4 slot embeddings of C
  int din[kMaxLayers], dout[kMaxLayers];
  int woff[kMaxLayers], boff[kMaxLayers];
};

MLPS_HD int model_input_dim(int xyzL, int dirL) {
  return (xyzL > 0 ? 6 * xyzL : 3) + (dirL > 0 ? 6 * dirL : 0);
}

// ------------------------------------------------------------------------------------------
// All device pointers and sizes of one call (passed by value to every kernel).
struct Work {
  // saved region
  int* saved_hdr;        // [0] status, [1] hit records used, [2] total MLP chunks
  int* hit_prim;
  int* hit_ray;
  float* hit_tmid;       // contact point t* (Eq. 2, before max(0, .)), world units
  float* hit_r0;         // t0 - t_mid
  float* hit_r1;         // t1 - t_mid
  float* hit_p;          // [3, cap] closest point p = o' + t_mid d' (normalised frame)
  float4* hit_out;       // interval partial composite (C_rgb, a = sum sigma Delta)
  float* hit_feat;       // [cap, F] interval partial feature composite
  int* ray_start;
  int* ray_count;
  int* prim_count;       // [K]
  int* prim_start;       // [K + 1]
  int* chunk_start;      // [K + 1]
  int* prim_list;        // [cap] hit ids grouped by primitive
  IntervalRec* rec;      // [cap] interval records in the same (primitive-major) order
  int* slot_of;          // [cap] hit index -> position in that order
  ViewData* views;       // [V]
  PrimGeo* geo;          // [K]
  PrimView* pview;       // [n_pairs]: per view, its primitives in order
  // scratch region
  int* scr_hdr;          // [0] status
  int* prim_cursor;      // [K]
  int* tile_count;       // [n_tiles_all]: per view, its tiles in row-major order
  int* tile_list;        // per view and tile, prim_n candidate slots (global primitive ids)
  float4* hit_grad;      // [cap] (dL/dC_j, dL/da_j) per interval, in primitive-major order
  float* hit_gfeat;      // [cap, F], same order
  float* dgeo;           // [K, 12] dL/dM (9) and dL/dmu (3)
  float* slot_ga;        // [cap] feature slots: dL/da_j of each interval (hit order)
  float4* slot_gu;       // [cap] feature slots: (dL/du, compositing weight w_j) (hit order)
  float* dwb;            // [n_sm, P] width-128 backward: per-block weight-gradient copies
  // Interval lists that select some intervals of the primitive-major order (launch_live_lists):
  // the backward's (the intervals with a nonzero gradient) and, with depth waves, the forward's
  // (a wave's intervals). An MLP kernel walking such lists gets a Work whose prim_count /
  // prim_start / chunk_start are the lists' and whose bslot maps a list position to the
  // interval's position in the primitive-major order (null: every interval, identity).
  const int* bslot;      // [hit_cap]
  int* live_slot;        // [hit_cap] storage of bslot
  int* live_bcount;      // [hit_cap / kLiveBlock + 2] per-block live counts, then their offsets
  int* live_prim_count;  // [K + 1]
  int* live_prim_start;  // [K + 1]
  int* live_chunk_start; // [K + 1]
  unsigned char* ray_alive;  // [n_rays] depth waves: the ray is still open after the first wave
  // sizes
  int K, V;
  int H, W, ntx, nty, n_tiles;  // view 0's sizes (the single-scene inspection calls use them)
  int tile;
  int tile_sort;         // 1: hits ordered by the tile-centre virtual ray (Sec. 3.3)
  int n_pairs;           // sum over views of prim_n
  int max_view_tiles;    // largest tile count of a view (grid size of the per-tile kernels)
  int n_tiles_all;       // tiles of all views
  int n_rays;
  int hit_cap;
  int max_hits;
  int ipc;               // intervals per MLP chunk
  int S;                 // samples per interval
  float t_eps;
};

// Chunks an MLP kernel walks (interval lists: count in scratch header word 1).
MLPS_DEV int walk_chunk_count(const Work& w) { return w.bslot ? w.scr_hdr[1] : w.saved_hdr[2]; }
// The map from list positions to forward positions, or null when it is the identity (no lists,
// or every interval is live: the lists are then the forward's).
MLPS_DEV const int* walk_map(const Work& w) {
  return (w.bslot && w.scr_hdr[2] != min(w.saved_hdr[1], w.hit_cap)) ? w.bslot : nullptr;
}
MLPS_DEV int walk_slot(const int* map, int j) { return map ? map[j] : j; }

// Rays of all views together (views are stored in ray order). With a device-resident item
// table the ray arrays are sized for the caps and the live total can be smaller.
MLPS_DEV int live_rays(const Work& w) {
  const ViewData& V = w.views[w.V - 1];
  return V.ray_base + V.width * V.height;
}

// View of a global ray (views are stored in ray order; at most kMaxViews, binary search).
MLPS_DEV int view_of_ray(const Work& w, int ray) {
  int lo = 0, hi = w.V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.views[mid].ray_base <= ray) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace mlps
