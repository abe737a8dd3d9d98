// k_geometry.cu -- primitive setup, 16x16 tile binning, ray-ellipsoid intersection with a
// per-ray depth sort, and the gather of hit intervals per primitive.
//
// Method steps (Sec. 3.2-3.3): every primitive is the unit-Mahalanobis ellipsoid of centre mu,
// scales s and rotation R(q/|q|). In its normalised frame o' = M (o - mu), d' = M d with
// M = S^-1 R^T. The soft contact point of Eq. 2 is t_mid = -(o'.d') / (d'.d'); the ray hits when
// m^2 = |o' + t_mid d'|^2 < 1 and the hit interval is [t_mid - h, t_mid + h],
// h = sqrt((1 - m^2) / (d'.d')), clipped below at the camera's near distance. Hits are ordered
// per ray by max(0, t_mid) (Eq. 2), ties by (t0, primitive index): the exact per-pixel order
// of Sec. 3.3. Primitives are binned into screen tiles with a conservative projected-support
// test (Sec. 3.3; the paper uses 8x8 tiles and an AABB test, here 16x16 tiles and the exact
// tangent-plane bounds of the ellipsoid, padded).
#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

namespace mlps {

// ------------------------------------------------------------------------------------------
// Views

// Ray origin -R^T t of a view record in double-float: each product R_ji t_j is exact as a float
// pair and their sum keeps ~48 bits (the hit test's precision).
MLPS_DEV void view_origin(ViewData& d) {
  for (int i = 0; i < 3; ++i) {
    dfl s = df_add(df_add(two_prod(d.R[i], d.t[0]), two_prod(d.R[3 + i], d.t[1])), two_prod(d.R[6 + i], d.t[2]));
    d.o_hi[i] = -s.hi;
    d.o_lo[i] = -s.lo;
  }
}

// Camera fields of a view record.
MLPS_DEV void view_camera(const mlps_camera& c, ViewData& d) {
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) d.R[i * 3 + j] = c.world_to_cam[i * 4 + j];
    d.t[i] = c.world_to_cam[i * 4 + 3];
  }
  d.fx = c.fx;
  d.fy = c.fy;
  d.cx = c.cx;
  d.cy = c.cy;
  d.near_t = c.near_t;
  d.width = c.width;
  d.height = c.height;
  view_origin(d);
}

// Host item table: bases and camera fields come in the launch parameters; the origin is formed
// here, as for a device table.
__global__ void k_store_views(Work w, ViewArray va) {
  int v = threadIdx.x;
  if (v < w.V) {
    ViewData d = va.v[v];
    view_origin(d);
    w.views[v] = d;
  }
}

// Device item table: each item checked against the caps and the scene (an invalid item becomes
// an empty view and raises MLPS_ERR_INVALID_ARGUMENT in the status word), then the bases of all
// views as running sums in item order (one thread: at most kMaxViews items).
__global__ void k_views_from_items(Work w, const mlps_batch_item* __restrict__ items, int max_w, int max_h,
                                   int max_p) {
  __shared__ ViewData sv[kMaxViews];
  const int v = threadIdx.x;
  if (v < w.V) {
    const mlps_batch_item it = items[v];
    const mlps_camera& c = it.cam;
    bool ok = c.width >= 1 && c.height >= 1 && c.width <= max_w && c.height <= max_h;
    ok = ok && it.prim_offset >= 0 && it.prim_count >= 0 && it.prim_count <= max_p &&
         (long long)it.prim_offset + it.prim_count <= (long long)w.K;
    float vals[17] = {c.fx, c.fy, c.cx, c.cy, c.near_t};
    for (int i = 0; i < 12; ++i) vals[5 + i] = c.world_to_cam[i];
    for (int i = 0; i < 17; ++i) ok = ok && isfinite(vals[i]);
    ok = ok && c.fx != 0.f && c.fy != 0.f && c.near_t >= 0.f;
    ViewData d;
    memset(&d, 0, sizeof(d));
    view_camera(c, d);
    if (ok) {
      d.prim_base = it.prim_offset;
      d.prim_n = it.prim_count;
      d.ntx = (d.width + w.tile - 1) / w.tile;
      d.nty = (d.height + w.tile - 1) / w.tile;
    } else {
      d.width = d.height = 0;
      d.prim_base = 0;
      d.prim_n = 0;
      d.ntx = d.nty = 0;
      set_status(w.saved_hdr, MLPS_ERR_INVALID_ARGUMENT);
    }
    sv[v] = d;
  }
  __syncthreads();
  if (v == 0) {
    int ray_base = 0, pv_base = 0, tile_base = 0;
    long long cand_base = 0;
    for (int i = 0; i < w.V; ++i) {
      ViewData& d = sv[i];
      d.ray_base = ray_base;
      d.pv_base = pv_base;
      d.tile_base = tile_base;
      d.cand_base = cand_base;
      ray_base += d.width * d.height;
      pv_base += d.prim_n;
      tile_base += d.ntx * d.nty;
      cand_base += (long long)d.ntx * d.nty * d.prim_n;
    }
  }
  __syncthreads();
  if (v < w.V) w.views[v] = sv[v];
}

// ------------------------------------------------------------------------------------------
// Primitive setup: M in double-float, o' per view, tile rectangles

MLPS_DEV bool finitef(float x) { return isfinite(x); }

__global__ void k_prim_geo(Work w, const float* __restrict__ centers,
                             const float* __restrict__ scales, const float* __restrict__ quats) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= w.K) return;
  PrimGeo g;
  float q[4], s[3], mu[3];
  bool ok = true;
  for (int i = 0; i < 4; ++i) { q[i] = quats[4 * p + i]; ok &= finitef(q[i]); }
  for (int i = 0; i < 3; ++i) {
    s[i] = scales[3 * p + i];
    mu[i] = centers[3 * p + i];
    ok &= finitef(s[i]) && finitef(mu[i]) && s[i] > 0.0f;
  }
  dfl n2 = {0.f, 0.f};
  for (int i = 0; i < 4; ++i) n2 = df_add(n2, two_prod(q[i], q[i]));
  ok &= n2.hi > 0.0f;
  dfl nrm = df_sqrt(n2);
  dfl qn[4];
  for (int i = 0; i < 4; ++i) qn[i] = ok ? df_div(df_make(q[i]), nrm) : df_make(i == 0 ? 1.f : 0.f);
  // R(qn): rotation matrix of a unit quaternion (w, x, y, z)
  dfl ww = qn[0], xx = qn[1], yy = qn[2], zz = qn[3];
  dfl one = df_make(1.0f);
  dfl x2 = df_mul(xx, xx), y2 = df_mul(yy, yy), z2 = df_mul(zz, zz);
  dfl xy = df_mul(xx, yy), xz = df_mul(xx, zz), yz = df_mul(yy, zz);
  dfl wx = df_mul(ww, xx), wy = df_mul(ww, yy), wz = df_mul(ww, zz);
  dfl R[9];
  R[0] = df_sub(one, df_mulf(df_add(y2, z2), 2.f));
  R[1] = df_mulf(df_sub(xy, wz), 2.f);
  R[2] = df_mulf(df_add(xz, wy), 2.f);
  R[3] = df_mulf(df_add(xy, wz), 2.f);
  R[4] = df_sub(one, df_mulf(df_add(x2, z2), 2.f));
  R[5] = df_mulf(df_sub(yz, wx), 2.f);
  R[6] = df_mulf(df_sub(xz, wy), 2.f);
  R[7] = df_mulf(df_add(yz, wx), 2.f);
  R[8] = df_sub(one, df_mulf(df_add(x2, y2), 2.f));
  dfl M[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i * 3 + j] = ok ? df_div(R[j * 3 + i], df_make(s[i])) : df_make(0.f);
  for (int i = 0; i < 9; ++i) { g.Mhi[i] = M[i].hi; g.Mlo[i] = M[i].lo; g.R[i] = df_to_f(R[i]); }
  for (int i = 0; i < 4; ++i) g.qn[i] = df_to_f(qn[i]);
  g.qlen = df_to_f(nrm);
  for (int i = 0; i < 3; ++i) { g.mu[i] = mu[i]; g.s[i] = s[i]; }
  g.valid = ok ? 1 : 0;
  w.geo[p] = g;
  if (!ok) set_status(w.saved_hdr, MLPS_ERR_NONFINITE);
}

// Per (view, primitive) record: o' = M (o - mu) in double-float and the conservative tile range.
__global__ void k_prim_view(Work w) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= w.n_pairs) return;
  int v = 0;
  {
    int lo = 0, hi = w.V - 1;  // the view whose record range holds j (views in pair order)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (w.views[mid].pv_base <= j) lo = mid;
      else hi = mid - 1;
    }
    v = lo;
  }
  const ViewData& V = w.views[v];
  if (j - V.pv_base >= V.prim_n) return;  // past the live total (device item table)
  const int p = V.prim_base + (j - V.pv_base);
  const PrimGeo& g = w.geo[p];
  const bool ok = g.valid != 0;
  float s[3], mu[3];
  dfl M[9];
  for (int i = 0; i < 3; ++i) { s[i] = g.s[i]; mu[i] = g.mu[i]; }
  for (int i = 0; i < 9; ++i) M[i] = {g.Mhi[i], g.Mlo[i]};
  {
    PrimView pv;
    // o' = M (o - mu) in double-float
    dfl rel[3];
    for (int i = 0; i < 3; ++i) rel[i] = df_sub({V.o_hi[i], V.o_lo[i]}, df_make(mu[i]));
    for (int i = 0; i < 3; ++i) {
      dfl a = df_add(df_add(df_mul(M[i * 3 + 0], rel[0]), df_mul(M[i * 3 + 1], rel[1])),
                     df_mul(M[i * 3 + 2], rel[2]));
      pv.op_hi[i] = a.hi;
      pv.op_lo[i] = a.lo;
    }
    // Conservative screen bounds. In camera coordinates the ellipsoid has centre c and
    // covariance-like matrix Sig = sum_i s_i^2 (Rc r_i)(Rc r_i)^T (r_i = column i of R(q)).
    // A plane X - m Z = 0 through the camera centre is tangent when
    // (c_x - m c_z)^2 = Sig_xx - 2 m Sig_xz + m^2 Sig_zz; the two roots m bound the image
    // column u = cx + fx m. The same in y.
    float c[3], cols[3][3];
    for (int i = 0; i < 3; ++i)
      c[i] = V.R[i * 3] * mu[0] + V.R[i * 3 + 1] * mu[1] + V.R[i * 3 + 2] * mu[2] + V.t[i];
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i)
        cols[k][i] = V.R[i * 3] * g.R[0 * 3 + k] + V.R[i * 3 + 1] * g.R[1 * 3 + k] +
                     V.R[i * 3 + 2] * g.R[2 * 3 + k];
    float Sg[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        float acc = 0.f;
        for (int k = 0; k < 3; ++k) acc += s[k] * s[k] * cols[k][i] * cols[k][j];
        Sg[i][j] = acc;
      }
    int tx0 = 0, ty0 = 0, tx1 = V.ntx - 1, ty1 = V.nty - 1;
    float sz = sqrtf(fmaxf(Sg[2][2], 0.f));
    if (!ok || c[2] + sz <= 0.0f) {
      tx0 = 1; tx1 = 0;  // entirely behind the camera: culled
    } else if (c[2] - sz > 1e-3f * (fabsf(c[2]) + sz)) {
      float A = c[2] * c[2] - Sg[2][2];
      float lim[2][2];
      bool good = A > 0.f;
      for (int ax = 0; ax < 2 && good; ++ax) {
        float B = c[ax] * c[2] - Sg[ax][2];
        float C = c[ax] * c[ax] - Sg[ax][ax];
        float disc = B * B - A * C;
        if (!(disc >= 0.f)) { good = false; break; }
        float sq = sqrtf(disc);
        float m0 = (B - sq) / A, m1 = (B + sq) / A;
        float f = ax == 0 ? V.fx : V.fy, cc = ax == 0 ? V.cx : V.cy;
        float u0 = cc + f * m0, u1 = cc + f * m1;
        float pad = 2.0f + 1e-3f * (fabsf(u0) + fabsf(u1));
        lim[ax][0] = u0 - pad;
        lim[ax][1] = u1 + pad;
      }
      if (good) {
        int n[2] = {V.ntx, V.nty};
        int lo[2], hi[2];
        for (int ax = 0; ax < 2; ++ax) {
          float a = floorf(lim[ax][0] / (float)w.tile);
          float b = floorf(lim[ax][1] / (float)w.tile);
          lo[ax] = a < 0.f ? 0 : (a >= (float)n[ax] ? n[ax] : (int)a);
          hi[ax] = b < 0.f ? -1 : (b >= (float)n[ax] ? n[ax] - 1 : (int)b);
        }
        tx0 = lo[0]; tx1 = hi[0]; ty0 = lo[1]; ty1 = hi[1];
        if (tx0 > tx1 || ty0 > ty1) { tx0 = 1; tx1 = 0; }
      }
    }
    pv.tx0 = tx0; pv.tx1 = tx1; pv.ty0 = ty0; pv.ty1 = ty1;
    w.pview[j] = pv;
  }
}


// ------------------------------------------------------------------------------------------
// Tile candidate lists: one warp per (view, tile), primitives in index order.

constexpr int kTileBlock = 256;
constexpr int kRectBatch = 512;

__global__ void __launch_bounds__(kTileBlock) k_tile_lists(Work w) {
  __shared__ int4 srect[kRectBatch];
  const int v = blockIdx.y;
  const ViewData& V = w.views[v];
  const int ntx = V.ntx, n_tiles = V.ntx * V.nty, K = V.prim_n;
  if ((int)blockIdx.x * (kTileBlock / 32) >= n_tiles) return;  // block-uniform
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * (kTileBlock / 32) + warp;
  const bool active = t < n_tiles;
  const int tx = active ? t % ntx : 0, ty = active ? t / ntx : 0;
  int count = 0;
  int* list = w.tile_list + V.cand_base + (size_t)(active ? t : 0) * K;
  for (int base = 0; base < K; base += kRectBatch) {
    int nb = min(kRectBatch, K - base);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += kTileBlock) {
      const PrimView& pv = w.pview[V.pv_base + base + i];
      srect[i] = make_int4(pv.tx0, pv.ty0, pv.tx1, pv.ty1);
    }
    __syncthreads();
    if (!active) continue;
    for (int i0 = 0; i0 < nb; i0 += 32) {
      int i = i0 + lane;
      bool in = false;
      if (i < nb) {
        int4 r = srect[i];
        in = tx >= r.x && tx <= r.z && ty >= r.y && ty <= r.w;
      }
      unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) list[count + __popc(m & ((1u << lane) - 1u))] = V.prim_base + base + i;
      count += __popc(m);
    }
  }
  if (active && lane == 0) w.tile_count[V.tile_base + t] = count;
}

// ------------------------------------------------------------------------------------------
// Intersection + per-ray sort. One block per (view, tile); one thread per pixel.

constexpr int kCandBatch = 128;
constexpr int kHist = 1024;

struct CandGeo {
  float Mhi[9], Mlo[9];
  float op_hi[3], op_lo[3];
};

struct HitGeom {
  bool hit;
  float key, tmid, r0, r1, p[3];
};

// Full double-float hit test of one (ray, primitive) pair.
MLPS_DEV HitGeom intersect_df(const float* Mhi, const float* Mlo, const float* op_hi,
                              const float* op_lo, const dfl d[3], float near_t) {
  HitGeom r;
  r.hit = false;
  dfl dp[3], op[3];
  for (int i = 0; i < 3; ++i) {
    dfl a = df_mul({Mhi[i * 3 + 0], Mlo[i * 3 + 0]}, d[0]);
    a = df_add(a, df_mul({Mhi[i * 3 + 1], Mlo[i * 3 + 1]}, d[1]));
    a = df_add(a, df_mul({Mhi[i * 3 + 2], Mlo[i * 3 + 2]}, d[2]));
    dp[i] = a;
    op[i] = {op_hi[i], op_lo[i]};
  }
  dfl a = df_dot3(dp, dp);
  dfl b = df_dot3(op, dp);
  dfl tmid = df_neg(df_div(b, a));
  dfl p[3];
  for (int i = 0; i < 3; ++i) p[i] = df_add(op[i], df_mul(tmid, dp[i]));
  dfl m2 = df_dot3(p, p);
  dfl rem = df_sub(df_make(1.0f), m2);  // 1 - m^2
  if (!(rem.hi > 0.0f)) return r;
  float h = sqrtf(df_to_f(rem) / df_to_f(a));
  float tm = df_to_f(tmid);
  float r0 = -h, r1 = h;
  // near clip: t0 = max(t_mid - h, near)
  dfl t0 = df_sub(tmid, df_make(h));
  if (t0.hi < near_t || (t0.hi == near_t && t0.lo < 0.f)) {
    dfl t1 = df_add(tmid, df_make(h));
    if (!(t1.hi > near_t || (t1.hi == near_t && t1.lo > 0.f))) return r;
    r0 = df_to_f(df_sub(df_make(near_t), tmid));
  }
  r.hit = true;
  r.tmid = tm;
  r.key = tm > 0.f ? tm : 0.f;
  r.r0 = r0;
  r.r1 = r1;
  for (int i = 0; i < 3; ++i) r.p[i] = df_to_f(p[i]);
  return r;
}

template <int TILE>
__global__ void __launch_bounds__(TILE* TILE) k_intersect(Work w) {
  constexpr int NT = TILE * TILE;
  __shared__ CandGeo scand[kCandBatch];
  __shared__ float skey[kCandBatch];  // tile-centre sort keys (tile_sort mode)
  __shared__ int shist[kHist];
  __shared__ int swarp[NT / 32];
  __shared__ int sbase;
  __shared__ ViewData sv;
  const int v = blockIdx.y, t = blockIdx.x;
  const ViewData& Vg = w.views[v];
  if (t >= Vg.ntx * Vg.nty) return;  // block-uniform: this view has fewer tiles
  const int tx = t % Vg.ntx, ty = t / Vg.ntx;
  const int x = tx * TILE + (int)(threadIdx.x % TILE);
  const int y = ty * TILE + (int)(threadIdx.x / TILE);
  const bool inside = x < Vg.width && y < Vg.height;
  if (threadIdx.x == 0) sv = Vg;
  const int ncand = w.tile_count[Vg.tile_base + t];
  const int* cand = w.tile_list + Vg.cand_base + (size_t)t * Vg.prim_n;
  const int pv_off = Vg.pv_base - Vg.prim_base;  // pview index of global primitive p: pv_off + p
  for (int i = threadIdx.x; i < kHist; i += NT) shist[i] = 0;
  __syncthreads();
  dfl d[3];
  if (inside) ray_dir_df(sv, x, y, d);
  const float near_t = sv.near_t;
  const int cap = w.max_hits;
  float lkey[kMaxHits], lt0[kMaxHits];
  int lc[kMaxHits];
  int n = 0;
  bool overflow = false;
  for (int base = 0; base < ncand; base += kCandBatch) {
    const int nb = min(kCandBatch, ncand - base);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += NT) {
      int p = cand[base + i];
      const PrimGeo& g = w.geo[p];
      const PrimView& pv = w.pview[pv_off + p];
      CandGeo cg;
      for (int k = 0; k < 9; ++k) { cg.Mhi[k] = g.Mhi[k]; cg.Mlo[k] = g.Mlo[k]; }
      for (int k = 0; k < 3; ++k) { cg.op_hi[k] = pv.op_hi[k]; cg.op_lo[k] = pv.op_lo[k]; }
      scand[i] = cg;
      if (w.tile_sort) {
        // max(0, t*) of the virtual ray through the tile centre, t* = -(o'.d'_c) / |d'_c|^2
        dfl dc[3], dp[3], op[3];
        ray_dir_df_uv(sv, (float)(tx * TILE) + 0.5f * TILE, (float)(ty * TILE) + 0.5f * TILE, dc);
        for (int k = 0; k < 3; ++k) {
          dfl a = df_mul({g.Mhi[k * 3 + 0], g.Mlo[k * 3 + 0]}, dc[0]);
          a = df_add(a, df_mul({g.Mhi[k * 3 + 1], g.Mlo[k * 3 + 1]}, dc[1]));
          a = df_add(a, df_mul({g.Mhi[k * 3 + 2], g.Mlo[k * 3 + 2]}, dc[2]));
          dp[k] = a;
          op[k] = {pv.op_hi[k], pv.op_lo[k]};
        }
        const float ts = df_to_f(df_neg(df_div(df_dot3(op, dp), df_dot3(dp, dp))));
        skey[i] = ts > 0.f ? ts : 0.f;
      }
    }
    __syncthreads();
    if (!inside) continue;
    for (int i = 0; i < nb; ++i) {
      const CandGeo& cg = scand[i];
      HitGeom hg = intersect_df(cg.Mhi, cg.Mlo, cg.op_hi, cg.op_lo, d, near_t);
      if (!hg.hit) continue;
      // exact order: the ray's own (key, t0); tile order: the tile-centre key, ties by index
      const float key = w.tile_sort ? skey[i] : hg.key, t0 = w.tile_sort ? 0.f : hg.tmid + hg.r0;
      const int c = base + i;
      // insertion from the back; equal (key, t0) keeps the lower primitive index first
      int j = n;
      while (j > 0 && (key < lkey[j - 1] || (key == lkey[j - 1] && t0 < lt0[j - 1]))) {
        if (j < cap) { lkey[j] = lkey[j - 1]; lt0[j] = lt0[j - 1]; lc[j] = lc[j - 1]; }
        --j;
      }
      if (j < cap) { lkey[j] = key; lt0[j] = t0; lc[j] = c; }
      if (n < cap) ++n; else overflow = true;
    }
  }
  if (overflow) set_status(w.saved_hdr, MLPS_ERR_CAPACITY_OVERFLOW);
  // block exclusive scan of per-ray counts
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = n;
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) swarp[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < NT / 32; ++i) { int c = swarp[i]; swarp[i] = acc; acc += c; }
    int b = atomicAdd(&w.saved_hdr[1], acc);
    if (b + acc > w.hit_cap) {
      set_status(w.saved_hdr, MLPS_ERR_CAPACITY_OVERFLOW);
      // the part of the reserved range inside the capacity stays unwritten: mark it invalid
      swarp[0] = b < w.hit_cap ? b : w.hit_cap;
      swarp[1] = min(b + acc, w.hit_cap);
      b = -1;
    }
    sbase = b;
  }
  __syncthreads();
  const int base = sbase;
  if (base < 0)
    for (int h = swarp[0] + threadIdx.x; h < swarp[1]; h += NT) w.hit_prim[h] = -1;
  const int excl = incl - n + swarp[warp];
  const int ray = sv.ray_base + y * sv.width + x;
  if (inside) {
    if (base < 0) {
      w.ray_start[ray] = 0;
      w.ray_count[ray] = 0;
    } else {
      const int start = base + excl;
      w.ray_start[ray] = start;
      w.ray_count[ray] = n;
      for (int j = 0; j < n; ++j) {
        const int c = lc[j];
        const int p = cand[c];
        const PrimGeo& g = w.geo[p];
        const PrimView& pv = w.pview[pv_off + p];
        HitGeom hg = intersect_df(g.Mhi, g.Mlo, pv.op_hi, pv.op_lo, d, near_t);
        const int h = start + j;
        w.hit_prim[h] = p;
        w.hit_ray[h] = ray;
        w.hit_tmid[h] = hg.tmid;
        w.hit_r0[h] = hg.r0;
        w.hit_r1[h] = hg.r1;
        w.hit_p[h] = hg.p[0];
        w.hit_p[(size_t)w.hit_cap + h] = hg.p[1];
        w.hit_p[2 * (size_t)w.hit_cap + h] = hg.p[2];
        if (c < kHist) atomicAdd(&shist[c], 1);
        else atomicAdd(&w.prim_count[p], 1);
      }
    }
  }
  __syncthreads();
  if (base >= 0)
    for (int c = threadIdx.x; c < min(ncand, kHist); c += NT)
      if (shist[c] > 0) atomicAdd(&w.prim_count[cand[c]], shist[c]);
}

// ------------------------------------------------------------------------------------------
// Exclusive scans over primitives: interval offsets and MLP chunk offsets.

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_prim_scan(Work w) {
  __shared__ int s0[kScanThreads / 32], s1[kScanThreads / 32];
  __shared__ int carry0, carry1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) { carry0 = 0; carry1 = 0; }
  __syncthreads();
  for (int base = 0; base < w.K; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const int c = i < w.K ? w.prim_count[i] : 0;
    const int ch = (c + w.ipc - 1) / w.ipc;
    int a = c, b = ch;
    for (int o = 1; o < 32; o <<= 1) {
      int ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o);
      if (lane >= o) { a += ua; b += ub; }
    }
    if (lane == 31) { s0[warp] = a; s1[warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
      int x0 = 0, x1 = 0;
      for (int k = 0; k < kScanThreads / 32; ++k) {
        int t0 = s0[k], t1 = s1[k];
        s0[k] = x0; s1[k] = x1;
        x0 += t0; x1 += t1;
      }
    }
    __syncthreads();
    if (i < w.K) {
      w.prim_start[i] = carry0 + s0[warp] + a - c;
      w.chunk_start[i] = carry1 + s1[warp] + b - ch;
      w.prim_cursor[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) {
      carry0 += s0[warp] + a;
      carry1 += s1[warp] + b;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.prim_start[w.K] = carry0;
    w.chunk_start[w.K] = carry1;
    w.saved_hdr[2] = carry1;
  }
}

// ------------------------------------------------------------------------------------------
// Scatter hit ids into per-primitive lists (warp-aggregated atomics).

__global__ void k_scatter(Work w) {
  const int n = min(w.saved_hdr[1], w.hit_cap);
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int h = base + threadIdx.x;
    const bool act = h < n;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    if (!act) continue;
    int p = w.hit_prim[h];
    if (p < 0 || p >= w.K) p = -1;  // records of an overflowed block (see k_intersect)
    const unsigned peers = __match_any_sync(am, p);
    if (p < 0) continue;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int off = 0;
    if (lane == leader) off = atomicAdd(&w.prim_cursor[p], __popc(peers));
    off = __shfl_sync(peers, off, leader);
    if (off + rank >= w.prim_count[p]) {
      set_status(w.saved_hdr, MLPS_ERR_CAPACITY_OVERFLOW);
      continue;
    }
    const int slot = w.prim_start[p] + off + rank;
    w.prim_list[slot] = h;
    w.slot_of[h] = slot;
    // the interval record: everything the MLP stage needs, contiguous per chunk
    const int ray = w.hit_ray[h];
    const int v = view_of_ray(w, ray);
    const int pix = ray - w.views[v].ray_base, vw = w.views[v].width;
    const int y = pix / vw, x = pix - y * vw;
    float d[3];
    ray_dir_f(w.views[v], x, y, d);
    const PrimGeo& g = w.geo[p];
    IntervalRec r;
    r.h = h;
    for (int i = 0; i < 3; ++i) {
      r.p[i] = w.hit_p[(size_t)i * w.hit_cap + h];
      r.d[i] = d[i];
      r.dp[i] = g.Mhi[i * 3] * d[0] + g.Mhi[i * 3 + 1] * d[1] + g.Mhi[i * 3 + 2] * d[2];
    }
    r.r0 = w.hit_r0[h];
    r.r1 = w.hit_r1[h];
    r.dt = (r.r1 - r.r0) / (float)w.S;
    r.tmid = w.hit_tmid[h];
    r.pad[0] = 0.f;
    r.pad[1] = 0.f;
    w.rec[slot] = r;
  }
}

// ------------------------------------------------------------------------------------------
// Inspection

__global__ void k_export_hits(Work w, int max_out, int* count, int* prim, float* t0, float* t1,
                              float* tmid) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= w.n_rays) return;
  const int n = w.ray_count[r], s = w.ray_start[r];
  count[r] = n;
  for (int j = 0; j < n && j < max_out; ++j) {
    const int h = s + j;
    const size_t o = (size_t)r * max_out + j;
    prim[o] = w.hit_prim[h];
    t0[o] = w.hit_tmid[h] + w.hit_r0[h];
    t1[o] = w.hit_tmid[h] + w.hit_r1[h];
    tmid[o] = w.hit_tmid[h];
  }
}

__global__ void k_export_tiles(Work w, int* count, int* list) {
  const size_t n = (size_t)w.V * w.n_tiles;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * w.K;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t tl = i / w.K;
    const int j = (int)(i % w.K);
    const int c = w.tile_count[tl];
    if (j == 0) count[tl] = c;
    list[i] = j < c ? w.tile_list[i] : -1;
  }
}

// ------------------------------------------------------------------------------------------
// Launchers

void launch_store_views(const Work& w, const ViewArray& va, cudaStream_t st) {
  k_store_views<<<1, kMaxViews, 0, st>>>(w, va);
}

void launch_views_from_items(const Work& w, const mlps_batch_item* items, int max_w, int max_h, int max_p,
                             cudaStream_t st) {
  k_views_from_items<<<1, kMaxViews, 0, st>>>(w, items, max_w, max_h, max_p);
}

int launch_prim_setup(const Work& w, const float* c, const float* s, const float* q,
                      cudaStream_t st) {
  if (w.K == 0) return 0;
  k_prim_geo<<<(w.K + 127) / 128, 128, 0, st>>>(w, c, s, q);
  if (w.n_pairs == 0) return 1;
  k_prim_view<<<(w.n_pairs + 127) / 128, 128, 0, st>>>(w);
  return 2;
}

void launch_tile_lists(const Work& w, cudaStream_t st) {
  dim3 grid((w.max_view_tiles + kTileBlock / 32 - 1) / (kTileBlock / 32), w.V);
  k_tile_lists<<<grid, kTileBlock, 0, st>>>(w);
}

bool launch_intersect(const Work& w, cudaStream_t st) {
  dim3 grid(w.max_view_tiles, w.V);
  if (w.tile == 16) k_intersect<16><<<grid, 256, 0, st>>>(w);
  else if (w.tile == 8) k_intersect<8><<<grid, 64, 0, st>>>(w);
  else return false;
  return true;
}

void launch_prim_scan(const Work& w, cudaStream_t st) {
  k_prim_scan<<<1, kScanThreads, 0, st>>>(w);
}

void launch_scatter(const Work& w, int n_sm, cudaStream_t st) {
  k_scatter<<<n_sm * 4, 256, 0, st>>>(w);
}

void launch_export_hits(const Work& w, int max_out, int* count, int* prim, float* t0, float* t1,
                        float* tmid, cudaStream_t st) {
  k_export_hits<<<(w.n_rays + 255) / 256, 256, 0, st>>>(w, max_out, count, prim, t0, t1, tmid);
}

void launch_export_tiles(const Work& w, int* count, int* list, cudaStream_t st) {
  k_export_tiles<<<1024, 256, 0, st>>>(w, count, list);
}

}  // namespace mlps
