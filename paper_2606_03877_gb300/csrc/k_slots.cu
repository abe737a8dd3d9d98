// k_slots.cu -- feature slots (Sec. 3.4): a C-channel semantic feature per hit, composited with
// the hits' volumetric weights, and its reverse pass.
//
// Every primitive carries four slot embeddings e_k in R^C (FP32, after its MLP in the packed
// blob). A hit's scale-normalised offset of the centre from the contact point is
//   u = clip_[-1,1]^3(R^T delta / s),  delta = mu - p*,  p* = o + max(0, t*) d   (Eq. 3),
// and in the primitive's normalised frame R^T delta / s = M delta = -p + min(t_mid, 0) d',
// with p = o' + t_mid d' the interval's closest point: no world-frame subtraction is needed.
// The slot weights are g_k = softmax_k(a_k . u) over the unit vertices a_k of a regular
// tetrahedron ((+-1, +-1, +-1) / sqrt 3, even number of minus signs), the hit's feature is
// f = sum_k g_k e_k, and the feature map is F = sum_j w_j f_j with the hit's compositing weight
// w_j = T_j (1 - e^{-a_j}) (the sum of T alpha over its samples), in the ray's t* order and
// with the same early termination as the colour composite.
//
// Layout and bounds. The work is wide-channel and memory-bound: per ray and hit the four
// embeddings (16 C bytes, L2-resident for any K of these scenes) are read and C floats of F are
// written (the HBM term). One warp per ray, each lane owning four channels of every 128-channel
// group (float4 loads and stores), up to 512 channels per pass.
//
// Reverse pass, with s_jk = e_jk . dL/dF and s_j = sum_k g_jk s_jk (= f_j . dL/dF):
//   dL/da_j = T_j e^{-a_j} s_j - sum_{l>j} w_l s_l           (k_slots_bwd_ray -> slot_ga)
//   dL/dg_jk = w_j s_jk,  dL/dz = g (dL/dg - g . dL/dg),  dL/du = sum_k dL/dz_k a_k (clip mask)
//   dL/de_pk = sum_{hits j of p} w_j g_jk dL/dF_ray(j)       (k_slots_bwd_prim, per primitive)
// and dL/du is chained to the pose: y = M delta gives dL/dM += g_y delta^T and
// dL/d delta = M^T g_y, which reaches mu directly and, where t_mid > 0, through t* = t_mid
// (dL/dt_mid = -d . dL/d delta), whose own chain into (M, mu) is that of the MLP kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

namespace mlps {
namespace {

constexpr int kSlotWarps = 8;       // rays (warps) per block
constexpr int kPrimThreads = 128;   // per-primitive reduction: 4 channels per thread per pass
constexpr int kPassCh = 512;        // channels per pass (32 lanes or 128 threads x 4)

MLPS_DEV float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// a_k . u for the four tetrahedral directions
MLPS_DEV void slot_logits(const float u[3], float z[4]) {
  const float r = 0.57735026918962576f;  // 1 / sqrt(3)
  z[0] = r * (u[0] + u[1] + u[2]);
  z[1] = r * (u[0] - u[1] - u[2]);
  z[2] = r * (-u[0] + u[1] - u[2]);
  z[3] = r * (-u[0] - u[1] + u[2]);
}

MLPS_DEV void slot_softmax(const float u[3], float g[4]) {
  float z[4];
  slot_logits(u, z);
  const float zm = fmaxf(fmaxf(z[0], z[1]), fmaxf(z[2], z[3]));
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    g[k] = expf(z[k] - zm);
    sum += g[k];
  }
  const float inv = 1.f / sum;
#pragma unroll
  for (int k = 0; k < 4; ++k) g[k] *= inv;
}

// y = -p + min(t_mid, 0) d' (= M delta) and u = clip(y)
MLPS_DEV void slot_offset(const float p[3], float tmid, const float dp[3], float y[3], float u[3]) {
  const float tn = fminf(tmid, 0.f);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    y[c] = fmaf(tn, dp[c], -p[c]);
    u[c] = fminf(fmaxf(y[c], -1.f), 1.f);
  }
}

// The offset of hit h (ray order): p from the hit record, d' (only needed when t_mid < 0) from
// the interval record.
MLPS_DEV void hit_offset(const Work& w, int h, float y[3], float u[3]) {
  const float tm = w.hit_tmid[h];
  float p[3], dp[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < 3; ++c) p[c] = w.hit_p[(size_t)c * w.hit_cap + h];
  if (tm < 0.f) {
    const IntervalRec& r = w.rec[w.slot_of[h]];
#pragma unroll
    for (int c = 0; c < 3; ++c) dp[c] = r.dp[c];
  }
  slot_offset(p, tm, dp, y, u);
}

MLPS_DEV const float* slot_emb(const unsigned char* blob, long long stride, long long slot_byte, int prim) {
  return reinterpret_cast<const float*>(blob + (size_t)prim * stride + slot_byte);
}

MLPS_DEV float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

MLPS_DEV void fma4(float4& a, float s, const float4& v) {
  a.x = fmaf(s, v.x, a.x);
  a.y = fmaf(s, v.y, a.y);
  a.z = fmaf(s, v.z, a.z);
  a.w = fmaf(s, v.w, a.w);
}

MLPS_DEV float dot4(const float4& a, const float4& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// dF row access: float4 when the row base is 16-byte aligned, else scalar
MLPS_DEV float4 ld_row4(const float* p, bool vec) {
  if (vec) return ld4(p);
  return make_float4(__ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3));
}

MLPS_DEV void st_row4(float* p, const float4& v, bool vec) {
  if (vec) {
    *reinterpret_cast<float4*>(p) = v;
  } else {
    p[0] = v.x; p[1] = v.y; p[2] = v.z; p[3] = v.w;
  }
}

// Rays are walked tile by tile (one block per screen tile of the binning grid): the rays of a
// tile meet the same few primitives, so their embeddings stay in the SM's L1 instead of being
// fetched from L2 once per (ray, hit).
struct TileRays {
  int base, W, x0, y0, tw, th;  // ray_base of the view, its width, the tile's origin and extent
};

MLPS_DEV TileRays tile_rays(const Work& w, int t) {
  int lo = 0, hi = w.V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.views[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  const ViewData& V = w.views[lo];
  const int lt = t - V.tile_base;
  TileRays r;
  if (lt >= V.ntx * V.nty) {  // past the live total (device item table): no rays
    r.base = r.W = r.x0 = r.y0 = r.tw = r.th = 0;
    return r;
  }
  r.base = V.ray_base;
  r.W = V.width;
  r.x0 = (lt % V.ntx) * w.tile;
  r.y0 = (lt / V.ntx) * w.tile;
  r.tw = min(w.tile, V.width - r.x0);
  r.th = min(w.tile, V.height - r.y0);
  return r;
}

MLPS_DEV int tile_ray(const TileRays& T, int i) {  // i < tw * th, row-major in the tile
  const int y = i / T.tw, x = i - y * T.tw;
  return T.base + (T.y0 + y) * T.W + T.x0 + x;
}

// Per-hit scalars of one ray, held lane-parallel: lane l keeps hit l in set 0 and hit l + 32 in
// set 1 (rays have at most 64 hits). The optical depths are summed in ray order exactly as the
// colour composite does, so the early-termination cut and T_j are the same floats.
struct HitSet {
  float T, W, wgt;  // transmittance before the hit, 1 - e^{-a}, weight T W
  float g[4];       // slot weights
  float y[3];       // unclipped offset (for the clip mask of the reverse pass)
  int prim;
};

MLPS_DEV void ray_hits(const Work& w, int s0, int n, int lane, HitSet (&hs)[2], int& used) {
  float A = 0.f, aex[2] = {0.f, 0.f}, a[2] = {0.f, 0.f};
  used = n;
  for (int j = 0; j < n; ++j) {
    const float aj = w.hit_out[s0 + j].w;
    if (lane == (j & 31)) {
      if (j < 32) { aex[0] = A; a[0] = aj; }
      else { aex[1] = A; a[1] = aj; }
    }
    A += aj;
    if (expf(-A) < w.t_eps) {
      used = j + 1;
      break;
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = lane + 32 * q;
    HitSet& H = hs[q];
    H.T = H.W = H.wgt = 0.f;
    H.prim = 0;
    for (int k = 0; k < 4; ++k) H.g[k] = 0.f;
    H.y[0] = H.y[1] = H.y[2] = 0.f;
    if (j < used) {
      const int h = s0 + j;
      float u[3];
      H.T = expf(-aex[q]);
      H.W = -expm1f(-a[q]);
      H.wgt = H.T * H.W;
      hit_offset(w, h, H.y, u);
      slot_softmax(u, H.g);
      H.prim = w.hit_prim[h];
    }
  }
}

// Hit j's scalars broadcast from its lane (register selects, no local-memory indexing).
MLPS_DEV void bcast_hit(const HitSet (&hs)[2], int j, float& wgt, float g[4], int& prim) {
  const bool hi = j >= 32;
  const int src = j & 31;
  wgt = __shfl_sync(0xffffffffu, hi ? hs[1].wgt : hs[0].wgt, src);
#pragma unroll
  for (int k = 0; k < 4; ++k) g[k] = __shfl_sync(0xffffffffu, hi ? hs[1].g[k] : hs[0].g[k], src);
  prim = __shfl_sync(0xffffffffu, hi ? hs[1].prim : hs[0].prim, src);
}

// ------------------------------------------------------------------------------------------
// Forward: F_r = sum_j w_j sum_k g_jk e_{p_j k}

__global__ void __launch_bounds__(32 * kSlotWarps) k_slots_fwd(Work w, int C, const unsigned char* blob,
                                                              long long stride, long long slot_byte,
                                                              float* __restrict__ feat, int FT, int vec) {
  const int lane = threadIdx.x & 31;
  for (int t = blockIdx.x; t < w.n_tiles_all; t += gridDim.x) {
    const TileRays TR = tile_rays(w, t);
    for (int i = threadIdx.x >> 5; i < TR.tw * TR.th; i += kSlotWarps) {
      const int r = tile_ray(TR, i);
      HitSet hs[2];
      int used;
      ray_hits(w, w.ray_start[r], w.ray_count[r], lane, hs, used);
      float* out = feat + (size_t)r * FT;
      for (int c0 = 0; c0 < C; c0 += kPassCh) {
        float4 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < used; ++j) {
          float wj, g[4];
          int prim;
          bcast_hit(hs, j, wj, g, prim);
#pragma unroll
          for (int k = 0; k < 4; ++k) g[k] *= wj;
          const float* e = slot_emb(blob, stride, slot_byte, prim);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = c0 + 128 * q + 4 * lane;
            if (c < C) {
#pragma unroll
              for (int k = 0; k < 4; ++k) fma4(acc[q], g[k], ld4(e + (size_t)k * C + c));
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = c0 + 128 * q + 4 * lane;
          if (c < C) st_row4(out + c, acc[q], vec);
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Reverse, ray-major: dL/da_j (slot_ga) and (dL/du, w_j) (slot_gu) per hit

MLPS_DEV float warp_excl_suffix(float v, int lane) {  // sum over higher lanes
  float incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_down_sync(0xffffffffu, incl, o);
    if (lane + o < 32) incl += u;
  }
  return incl - v;
}

__global__ void __launch_bounds__(32 * kSlotWarps) k_slots_bwd_ray(Work w, int C, const unsigned char* blob,
                                                                  long long stride, long long slot_byte,
                                                                  const float* __restrict__ dF, int FT,
                                                                  int vec) {
  const int lane = threadIdx.x & 31;
  for (int t = blockIdx.x; t < w.n_tiles_all; t += gridDim.x) {
    const TileRays TR = tile_rays(w, t);
    for (int i = threadIdx.x >> 5; i < TR.tw * TR.th; i += kSlotWarps) {
      const int r = tile_ray(TR, i);
      const int n = w.ray_count[r], s0 = w.ray_start[r];
      HitSet hs[2];
      int used;
      ray_hits(w, s0, n, lane, hs, used);
      const float* gF = dF + (size_t)r * FT;
      // s_jk = e_jk . dL/dF, kept by the hit's own lane
      float my_s[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      for (int j = 0; j < used; ++j) {
        const int prim = __shfl_sync(0xffffffffu, j < 32 ? hs[0].prim : hs[1].prim, j & 31);
        const float* e = slot_emb(blob, stride, slot_byte, prim);
        float sk[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = 0; c0 < C; c0 += kPassCh) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = c0 + 128 * q + 4 * lane;
            if (c < C) {
              const float4 gv = ld_row4(gF + c, vec);
#pragma unroll
              for (int k = 0; k < 4; ++k) sk[k] += dot4(ld4(e + (size_t)k * C + c), gv);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) sk[k] = warp_sum(sk[k]);
        if (lane == (j & 31)) {
          if (j < 32) {
#pragma unroll
            for (int k = 0; k < 4; ++k) my_s[0][k] = sk[k];
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) my_s[1][k] = sk[k];
          }
        }
      }
      // per hit (lane-parallel): s_j, the suffix sum of w_l s_l over later hits, dL/da_j, dL/du
      float ws[2], sj[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const HitSet& H = hs[q];
        sj[q] = H.g[0] * my_s[q][0] + H.g[1] * my_s[q][1] + H.g[2] * my_s[q][2] + H.g[3] * my_s[q][3];
        ws[q] = H.wgt * sj[q];  // zero beyond `used`
      }
      const float tot1 = warp_sum(ws[1]);
      const float R0 = warp_excl_suffix(ws[0], lane) + tot1;
      const float R1 = warp_excl_suffix(ws[1], lane);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int j = lane + 32 * q;
        if (j >= n) continue;
        const int h = s0 + j;
        if (j >= used) {  // beyond early termination: no gradient
          w.slot_ga[h] = 0.f;
          w.slot_gu[h] = make_float4(0.f, 0.f, 0.f, 0.f);
          continue;
        }
        const HitSet& H = hs[q];
        w.slot_ga[h] = H.T * (1.f - H.W) * sj[q] - (q == 0 ? R0 : R1);
        // softmax and clip: dL/du
        float dg[4], mean = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          dg[k] = H.wgt * my_s[q][k];
          mean = fmaf(H.g[k], dg[k], mean);
        }
        float dz[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) dz[k] = H.g[k] * (dg[k] - mean);
        const float rr = 0.57735026918962576f;
        float gu[3];
        gu[0] = rr * (dz[0] + dz[1] - dz[2] - dz[3]);
        gu[1] = rr * (dz[0] - dz[1] + dz[2] - dz[3]);
        gu[2] = rr * (dz[0] - dz[1] - dz[2] + dz[3]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (H.y[c] < -1.f || H.y[c] > 1.f) gu[c] = 0.f;
        w.slot_gu[h] = make_float4(gu[0], gu[1], gu[2], H.wgt);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Reverse, primitive-major: dL/de and the pose chain of dL/du. Each block takes a contiguous
// range of the primitive-major interval order, in batches of kPrimThreads hits; accumulators
// are flushed with atomics when the range moves to another primitive.

struct PrimBatch {
  int ray[kPrimThreads];
  float c[kPrimThreads][4];  // w_j g_jk
};

__global__ void __launch_bounds__(kPrimThreads) k_slots_bwd_prim(Work w, int C, const unsigned char* blob,
                                                                long long stride, long long slot_byte,
                                                                const float* __restrict__ dF, int FT,
                                                                int vec, float* __restrict__ d_weights,
                                                                int Prow, int Pmlp) {
  __shared__ PrimBatch sb;
  __shared__ float sgeo[12];
  __shared__ int sprim[kPrimThreads];
  const int total = w.prim_start[w.K];
  const int b0 = (int)((long long)total * blockIdx.x / gridDim.x);
  const int b1 = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  if (b0 >= b1) return;
  const int t = threadIdx.x;
  for (int c0 = 0; c0 < C; c0 += kPassCh) {
    const bool pose = c0 == 0;  // the pose chain once, with the first channel pass
    float4 acc[4];
    auto zero = [&]() {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    zero();
    if (t < 12) sgeo[t] = 0.f;
    // first primitive of the range
    int lo = 0, hi = w.K - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (w.prim_start[mid] <= b0) lo = mid; else hi = mid - 1;
    }
    int prim = lo;
    auto flush = [&](int p) {
      float* dE = d_weights + (size_t)p * Prow + Pmlp;
      // thread t owns channels c0 + 4 t .. + 3 of each slot
      const int c = c0 + 4 * t;
      if (c < C) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float* d = dE + (size_t)k * C + c;
          if (acc[k].x != 0.f) atomicAdd(d, acc[k].x);
          if (acc[k].y != 0.f) atomicAdd(d + 1, acc[k].y);
          if (acc[k].z != 0.f) atomicAdd(d + 2, acc[k].z);
          if (acc[k].w != 0.f) atomicAdd(d + 3, acc[k].w);
        }
      }
      zero();
      if (pose) {
        __syncthreads();
        if (t < 12) {
          if (sgeo[t] != 0.f) atomicAdd(&w.dgeo[12 * (size_t)p + t], sgeo[t]);
          sgeo[t] = 0.f;
        }
        __syncthreads();
      }
    };
    for (int s = b0; s < b1; s += kPrimThreads) {
      const int nb = min(kPrimThreads, b1 - s);
      __syncthreads();
      // per hit of the batch: its ray, coefficients and (first pass) pose contribution
      float mine[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) mine[e] = 0.f;
      int my_prim = -1;
      if (t < nb) {
        const int slot = s + t;
        const int h = w.prim_list[slot];
        my_prim = w.hit_prim[h];
        const IntervalRec& rc = w.rec[slot];
        const float4 gu4 = w.slot_gu[h];
        float y[3], u[3], g[4];
        slot_offset(rc.p, rc.tmid, rc.dp, y, u);
        slot_softmax(u, g);
        sb.ray[t] = w.hit_ray[h];
#pragma unroll
        for (int k = 0; k < 4; ++k) sb.c[t][k] = gu4.w * g[k];
        if (pose && (gu4.x != 0.f || gu4.y != 0.f || gu4.z != 0.f)) {
          const PrimGeo& G = w.geo[my_prim];
          const float gy[3] = {gu4.x, gu4.y, gu4.z};
          // delta = -R S p + min(t_mid, 0) d (world frame)
          float del[3], ymid[3];
          const float tn = fminf(rc.tmid, 0.f);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            ymid[q] = G.R[q * 3] * G.s[0] * rc.p[0] + G.R[q * 3 + 1] * G.s[1] * rc.p[1] +
                      G.R[q * 3 + 2] * G.s[2] * rc.p[2];
            del[q] = fmaf(tn, rc.d[q], -ymid[q]);
          }
          float gdel[3];
#pragma unroll
          for (int e2 = 0; e2 < 3; ++e2)
            gdel[e2] = G.Mhi[e2] * gy[0] + G.Mhi[3 + e2] * gy[1] + G.Mhi[6 + e2] * gy[2];
#pragma unroll
          for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int e2 = 0; e2 < 3; ++e2) mine[q * 3 + e2] = gy[q] * del[e2];
#pragma unroll
          for (int e2 = 0; e2 < 3; ++e2) mine[9 + e2] = gdel[e2];
          if (rc.tmid > 0.f) {
            const float gtm = -(gdel[0] * rc.d[0] + gdel[1] * rc.d[1] + gdel[2] * rc.d[2]);
            const float aa = rc.dp[0] * rc.dp[0] + rc.dp[1] * rc.dp[1] + rc.dp[2] * rc.dp[2];
            float go[3], cd[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              go[q] = -gtm * rc.dp[q] / aa;
              cd[q] = -gtm * rc.p[q] / aa;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
              for (int e2 = 0; e2 < 3; ++e2) mine[q * 3 + e2] += go[q] * ymid[e2] + cd[q] * rc.d[e2];
#pragma unroll
            for (int e2 = 0; e2 < 3; ++e2)
              mine[9 + e2] -= G.Mhi[e2] * go[0] + G.Mhi[3 + e2] * go[1] + G.Mhi[6 + e2] * go[2];
          }
        }
      }
      sprim[t] = my_prim;
      __syncthreads();
      // walk the batch in order; the primitive changes at most a few times per batch
      int i = 0;
      while (i < nb) {
        const int p = sprim[i];
        if (p != prim) {
          flush(prim);
          prim = p;
        }
        int i1 = i;
        while (i1 < nb && sprim[i1] == p) ++i1;
        const int c = c0 + 4 * t;
        if (c < C) {
          for (int k2 = i; k2 < i1; ++k2) {
            const float4 gv = ld_row4(dF + (size_t)sb.ray[k2] * FT + c, vec);
#pragma unroll
            for (int k = 0; k < 4; ++k) fma4(acc[k], sb.c[k2][k], gv);
          }
        }
        if (pose) {
          // block sum of the pose contributions of hits i .. i1 - 1 (all of primitive p)
          const bool in = t >= i && t < i1;
#pragma unroll
          for (int e = 0; e < 12; ++e) {
            const float v = warp_sum(in ? mine[e] : 0.f);
            if ((t & 31) == 0 && v != 0.f) atomicAdd(&sgeo[e], v);
          }
        }
        i = i1;
      }
    }
    flush(prim);
    __syncthreads();
  }
}

}  // namespace

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

void launch_slots_fwd(const Work& w, const Model& m, const Packed& pk, const unsigned char* weights,
                      float* feat, int row_stride, cudaStream_t st) {
  if (w.n_rays == 0 || w.n_tiles_all == 0 || m.C == 0) return;
  const int vec = aligned16(feat) && row_stride % 4 == 0;
  const int grid = std::min(w.n_tiles_all, 1 << 20);
  k_slots_fwd<<<grid, 32 * kSlotWarps, 0, st>>>(
      w, m.C, weights, pk.stride, pk.slot_byte, feat, row_stride, vec);
}

void launch_slots_bwd_ray(const Work& w, const Model& m, const Packed& pk, const unsigned char* weights,
                          const float* d_feat, int row_stride, cudaStream_t st) {
  if (w.n_rays == 0 || w.n_tiles_all == 0 || m.C == 0) return;
  const int vec = aligned16(d_feat) && row_stride % 4 == 0;
  const int grid = std::min(w.n_tiles_all, 1 << 20);
  k_slots_bwd_ray<<<grid, 32 * kSlotWarps, 0, st>>>(
      w, m.C, weights, pk.stride, pk.slot_byte, d_feat, row_stride, vec);
}

void launch_slots_bwd_prim(const Work& w, const Model& m, const Packed& pk, const unsigned char* weights,
                           const float* d_feat, int row_stride, float* d_weights, int n_sm, cudaStream_t st) {
  if (w.K == 0 || m.C == 0) return;
  const int vec = aligned16(d_feat) && row_stride % 4 == 0;
  k_slots_bwd_prim<<<n_sm * 8, kPrimThreads, 0, st>>>(w, m.C, weights, pk.stride, pk.slot_byte, d_feat,
                                                      row_stride, vec, d_weights, m.Prow, m.P);
}

}  // namespace mlps
