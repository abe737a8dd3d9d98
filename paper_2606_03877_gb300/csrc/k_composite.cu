// k_composite.cu -- per-ray front-to-back compositing of the sorted hit intervals (Eq. 6), its
// reverse pass, and the final chain of the pose gradient to (centre, scale, quaternion).
//
// Each hit interval j of a ray carries its partial composite (C_j, a_j) from the MLP stage:
// C_j = sum_k T_k alpha_k c_k with T_k the transmittance inside the interval, and
// a_j = sum_k sigma_k Delta its optical depth. Along the ray, in t* order,
// C = sum_j T_j C_j and T_j = exp(-sum_{l<j} a_l) (log-space transmittance). Compositing stops
// once T drops below t_eps (early termination, Sec. B.2); the rest of the ray is skipped.
#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

namespace mlps {

__global__ void k_composite_fwd(Work w, int F, int FT, float* __restrict__ rgb, float* __restrict__ trans,
                                float* __restrict__ feat) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= w.n_rays || r >= live_rays(w)) return;
  const int n = w.ray_count[r], s = w.ray_start[r];
  float A = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  float Fv[kMaxFeat];
  for (int f = 0; f < F; ++f) Fv[f] = 0.f;
  for (int j = 0; j < n; ++j) {
    const float4 o = w.hit_out[s + j];
    const float T = expf(-A);
    C0 = fmaf(T, o.x, C0);
    C1 = fmaf(T, o.y, C1);
    C2 = fmaf(T, o.z, C2);
    for (int f = 0; f < F; ++f) Fv[f] = fmaf(T, w.hit_feat[(size_t)(s + j) * F + f], Fv[f]);
    A += o.w;
    if (expf(-A) < w.t_eps) break;
  }
  rgb[3 * (size_t)r] = C0;
  rgb[3 * (size_t)r + 1] = C1;
  rgb[3 * (size_t)r + 2] = C2;
  trans[r] = expf(-A);
  for (int f = 0; f < F; ++f) feat[(size_t)r * FT + f] = Fv[f];
}

// Reverse pass. With C = sum_j T_j C_j, T_final = exp(-sum_j a_j):
//   dL/dC_j = T_j dL/dC,   dL/dF_j = T_j dL/dF,
//   dL/da_j = -dL/dC . sum_{l>j} T_l C_l - dL/dF . sum_{l>j} T_l F_l - dL/dT_final T_final.
// Two forward sweeps, no per-hit array: the first repeats the forward composite (the same
// operations, so the same T_j, early-termination cut and totals C, F); the second walks the
// intervals again with the prefix P_j = sum_{l<j} T_l C_l and takes the suffix sums as
// sum_{l>j} T_l C_l = C - P_j - T_j C_j.
// Intervals skipped by early termination get zero gradient. The per-interval gradients are
// written in the primitive-major order of the interval records, so that the MLP backward
// reads one contiguous block per chunk. With feature slots, `slot_ga` adds the slot features'
// own dL/da_j per interval (hit order).
__global__ void k_composite_bwd(Work w, int F, int FT, const float* __restrict__ d_rgb,
                                const float* __restrict__ d_trans,
                                const float* __restrict__ d_feat,
                                const float* __restrict__ slot_ga) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= w.n_rays || r >= live_rays(w)) return;
  const int n = w.ray_count[r], s = w.ray_start[r];
  float A = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  float RF[kMaxFeat];  // sweep 1: the totals F; sweep 2: the suffix sums
  for (int f = 0; f < F; ++f) RF[f] = 0.f;
  int used = 0;
  for (int j = 0; j < n; ++j) {
    const float4 o = w.hit_out[s + j];
    const float T = expf(-A);
    C0 = fmaf(T, o.x, C0);
    C1 = fmaf(T, o.y, C1);
    C2 = fmaf(T, o.z, C2);
    for (int f = 0; f < F; ++f) RF[f] = fmaf(T, w.hit_feat[(size_t)(s + j) * F + f], RF[f]);
    A += o.w;
    used = j + 1;
    if (expf(-A) < w.t_eps) break;
  }
  const float Tfin = expf(-A);
  const float g0 = d_rgb[3 * (size_t)r], g1 = d_rgb[3 * (size_t)r + 1], g2 = d_rgb[3 * (size_t)r + 2];
  const float gT = d_trans ? d_trans[r] : 0.f;
  float gF[kMaxFeat];
  for (int f = 0; f < F; ++f) gF[f] = d_feat ? d_feat[(size_t)r * FT + f] : 0.f;
  float P0 = 0.f, P1 = 0.f, P2 = 0.f;  // prefix sums of T_l C_l over l < j
  A = 0.f;
  for (int j = 0; j < used; ++j) {
    const int h = s + j;
    const float4 o = w.hit_out[h];
    const float T = expf(-A);
    const float Q0 = fmaf(T, o.x, P0), Q1 = fmaf(T, o.y, P1), Q2 = fmaf(T, o.z, P2);  // P_{j+1}
    float ga = -(g0 * (C0 - Q0) + g1 * (C1 - Q1) + g2 * (C2 - Q2)) - gT * Tfin;
    const int sl = w.slot_of[h];
    for (int f = 0; f < F; ++f) {
      const float TFj = T * w.hit_feat[(size_t)h * F + f];
      RF[f] -= TFj;  // now sum over l > j
      ga -= gF[f] * RF[f];
      w.hit_gfeat[(size_t)sl * F + f] = T * gF[f];
    }
    if (slot_ga) ga += slot_ga[h];
    w.hit_grad[sl] = make_float4(T * g0, T * g1, T * g2, ga);
    P0 = Q0;
    P1 = Q1;
    P2 = Q2;
    A += o.w;
  }
  for (int j = used; j < n; ++j) {
    const int sl = w.slot_of[s + j];
    w.hit_grad[sl] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int f = 0; f < F; ++f) w.hit_gfeat[(size_t)sl * F + f] = 0.f;
  }
}

// dL/dM (9) and dL/dmu (3) per primitive -> centre, scale, quaternion.
// M_ij = R_ji / s_i with R = R(q/|q|); the quaternion gradient is projected through the
// normalisation: dL/dq = (g - qn (qn . g)) / |q|.
__global__ void k_pose_bwd(Work w, float* d_centers, float* d_scales, float* d_quats) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= w.K) return;
  const PrimGeo& g = w.geo[p];
  const float* dM = w.dgeo + 12 * (size_t)p;
  for (int i = 0; i < 3; ++i) d_centers[3 * p + i] = dM[9 + i];
  float dR[9];
  for (int i = 0; i < 9; ++i) dR[i] = 0.f;
  for (int i = 0; i < 3; ++i) {
    float acc = 0.f;
    for (int j = 0; j < 3; ++j) {
      acc += dM[i * 3 + j] * (-g.R[j * 3 + i] / (g.s[i] * g.s[i]));
      dR[j * 3 + i] += dM[i * 3 + j] / g.s[i];
    }
    d_scales[3 * p + i] = acc;
  }
  const float qw = g.qn[0], qx = g.qn[1], qy = g.qn[2], qz = g.qn[3];
  float gq[4];
  gq[0] = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
  gq[1] = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - qw * dR[5] + qz * dR[6] +
                 qw * dR[7] - 2.f * qx * dR[8]);
  gq[2] = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] +
                 qz * dR[7] - 2.f * qy * dR[8]);
  gq[3] = 2.f * (-2.f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.f * qz * dR[4] +
                 qy * dR[5] + qx * dR[6] + qy * dR[7]);
  const float dot = gq[0] * qw + gq[1] * qx + gq[2] * qy + gq[3] * qz;
  for (int i = 0; i < 4; ++i) d_quats[4 * p + i] = g.valid ? (gq[i] - g.qn[i] * dot) / g.qlen : 0.f;
}

void launch_composite_fwd(const Work& w, int F, int FT, float* rgb, float* trans, float* feat,
                          cudaStream_t st) {
  if (w.n_rays == 0) return;
  k_composite_fwd<<<(w.n_rays + 255) / 256, 256, 0, st>>>(w, F, FT, rgb, trans, feat);
}

void launch_composite_bwd(const Work& w, int F, int FT, const float* d_rgb, const float* d_trans,
                          const float* d_feat, const float* slot_ga, cudaStream_t st) {
  if (w.n_rays == 0) return;
  k_composite_bwd<<<(w.n_rays + 255) / 256, 256, 0, st>>>(w, F, FT, d_rgb, d_trans, d_feat, slot_ga);
}

// ------------------------------------------------------------------------------------------
// The MLP backward's interval lists. An interval is live when it has a nonzero gradient:
// dL/dC_j, dL/da_j or a feature gradient. Intervals behind a ray's early-termination point get
// none from the reverse composite, nor do the intervals of rays whose dL/dC is zero (pixels
// outside a training step's tile mask); such an interval adds nothing to any weight or pose
// gradient (its delta rows and its pose-chain terms are all zero). The backward therefore gets
// lists of the live intervals only, in the forward's primitive-major order: per primitive its
// live count, start and chunk start, and for each list position the interval's forward
// position. Four passes: flags with per-block counts, one scan of the counts, the ordered
// write, and per primitive its range in the list (binary search) with the scan of its chunks.

MLPS_DEV bool interval_live(const Work& w, int j, int F) {
  const float4 g = w.hit_grad[j];
  bool live = g.x != 0.f || g.y != 0.f || g.z != 0.f || g.w != 0.f;
  for (int f = 0; f < F && !live; ++f) live = w.hit_gfeat[(size_t)j * F + f] != 0.f;
  return live;
}

MLPS_DEV int n_intervals(const Work& w) { return min(w.saved_hdr[1], w.hit_cap); }

// Whether list `mode` takes the interval at primitive-major position j: 0 = a nonzero gradient
// (the backward's list); 1 = among its ray's first k1 hits (the first depth wave); 2 = later
// than its ray's first k1 hits, on a ray still open after the first wave (the second wave).
MLPS_DEV bool list_takes(const Work& w, int j, int F, int mode, int k1) {
  if (mode == 0) return interval_live(w, j, F);
  const int h = w.prim_list[j];
  const int r = w.hit_ray[h];
  const int rank = h - w.ray_start[r];
  return mode == 1 ? rank < k1 : (rank >= k1 && w.ray_alive[r] != 0);
}

constexpr int kLivePer = 4;  // intervals per thread (consecutive)

// Live flags of this thread's intervals as bits, and their count.
MLPS_DEV int live_bits(const Work& w, int j0, int F, int mode, int k1) {
  const int n = n_intervals(w);
  int bits = 0;
#pragma unroll
  for (int e = 0; e < kLivePer; ++e)
    if (j0 + e < n && list_takes(w, j0 + e, F, mode, k1)) bits |= 1 << e;
  return bits;
}

// Block-wide exclusive scan of one value per thread (kLiveBlock threads).
MLPS_DEV int block_excl_scan(int v, int* swarp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += u;
  }
  if (lane == 31) swarp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int t = swarp[lane];
    int y = t;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += u;
    }
    swarp[lane] = y - t;  // exclusive over warps
  }
  __syncthreads();
  return swarp[warp] + x - v;
}

__global__ void __launch_bounds__(kLiveBlock) k_live_count(Work w, int F, int mode, int k1) {
  __shared__ int scount;
  const int j0 = (blockIdx.x * kLiveBlock + threadIdx.x) * kLivePer;
  if (threadIdx.x == 0) scount = 0;
  __syncthreads();
  int c = __popc(live_bits(w, j0, F, mode, k1));
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&scount, c);
  __syncthreads();
  if (threadIdx.x == 0) w.live_bcount[blockIdx.x] = scount;
}

// Exclusive scan of the per-block counts (one block); the total goes to scratch header word 2.
__global__ void __launch_bounds__(1024) k_live_scan(Work w, int nb) {
  __shared__ int swarp[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? w.live_bcount[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) swarp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int y = swarp[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      swarp[lane] = y;  // inclusive over warps
    }
    __syncthreads();
    const int before = carry + (warp > 0 ? swarp[warp - 1] : 0) + x - v;
    if (i < nb) w.live_bcount[i] = before;
    __syncthreads();
    if (threadIdx.x == 1023) carry = before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) w.scr_hdr[2] = carry;
}

__global__ void __launch_bounds__(kLiveBlock) k_live_write(Work w, int F, int mode, int k1) {
  __shared__ int swarp[32];
  const int j0 = (blockIdx.x * kLiveBlock + threadIdx.x) * kLivePer;
  const int bits = live_bits(w, j0, F, mode, k1);
  int pos = w.live_bcount[blockIdx.x] + block_excl_scan(__popc(bits), swarp);
#pragma unroll
  for (int e = 0; e < kLivePer; ++e)
    if (bits & (1 << e)) w.live_slot[pos++] = j0 + e;
}

// First list position whose forward position is >= x.
MLPS_DEV int live_lower_bound(const int* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Per primitive: its range of live intervals and (scan over the primitives, one block) its first
// chunk; the chunk total goes to scratch header word 1. With `count`, the list's intervals are
// added to scratch header word 3 (the forward's evaluated intervals).
__global__ void __launch_bounds__(1024) k_live_prims(Work w, int count) {
  __shared__ int swarp[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_live = w.scr_hdr[2];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < w.K; base += 1024) {
    const int p = base + threadIdx.x;
    int cnt = 0, ch = 0;
    if (p < w.K) {
      const int s0 = live_lower_bound(w.live_slot, n_live, w.prim_start[p]);
      const int s1 = live_lower_bound(w.live_slot, n_live, w.prim_start[p] + w.prim_count[p]);
      cnt = s1 - s0;
      ch = (cnt + w.ipc - 1) / w.ipc;
      w.live_prim_start[p] = s0;
      w.live_prim_count[p] = cnt;
    }
    int x = ch;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) swarp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int y = swarp[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += u;
      }
      swarp[lane] = y;
    }
    __syncthreads();
    const int before = carry + (warp > 0 ? swarp[warp - 1] : 0) + x - ch;
    if (p < w.K) w.live_chunk_start[p] = before;
    __syncthreads();
    if (threadIdx.x == 1023) carry = before + ch;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.live_chunk_start[w.K] = carry;
    w.live_prim_start[w.K] = n_live;
    w.scr_hdr[1] = carry;
    if (count) w.scr_hdr[3] += n_live;
  }
}

// After the first depth wave: a ray stays open when it has hits past its first k1 and the
// composite would not have stopped within them. The optical depth is summed in the composite's
// own order with its own operations, and it only grows along the ray, so "T < t_eps after the
// first k1 intervals" holds exactly when the composite stops at or before interval k1.
__global__ void k_wave_alive(Work w, int k1) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= w.n_rays || r >= live_rays(w)) return;
  const int n = w.ray_count[r], s = w.ray_start[r];
  float A = 0.f;
  for (int j = 0; j < n && j < k1; ++j) A += w.hit_out[s + j].w;
  w.ray_alive[r] = (n > k1 && !(expf(-A) < w.t_eps)) ? 1 : 0;
}

void launch_live_lists(const Work& w, int F, int mode, int k1, cudaStream_t st) {
  const int nb = (w.hit_cap + kLiveBlock * kLivePer - 1) / (kLiveBlock * kLivePer);
  k_live_count<<<nb, kLiveBlock, 0, st>>>(w, F, mode, k1);
  k_live_scan<<<1, 1024, 0, st>>>(w, nb);
  k_live_write<<<nb, kLiveBlock, 0, st>>>(w, F, mode, k1);
  k_live_prims<<<1, 1024, 0, st>>>(w, mode != 0);
}

void launch_wave_alive(const Work& w, int k1, cudaStream_t st) {
  if (w.n_rays == 0) return;
  k_wave_alive<<<(w.n_rays + 255) / 256, 256, 0, st>>>(w, k1);
}

void launch_pose_bwd(const Work& w, float* d_centers, float* d_scales, float* d_quats,
                     cudaStream_t st) {
  if (w.K == 0) return;
  k_pose_bwd<<<(w.K + 127) / 128, 128, 0, st>>>(w, d_centers, d_scales, d_quats);
}

}  // namespace mlps
