// k_mlp_simt_bwd.cu -- FP32 backward of the grouped per-primitive MLP stage.
//
// For every chunk of hit intervals of one primitive (64 sample rows per sub-chunk):
//  1. recompute the forward (encoding, layers) and keep every layer's input in shared memory;
//  2. reverse the interval composite of Eq. 6 with a warp per interval: given the interval's
//     dL/dC_j and dL/da_j from the per-ray reverse pass, with tau_k the transmittance inside
//     the interval, w_k = tau_k alpha_k and R_k = sum_{m>k} w_m c_m,
//       dL/dc_k = w_k dL/dC_j,
//       dL/da_k = dL/dC_j . (tau_k e^{-a_k} c_k - R_k) + dL/da_j,   a_k = sigma_k Delta
//     (features likewise), then through sigmoid / softplus;
//  3. back-propagate through the layers: dgrad (register-tiled FP32 FMA, ReLU masks from the
//     stored activations) and wgrad (each thread owns up to four 4x4 weight-gradient tiles in
//     registers for the whole primitive segment; flushed with one atomicAdd per entry when the
//     block moves to another primitive);
//  4. chain dL/dx'_k (through the encoding derivative) to the primitive pose. With
//     y_k = R S x'_k the sample's offset from the centre, the closest point p, a = |d'|^2 and
//     h the half chord in t:
//       dL/dM  = sum_k g_k y_k^T + g_o' y_mid^T - (g_tm p / a + g_h h d' / a) d^T,
//       dL/dmu = -M^T (sum_k g_k + g_o'),      g_o' = -g_tm d' / a - g_h p / (a h),
//     where g_tm, g_h are the gradients on t_mid and h collected from t_k = t0 + (k + 1/2) Delta
//     and Delta = (t1 - t0) / S. This form has no cancellation between the ~3-unit camera
//     distances; it is the same derivative as the one written with o' and d'.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "mlps_common.cuh"
#include "mlps_kernels.h"
#include "simt_common.cuh"

namespace mlps {

using namespace simt;

namespace {

constexpr int kRB = 64;          // sample rows per sub-chunk
constexpr int kRS = kRB + 4;     // row stride of [feature][row] buffers (bank spread)
constexpr int kMaxTiles = 4;     // 4x4 weight-gradient tiles per thread
constexpr int kMaxBias = 3;

struct BwdPlan {
  int wt_floats;                 // packed W^T + b (resident)
  int wc_off[kMaxLayers];        // canonical W [dout][din] per layer in shared memory
  int wc_floats;
  int act_off[kMaxLayers];       // input of layer l: [din_pad][kRS]
  int din_pad[kMaxLayers], dout_pad[kMaxLayers];
  int act_floats;
  int gbuf;                      // one gradient buffer [maxpad][kRS]
  int zbuf;                      // the forward output [round4(nout)][kRS]
  int nxyz;                      // encoded local-position (contact mode: residual) features
  int x0;                        // their first input row (after the direction in contact mode)
  int tiles;                     // total 4x4 tiles over all layers
  int tile_base[kMaxLayers + 1];
  int ni[kMaxLayers];            // input tiles per layer (ceil(din / 4))
  int bias_base[kMaxLayers + 1];
};

BwdPlan make_plan(const MlpArgs& a) {
  BwdPlan P;
  const Model& m = a.m;
  P.wt_floats = a.pk.boff[m.nl - 1] + round4(m.dout[m.nl - 1]);
  int off = 0, act = 0, maxpad = 0, tiles = 0, bias = 0;
  for (int l = 0; l < m.nl; ++l) {
    P.wc_off[l] = off;
    off += round4(m.din[l] * m.dout[l]);
    P.din_pad[l] = round4(m.din[l]);
    P.dout_pad[l] = round4(m.dout[l]);
    P.act_off[l] = act;
    act += P.din_pad[l] * kRS;
    maxpad = max(maxpad, max(P.din_pad[l], P.dout_pad[l]));
    P.tile_base[l] = tiles;
    P.ni[l] = P.din_pad[l] / 4;
    tiles += (P.dout_pad[l] / 4) * P.ni[l];
    P.bias_base[l] = bias;
    bias += m.dout[l];
  }
  P.tile_base[m.nl] = tiles;
  P.bias_base[m.nl] = bias;
  P.wc_floats = off;
  P.act_floats = act;
  P.gbuf = maxpad * kRS;
  P.zbuf = round4(m.nout) * kRS;
  P.nxyz = m.xyzL > 0 ? 6 * m.xyzL : 3;
  P.x0 = m.contact && m.dirL > 0 ? 6 * m.dirL : 0;
  P.tiles = tiles;
  return P;
}

size_t bwd_smem(const MlpArgs& a, const BwdPlan& P) {
  const Model& m = a.m;
  size_t f = (size_t)P.wt_floats + P.wc_floats + P.act_floats + 2 * (size_t)P.gbuf + P.zbuf;
  f += 16;  // geometry accumulators
  const int ipcb = kRB / m.S;
  size_t bytes = f * sizeof(float) + (size_t)ipcb * (sizeof(IntervalInfo) + sizeof(float4)) +
                 (size_t)ipcb * m.F * sizeof(float) + 64;
  return bytes;
}

// Y[c][r] = act(b[c] + sum_k X[k][r] Wt[k][c]), dout = 8 * TN, 64 rows (2 per lane); the rows
// of Wt are WS floats apart.
template <int TN, int WS = 8 * TN>
MLPS_DEV void fwd_layer(const float* __restrict__ X, int din, const float* __restrict__ Wt,
                        const float* __restrict__ b, float* __restrict__ Y, bool relu) {
  static_assert(WS % 4 == 0 && WS >= 8 * TN, "weight rows are read as float4");
  const int cg = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = cg * TN, r0 = lane * 2;
  float acc[2][TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) { acc[0][j] = b[c0 + j]; acc[1][j] = b[c0 + j]; }
#pragma unroll 2
  for (int k = 0; k < din; ++k) {
    const float2 xv = *reinterpret_cast<const float2*>(&X[k * kRS + r0]);
    float wr[TN];
#pragma unroll
    for (int j4 = 0; j4 < TN / 4; ++j4) {
      const float4 wv = *reinterpret_cast<const float4*>(&Wt[k * WS + c0 + 4 * j4]);
      wr[4 * j4] = wv.x; wr[4 * j4 + 1] = wv.y; wr[4 * j4 + 2] = wv.z; wr[4 * j4 + 3] = wv.w;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[0][j] = fmaf(xv.x, wr[j], acc[0][j]);
      acc[1][j] = fmaf(xv.y, wr[j], acc[1][j]);
    }
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    float2 o = make_float2(acc[0][j], acc[1][j]);
    if (relu) { o.x = fmaxf(o.x, 0.f); o.y = fmaxf(o.y, 0.f); }
    *reinterpret_cast<float2*>(&Y[(c0 + j) * kRS + r0]) = o;
  }
}

MLPS_DEV void fwd_small(const float* __restrict__ X, int din, const float* __restrict__ Wt,
                        const float* __restrict__ b, int dout, float* __restrict__ Y) {
  for (int i = threadIdx.x; i < kRB * dout; i += blockDim.x) {
    const int r = i % kRB, o = i / kRB;
    float acc = b[o];
    for (int k = 0; k < din; ++k) acc = fmaf(X[k * kRS + r], Wt[k * dout + o], acc);
    Y[o * kRS + r] = acc;
  }
}

// G[i][r] = sum_o Wc[o][i] D[o][r], masked by act[i][r] > 0; din = 8 * TN; the rows of Wc are
// WS floats apart.
template <int TN, int WS = 8 * TN>
MLPS_DEV void dgrad_layer(const float* __restrict__ D, int dout, const float* __restrict__ Wc,
                          const float* __restrict__ act, float* __restrict__ G) {
  static_assert(WS % 4 == 0 && WS >= 8 * TN, "weight rows are read as float4");
  const int cg = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = cg * TN, r0 = lane * 2;
  float acc[2][TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) { acc[0][j] = 0.f; acc[1][j] = 0.f; }
#pragma unroll 2
  for (int o = 0; o < dout; ++o) {
    const float2 dv = *reinterpret_cast<const float2*>(&D[o * kRS + r0]);
    float wr[TN];
#pragma unroll
    for (int j4 = 0; j4 < TN / 4; ++j4) {
      const float4 wv = *reinterpret_cast<const float4*>(&Wc[o * WS + c0 + 4 * j4]);
      wr[4 * j4] = wv.x; wr[4 * j4 + 1] = wv.y; wr[4 * j4 + 2] = wv.z; wr[4 * j4 + 3] = wv.w;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[0][j] = fmaf(dv.x, wr[j], acc[0][j]);
      acc[1][j] = fmaf(dv.y, wr[j], acc[1][j]);
    }
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const float2 av = *reinterpret_cast<const float2*>(&act[(c0 + j) * kRS + r0]);
    float2 o = make_float2(av.x > 0.f ? acc[0][j] : 0.f, av.y > 0.f ? acc[1][j] : 0.f);
    *reinterpret_cast<float2*>(&G[(c0 + j) * kRS + r0]) = o;
  }
}

// First-layer input gradient, local-position part only: G[f][r] for f < nx.
// G[f][r] = sum_o Wc[o][x0 + f] D[o][r] for the nx encoded position (or residual) features:
// each lane owns two rows, each warp every 8th feature, up to 8 features per pass in registers.
MLPS_DEV void dgrad_input(const float* __restrict__ D, int dout, const float* __restrict__ Wc,
                          int din, int x0, int nx, float* __restrict__ G) {
  constexpr int kCols = 8;
  const int cg = threadIdx.x >> 5, lane = threadIdx.x & 31, r0 = lane * 2;
  const int ng = blockDim.x >> 5;
  for (int f0 = cg; f0 < nx; f0 += ng * kCols) {
    float acc[2][kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) acc[0][j] = acc[1][j] = 0.f;
    for (int o = 0; o < dout; ++o) {
      const float2 dv = *reinterpret_cast<const float2*>(&D[o * kRS + r0]);
      const float* wrow = Wc + o * din + x0;
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        const int f = f0 + j * ng;
        const float wv = f < nx ? wrow[f] : 0.f;
        acc[0][j] = fmaf(dv.x, wv, acc[0][j]);
        acc[1][j] = fmaf(dv.y, wv, acc[1][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      const int f = f0 + j * ng;
      if (f < nx) *reinterpret_cast<float2*>(&G[f * kRS + r0]) = make_float2(acc[0][j], acc[1][j]);
    }
  }
}

MLPS_DEV float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

MLPS_DEV float warp_excl_scan(float v, int lane) {
  float incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  return incl - v;
}

MLPS_DEV float warp_excl_suffix(float v, int lane) {  // sum over higher lanes
  float incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_down_sync(0xffffffffu, incl, o);
    if (lane + o < 32) incl += u;
  }
  return incl - v;
}

// Per-interval sums of the chain from the encoded inputs to the pose: sum_k g_k, sum_k g_k y_k^T,
// the t0 / t1 weights of the sample positions (midpoint mode), and dL/d delta (contact mode).
struct ChainAcc {
  float sg[3], gy[9], gt0, gt1, gdel[3];
};

MLPS_DEV void chain_zero(ChainAcc& c) {
  for (int q = 0; q < 3; ++q) c.sg[q] = c.gdel[q] = 0.f;
  for (int e = 0; e < 9; ++e) c.gy[e] = 0.f;
  c.gt0 = c.gt1 = 0.f;
}

// d gamma(v) / d v applied to rows [f0, f0 + 6 L) (or 3 raw rows) of column `col` of D.
MLPS_DEV void encode_grad(int L, const float v[3], const float* D, int col, float g[3]) {
  if (L == 0) {
    for (int q = 0; q < 3; ++q) g[q] = D[q * kRS + col];
    return;
  }
  int f = 0;
  for (int q = 0; q < 3; ++q) {
    g[q] = 0.f;
    for (int l = 0; l < L; ++l) {
      float s_, c_;
      sincospif(ldexpf(v[q], l), &s_, &c_);
      const float wq = 3.14159265358979f * ldexpf(1.f, l);
      g[q] += wq * (D[f * kRS + col] * c_ - D[(f + 1) * kRS + col] * s_);
      f += 2;
    }
  }
}

// Sample k of S (column `col` of D) in midpoint mode: x'_k = p + (r0 + (k + 1/2) Delta) d'.
MLPS_DEV void chain_sample(const Model& m, const PrimGeo& G, const IntervalInfo& I, const float* D,
                           int col, int k, int S, ChainAcc& c) {
  const float u = ((float)k + 0.5f) / (float)S;
  const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
  float xl[3], gx[3];
  for (int q = 0; q < 3; ++q) xl[q] = fmaf(tr, I.dp[q], I.p[q]);
  encode_grad(m.xyzL, xl, D, col, gx);
  // y = R S x' (offset of the sample from the centre, world frame)
  float y[3];
  for (int q = 0; q < 3; ++q)
    y[q] = G.R[q * 3] * G.s[0] * xl[0] + G.R[q * 3 + 1] * G.s[1] * xl[1] + G.R[q * 3 + 2] * G.s[2] * xl[2];
  const float gt = gx[0] * I.dp[0] + gx[1] * I.dp[1] + gx[2] * I.dp[2];
  c.gt0 = fmaf(gt, 1.f - u, c.gt0);
  c.gt1 = fmaf(gt, u, c.gt1);
  for (int q = 0; q < 3; ++q) {
    c.sg[q] += gx[q];
    for (int e = 0; e < 3; ++e) c.gy[q * 3 + e] = fmaf(gx[q], y[e], c.gy[q * 3 + e]);
  }
}

// Contact mode: delta = mu - o - max(0, t_mid) d (Eq. 3), dL/d delta from gamma's derivative.
MLPS_DEV void chain_contact(const Model& m, const PrimGeo& G, const IntervalInfo& I, const float* D,
                            int col, ChainAcc& c) {
  float del[3];
  contact_residual(G, I.p, I.tmid, I.d, del);
  encode_grad(m.xyzL, del, D, col, c.gdel);
}

// The interval's 12 pose-gradient contributions (dL/dM row-major, then dL/dmu) from the summed
// chain, dL/dDelta and the geometry of the interval (the formulas in the file header).
MLPS_DEV void chain_pose(const PrimGeo& G, const IntervalInfo& I, const ChainAcc& c, float dDelta,
                         int S, float out[12]) {
  const float gt1 = c.gt1 + dDelta / (float)S;
  const float gt0 = c.gt0 - dDelta / (float)S;
  const bool clamped = I.r0 != -I.r1;
  // contact mode: t* = t_mid when t_mid > 0 moves p* along d
  const float gtd = I.tmid > 0.f ? -(c.gdel[0] * I.d[0] + c.gdel[1] * I.d[1] + c.gdel[2] * I.d[2]) : 0.f;
  const float gtm = gt1 + (clamped ? 0.f : gt0) + gtd;
  const float gh = gt1 - (clamped ? 0.f : gt0);
  const float aa = I.dp[0] * I.dp[0] + I.dp[1] * I.dp[1] + I.dp[2] * I.dp[2];
  const float hh = I.r1;
  float go[3], ymid[3], cd[3];
  for (int q = 0; q < 3; ++q) {
    go[q] = -gtm * I.dp[q] / aa - (hh > 0.f ? gh * I.p[q] / (aa * hh) : 0.f);
    cd[q] = -(gtm * I.p[q] / aa + gh * hh * I.dp[q] / aa);
  }
  for (int q = 0; q < 3; ++q)
    ymid[q] = G.R[q * 3] * G.s[0] * I.p[0] + G.R[q * 3 + 1] * G.s[1] * I.p[1] + G.R[q * 3 + 2] * G.s[2] * I.p[2];
  for (int q = 0; q < 3; ++q)
    for (int e = 0; e < 3; ++e) out[q * 3 + e] = c.gy[q * 3 + e] + go[q] * ymid[e] + cd[q] * I.d[e];
  // dmu = -M^T (sum g + g_o') (+ dL/d delta in contact mode)
  for (int e = 0; e < 3; ++e) {
    float acc2 = 0.f;
    for (int q = 0; q < 3; ++q) acc2 += G.Mhi[q * 3 + e] * (c.sg[q] + go[q]);
    out[9 + e] = c.gdel[e] - acc2;
  }
}

}  // namespace

// Reverse of the interval composite (the file header's step 2) for the sub-chunk's nint
// intervals: dL/dZ of every sample row into sG0 (rows beyond the intervals zeroed), and
// dL/dDelta of each interval into sGrad[i].w. Thread per interval for S = 1 (tau = 1 and no
// later samples inside the interval), else warp per interval.
MLPS_DEV void reverse_composite(const Model& m, int S, int F, int nint, const IntervalInfo* sI, float4* sGrad,
                                const float* sGF, const float* sZ, float* sG0, int dout_pad_last) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (S == 1 && threadIdx.x < nint) {
    const int i = threadIdx.x;
    const float dt = sI[i].dt;
    const float4 g = sGrad[i];
    const float* gF = sGF + i * F;
    const float zs = sZ[3 * kRS + i];
    const float sig = softplusf_acc(zs);
    const float ak = sig * dt;
    const float ea = expf(-ak);
    const float wk = -expm1f(-ak);
    float cq[3];
    for (int q = 0; q < 3; ++q) cq[q] = sigmoidf_acc(sZ[q * kRS + i]);
    float ga = g.w;
    ga += g.x * (ea * cq[0]) + g.y * (ea * cq[1]) + g.z * (ea * cq[2]);
    for (int f = 0; f < F; ++f) {
      ga += gF[f] * (ea * sZ[(4 + f) * kRS + i]);
      sG0[(4 + f) * kRS + i] = wk * gF[f];
    }
    const float gcs[3] = {g.x, g.y, g.z};
    for (int q = 0; q < 3; ++q) sG0[q * kRS + i] = wk * gcs[q] * cq[q] * (1.f - cq[q]);
    sG0[3 * kRS + i] = ga * dt * sigmoidf_acc(zs);
    sGrad[i].w = ga * sig;  // from here on: dL/dDelta of the interval
  }
  for (int i = warp; i < nint && S > 1; i += kThreads / 32) {
    const IntervalInfo& I = sI[i];
    const float4 g = sGrad[i];
    const float* gF = sGF + i * F;
    const int PL = (S + 31) / 32;
    const int k0 = min(S, lane * PL), k1 = min(S, k0 + PL);
    const int rb = i * S;
    float aloc = 0.f;
    for (int k = k0; k < k1; ++k) aloc += softplusf_acc(sZ[3 * kRS + rb + k]) * I.dt;
    const float A0 = warp_excl_scan(aloc, lane);
    // lane totals of w c and w f for the suffix sums
    float wc[3] = {0.f, 0.f, 0.f};
    float A = A0;
    for (int k = k0; k < k1; ++k) {
      const float ak = softplusf_acc(sZ[3 * kRS + rb + k]) * I.dt;
      const float wk = expf(-A) * -expm1f(-ak);
      for (int q = 0; q < 3; ++q) wc[q] = fmaf(wk, sigmoidf_acc(sZ[q * kRS + rb + k]), wc[q]);
      A += ak;
    }
    float R[3];
    for (int q = 0; q < 3; ++q) R[q] = warp_excl_suffix(wc[q], lane);
    // feature suffix sums (one scan per feature)
    float RFl[kMaxFeat];
    for (int f = 0; f < F; ++f) {
      float v = 0.f;
      float A2 = A0;
      for (int k = k0; k < k1; ++k) {
        const float ak = softplusf_acc(sZ[3 * kRS + rb + k]) * I.dt;
        v = fmaf(expf(-A2) * -expm1f(-ak), sZ[(4 + f) * kRS + rb + k], v);
        A2 += ak;
      }
      RFl[f] = warp_excl_suffix(v, lane);
    }
    // backward over the lane's samples
    float dDelta = 0.f;
    float Aend = A;  // exclusive prefix after the lane's last sample
    for (int k = k1 - 1; k >= k0; --k) {
      const float zs = sZ[3 * kRS + rb + k];
      const float sig = softplusf_acc(zs);
      const float ak = sig * I.dt;
      const float Aex = Aend - ak;
      const float tau = expf(-Aex);
      const float ea = expf(-ak);
      const float wk = tau * -expm1f(-ak);
      float cq[3];
      for (int q = 0; q < 3; ++q) cq[q] = sigmoidf_acc(sZ[q * kRS + rb + k]);
      float ga = g.w;
      ga += g.x * (tau * ea * cq[0] - R[0]) + g.y * (tau * ea * cq[1] - R[1]) +
            g.z * (tau * ea * cq[2] - R[2]);
      for (int f = 0; f < F; ++f) {
        const float fk = sZ[(4 + f) * kRS + rb + k];
        ga += gF[f] * (tau * ea * fk - RFl[f]);
        RFl[f] = fmaf(wk, fk, RFl[f]);
        sG0[(4 + f) * kRS + rb + k] = wk * gF[f];
      }
      const float gcs[3] = {g.x, g.y, g.z};
      for (int q = 0; q < 3; ++q) {
        sG0[q * kRS + rb + k] = wk * gcs[q] * cq[q] * (1.f - cq[q]);
        R[q] = fmaf(wk, cq[q], R[q]);
      }
      sG0[3 * kRS + rb + k] = ga * I.dt * sigmoidf_acc(zs);
      dDelta = fmaf(ga, sig, dDelta);
      Aend = Aex;
    }
    dDelta = warp_sum(dDelta);
    if (lane == 0) sGrad[i].w = dDelta;  // from here on: dL/dDelta of the interval
  }
  // rows beyond the valid intervals carry zero gradient
  for (int i = threadIdx.x; i < m.nout * kRB; i += kThreads) {
    const int r = i % kRB, o = i / kRB;
    if (r >= nint * S) sG0[o * kRS + r] = 0.f;
  }
  for (int i = threadIdx.x; i < (dout_pad_last - m.nout) * kRB; i += kThreads) {
    const int r = i % kRB, o = m.nout + i / kRB;
    sG0[o * kRS + r] = 0.f;
  }
}

// Encoding derivative and pose chain (the file header's step 4) of the sub-chunk's intervals from
// D = dL/d(encoded position or residual) rows [0, nxyz): thread per interval for S = 1 (warp
// sums of the 12 contributions), else warp per interval with a lane per sample; the 12 pose
// contributions are added into sGeo.
MLPS_DEV void pose_step(const Model& m, int S, int nint, const IntervalInfo* sI, const float4* sGrad,
                        const float* D, const PrimGeo& G, float* sGeo) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (S == 1) {
    if (warp * 32 < nint) {
      const int i = threadIdx.x;
      float out[12];
      for (int e = 0; e < 12; ++e) out[e] = 0.f;
      if (i < nint) {
        const IntervalInfo& I = sI[i];
        ChainAcc c;
        chain_zero(c);
        if (m.contact) chain_contact(m, G, I, D, i, c);
        else chain_sample(m, G, I, D, i, 0, 1, c);
        chain_pose(G, I, c, sGrad[i].w, 1, out);
      }
      for (int e = 0; e < 12; ++e) {
        const float v = warp_sum(out[e]);
        if (lane == 0) atomicAdd(&sGeo[e], v);
      }
    }
  } else {
    for (int i = warp; i < nint; i += kThreads / 32) {
      const IntervalInfo& I = sI[i];
      const int rb = i * S;
      ChainAcc c;
      chain_zero(c);
      for (int k = lane; k < S; k += 32) chain_sample(m, G, I, D, rb + k, k, S, c);
      for (int q = 0; q < 3; ++q) c.sg[q] = warp_sum(c.sg[q]);
      for (int e = 0; e < 9; ++e) c.gy[e] = warp_sum(c.gy[e]);
      c.gt0 = warp_sum(c.gt0);
      c.gt1 = warp_sum(c.gt1);
      if (lane == 0) {
        float out[12];
        chain_pose(G, I, c, sGrad[i].w, S, out);
        for (int e = 0; e < 12; ++e) atomicAdd(&sGeo[e], out[e]);
      }
    }
  }
}

// MT: weight-gradient tiles per thread (1, 2 or 4). Models with at most 2 x 256 tiles are
// compiled for two resident blocks per SM, so that one block's barriers overlap the other's work.
template <int TN, int MT>
__global__ void __launch_bounds__(kThreads, MT <= 2 ? 2 : 1) k_mlp_bwd_simt(Work w, MlpArgs a, BwdPlan P) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const Model& m = a.m;
  const int S = m.S, F = m.F, nl = m.nl;
  const int ipcb = kRB / S;
  float* sWt = smem;
  float* sWc = sWt + P.wt_floats;
  float* sAct = sWc + P.wc_floats;
  float* sG0 = sAct + P.act_floats;
  float* sG1 = sG0 + P.gbuf;
  float* sZ = sG1 + P.gbuf;
  float* sGeo = sZ + P.zbuf;  // [0..8] dM, [9..11] dmu
  float4* sGrad = reinterpret_cast<float4*>(sGeo + 16);
  IntervalInfo* sI = reinterpret_cast<IntervalInfo*>(sGrad + ipcb);
  float* sGF = reinterpret_cast<float*>(sI + ipcb);

  const int total = walk_chunk_count(w);
  const int* const bmap = walk_map(w);  // list position -> forward position
  const int cb = (int)((long long)total * blockIdx.x / gridDim.x);
  const int ce = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  if (cb >= ce) return;

  // this thread's weight-gradient tiles
  int t_layer[MT], t_o0[MT], t_it[MT];
  float acc[MT][16];
  float bacc[kMaxBias];
  int nt = 0;
  for (int t = threadIdx.x; t < P.tiles && nt < MT; t += kThreads, ++nt) {
    int l = 0;
    while (t >= P.tile_base[l + 1]) ++l;
    const int loc = t - P.tile_base[l];
    t_layer[nt] = l;
    t_o0[nt] = (loc / P.ni[l]) * 4;
    t_it[nt] = loc % P.ni[l];
  }
  auto zero_acc = [&]() {
#pragma unroll
    for (int j = 0; j < MT; ++j)
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[j][e] = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxBias; ++j) bacc[j] = 0.f;
  };
  zero_acc();
  if (threadIdx.x < 16) sGeo[threadIdx.x] = 0.f;

  const float* wbase = reinterpret_cast<const float*>(a.weights);
  const int wstride = (int)(a.pk.stride / 4);
  int prim = find_prim(w, cb);
  int loaded = -1;

  auto flush = [&](int p) {
    float* dW = a.d_weights + (size_t)p * m.Prow;
#pragma unroll
    for (int j = 0; j < MT; ++j) {
      if (j >= nt) break;
      const int l = t_layer[j], din = m.din[l], dout = m.dout[l], ni = P.ni[l];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int o = t_o0[j] + (e >> 2), i = t_it[j] + ni * (e & 3);
        if (o < dout && i < din && acc[j][e] != 0.f) atomicAdd(&dW[m.woff[l] + o * din + i], acc[j][e]);
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxBias; ++j) {
      const int bi = threadIdx.x + j * kThreads;
      if (bi < P.bias_base[nl] && bacc[j] != 0.f) {
        int l = 0;
        while (bi >= P.bias_base[l + 1]) ++l;
        atomicAdd(&dW[m.boff[l] + (bi - P.bias_base[l])], bacc[j]);
      }
    }
    __syncthreads();
    if (threadIdx.x < 12) {
      const float v = sGeo[threadIdx.x];
      if (v != 0.f) atomicAdd(&w.dgeo[12 * (size_t)p + threadIdx.x], v);
      sGeo[threadIdx.x] = 0.f;
    }
    zero_acc();
  };

  for (int c = cb; c < ce; ++c) {
    while (c >= w.chunk_start[prim + 1]) ++prim;
    const int first = (c - w.chunk_start[prim]) * w.ipc;
    const int nint_c = min(w.ipc, w.prim_count[prim] - first);
    if (prim != loaded) {
      if (loaded >= 0) flush(loaded);
      __syncthreads();
      // W^T blocks (forward) and canonical W (dgrad)
      stage_f4(sWt, wbase + (size_t)prim * wstride, P.wt_floats);
      const float* src = wbase + (size_t)prim * wstride;
      for (int l = 0; l < nl; ++l) {
        const int din = m.din[l], dout = m.dout[l];
        for (int i = threadIdx.x; i < din * dout; i += kThreads) {
          const int o = i / din, k = i - o * din;
          sWc[P.wc_off[l] + i] = src[a.pk.woff[l] + k * dout + o];
        }
      }
      // zero padded activation rows once (rows din..din_pad of every layer input)
      for (int l = 0; l < nl; ++l)
        for (int i = threadIdx.x; i < (P.din_pad[l] - m.din[l]) * kRS; i += kThreads)
          sAct[P.act_off[l] + m.din[l] * kRS + i] = 0.f;
      loaded = prim;
    }
    const PrimGeo& G = w.geo[prim];
    for (int sub = 0; sub * ipcb < nint_c; ++sub) {
      const int i0 = sub * ipcb;
      const int nint = min(ipcb, nint_c - i0);
      __syncthreads();
      if (threadIdx.x < nint) {
        const int slot = walk_slot(bmap, w.prim_start[prim] + first + i0 + threadIdx.x);
        load_interval(w, m, slot, sI[threadIdx.x]);
        sGrad[threadIdx.x] = w.hit_grad[slot];
        for (int f = 0; f < F; ++f) sGF[threadIdx.x * F + f] = w.hit_gfeat[(size_t)slot * F + f];
      }
      __syncthreads();
      // 1. encode the samples into the input of layer 0
      float* X0 = sAct + P.act_off[0];
      if (threadIdx.x < kRB) {
        const int row = threadIdx.x, i = row / S, k = row - i * S;
        if (i < nint) {
          const IntervalInfo& I = sI[i];
          const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
          float xl[3];
          if (m.contact) contact_residual(G, I.p, I.tmid, I.d, xl);
          else for (int q = 0; q < 3; ++q) xl[q] = fmaf(tr, I.dp[q], I.p[q]);
          encode_row(m, xl, I.d, X0, row, kRS);
        } else {
          for (int f = 0; f < m.nin; ++f) X0[f * kRS + row] = 0.f;
        }
      }
      __syncthreads();
      // 2. forward recompute, keeping every layer's input
      for (int l = 0; l < nl; ++l) {
        const float* Xl = sAct + P.act_off[l];
        const float* Wt = sWt + a.pk.woff[l];
        const float* bb = sWt + a.pk.boff[l];
        if (l < nl - 1) fwd_layer<TN>(Xl, m.din[l], Wt, bb, sAct + P.act_off[l + 1], true);
        else fwd_small(Xl, m.din[l], Wt, bb, m.dout[l], sZ);
        __syncthreads();
      }
      // 3. reverse of the interval composite -> dZ in sG0
      reverse_composite(m, S, F, nint, sI, sGrad, sGF, sZ, sG0, P.dout_pad[nl - 1]);
      __syncthreads();
      // 4. layers, last to first: wgrad (+ bias) then dgrad
      float* D = sG0;
      float* Gn = sG1;
      for (int l = nl - 1; l >= 0; --l) {
        const float* Al = sAct + P.act_off[l];
#pragma unroll
        for (int j = 0; j < MT; ++j) {
          if (j >= nt || t_layer[j] != l) continue;
          const int o0 = t_o0[j], it = t_it[j], ni = P.ni[l];
          for (int r = 0; r < kRB; r += 4) {
            float4 dv[4], av[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              dv[u] = *reinterpret_cast<const float4*>(&D[(o0 + u) * kRS + r]);
              av[u] = *reinterpret_cast<const float4*>(&Al[(it + ni * u) * kRS + r]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                float s_ = acc[j][u * 4 + v];
                s_ = fmaf(dv[u].x, av[v].x, s_);
                s_ = fmaf(dv[u].y, av[v].y, s_);
                s_ = fmaf(dv[u].z, av[v].z, s_);
                s_ = fmaf(dv[u].w, av[v].w, s_);
                acc[j][u * 4 + v] = s_;
              }
          }
        }
#pragma unroll
        for (int j = 0; j < kMaxBias; ++j) {
          const int bi = threadIdx.x + j * kThreads - P.bias_base[l];
          if (bi >= 0 && bi < m.dout[l]) {
            float s_ = 0.f;
            for (int r = 0; r < kRB; ++r) s_ += D[bi * kRS + r];
            bacc[j] += s_;
          }
        }
        if (l > 0) {
          dgrad_layer<TN>(D, m.dout[l], sWc + P.wc_off[l], Al, Gn);
        } else {
          dgrad_input(D, m.dout[0], sWc + P.wc_off[0], m.din[0], P.x0, P.nxyz, Gn);
        }
        __syncthreads();
        float* t = D; D = Gn; Gn = t;
      }
      // D now holds dL/d(encoded local position), or dL/d(encoded delta), rows [0, nxyz)
      // 5. encoding derivative and pose chain
      pose_step(m, S, nint, sI, sGrad, D, G, sGeo);
    }
  }
  if (loaded >= 0) flush(loaded);
}

// ------------------------------------------------------------------------------------------
// Wide models (hidden width 128, e.g. 4 x 128 with a feature head). Neither the weight
// gradients (~60 k values per primitive) nor both weight copies fit on chip, so:
//  * each layer's weights are streamed through shared memory, 64 output (forward) or input
//    (dgrad) columns at a time, from the FP32 blob or, for the tensor-core precisions, from the
//    BF16 tiles of their blob (the backward then recomputes with the BF16-rounded weights the
//    forward used). Each thread issues all of its loads of a block before its first store;
//  * dgrad writes delta_{l-1} over H_l in place (each element's ReLU mask is read by the thread
//    that overwrites it), and the encoded input is rebuilt for layer 0's wgrad, so every layer
//    input has one buffer;
//  * the 4 x 4 weight-gradient tiles are accumulated over a sub-chunk in registers and added
//    into a block-private FP32 copy of dW in global memory (L2-resident; a tile's entries are
//    read before its FMA loop), flushed with atomics when the block moves to another primitive.
//    Bias gradients stay in registers as above.

// Row stride of a staged 64-column block of BF16-tile weights: the transposing stores of the
// coalesced reads meet at most 4-way bank conflicts. (FP32-blob blocks keep rows 64 apart.)
constexpr int kWideWS = 68;

struct WidePlan {
  int nl, nin, nout, nx, x0;
  int act_floats;                  // (nl - 1) layer inputs of 128 rows
  int gbuf_rows;                   // encoded input / dL/dZ / dL/dx buffer
  int zrows;                       // forward output rows
  int stage_floats;
  int tile_base[kMaxLayers + 1], ni[kMaxLayers];
  int bias_base[kMaxLayers + 1];
  // weight sources
  int bf16;                        // 1: BF16 tiles of a tensor-core blob
  int gw_row[kMaxLayers], npad[kMaxLayers], bias_off[kMaxLayers], gbias_byte;
};

MLPS_HD int wide_rows(int n) { return round4(n); }

WidePlan make_wide_plan(const MlpArgs& a, const TcPlan* tp) {
  const Model& m = a.m;
  WidePlan P;
  std::memset(&P, 0, sizeof(P));
  P.nl = m.nl;
  P.nin = m.nin;
  P.nout = m.nout;
  P.nx = m.xyzL > 0 ? 6 * m.xyzL : 3;
  P.x0 = m.contact && m.dirL > 0 ? 6 * m.dirL : 0;
  P.act_floats = (m.nl - 1) * m.width * kRS;
  P.gbuf_rows = max(max(wide_rows(m.nin), wide_rows(m.nout)), wide_rows(P.nx));
  P.zrows = wide_rows(m.nout);
  int tiles = 0, bias = 0;
  for (int l = 0; l < m.nl; ++l) {
    P.tile_base[l] = tiles;
    P.ni[l] = wide_rows(m.din[l]) / 4;
    tiles += (wide_rows(m.dout[l]) / 4) * P.ni[l];
    P.bias_base[l] = bias;
    bias += m.dout[l];
  }
  P.tile_base[m.nl] = tiles;
  P.bias_base[m.nl] = bias;
  P.stage_floats = m.width * kWideWS + 64;  // the largest staged block: 128 rows of 64 (+ pad), bias
  if (tp) {
    P.bf16 = 1;
    for (int l = 0; l < m.nl; ++l) {
      P.gw_row[l] = tp->gw_row[l];
      P.npad[l] = tp->npad[l];
      P.bias_off[l] = tp->bias_off[l];
    }
    P.gbias_byte = tp->gbias_byte;
  }
  return P;
}

size_t wide_smem(const MlpArgs& a, const WidePlan& P) {
  const int S = a.m.S;
  const int ipcb = kRB / S;
  size_t f = (size_t)P.stage_floats + P.act_floats + (size_t)(P.gbuf_rows + P.zrows) * kRS + 16;
  return f * sizeof(float) + (size_t)ipcb * (sizeof(IntervalInfo) + sizeof(float4)) +
         (size_t)ipcb * a.m.F * sizeof(float) + 64;
}

// Weight sources of the staged primitive's blob: the FP32 W^T [din][dout] per layer, or the BF16
// tiles (64-wide K blocks of W [npad][64]); b_l[o] from either.
struct WideWeights {
  const unsigned char* blob;
  const float* f32;
  const Packed* pk;
  const WidePlan* P;
  MLPS_DEV float b(int l, int o) const {
    if (P->bf16) return reinterpret_cast<const float*>(blob + P->gbias_byte)[P->bias_off[l] + o];
    return f32[pk->boff[l] + o];
  }
  MLPS_DEV const __nv_bfloat16* tile(int l) const {
    return reinterpret_cast<const __nv_bfloat16*>(blob + (size_t)P->gw_row[l] * 128);
  }
};

// dst[i] = src(i) for i < n <= kWideStageMax, all of a thread's loads before its first store.
constexpr int kWideStageMax = 128 * 64;
template <class Src>
MLPS_DEV void wide_stage_flat(int n, Src src, float* __restrict__ dst) {
  constexpr int kPer = kWideStageMax / kThreads;
  float r[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + j * kThreads;
    r[j] = i < n ? src(i) : 0.f;
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + j * kThreads;
    if (i < n) dst[i] = r[j];
  }
}

// dst[at(a, b)] = src(a, b) over the n elements i = a * d + b (b < d) of a staged block. Element
// i goes to thread i mod 256; (a, b) steps by (256 / d, 256 mod d) from one element of a thread to
// the next, so no thread divides more than once. Every thread issues all of its loads before its
// first store: one staging pass costs one memory round trip rather than one per element.
template <class Src, class At>
MLPS_DEV void wide_stage(int n, int d, Src src, At at, float* __restrict__ dst) {
  constexpr int kPer = kWideStageMax / kThreads;
  const int a0 = threadIdx.x / d, b0 = threadIdx.x - a0 * d;
  const int qa = kThreads / d, qb = kThreads - qa * d;
  float r[kPer];
  int a = a0, b = b0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    r[j] = threadIdx.x + j * kThreads < n ? src(a, b) : 0.f;
    a += qa;
    b += qb;
    if (b >= d) { b -= d; ++a; }
  }
  a = a0;
  b = b0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (threadIdx.x + j * kThreads < n) dst[at(a, b)] = r[j];
    a += qa;
    b += qb;
    if (b >= d) { b -= d; ++a; }
  }
}

// The four staged blocks of the wide backward. FP32 blob: W^T [din][dout] per layer, staged
// with consecutive threads on consecutive shared-memory words (rows WS = 64 apart; the dgrad
// blocks then read the blob with a stride). BF16 blob:
// 64-wide K blocks of W, [npad][64] each, staged with consecutive threads on consecutive global
// addresses (rows WS = 68 apart, so the transposing stores meet at most 4-way bank conflicts).
// Each was the faster of the two mappings for its source in a per-phase cycle count of the
// 4 x 128 model.
template <bool BF16>
struct WideStager {
  static constexpr int WS = BF16 ? kWideWS : 64;
  const WideWeights& W;
  const Model& m;
  const WidePlan& P;
  float* s;
  // Wt[k][c] = W_l[64 h + c][k] (k < din, c < 64) at s[k * WS + c], then 64 biases
  MLPS_DEV void fwd_half(int l, int h) const {
    const int din = m.din[l];
    if constexpr (BF16) {
      const __nv_bfloat16* t = W.tile(l) + (size_t)64 * h * 64;
      const int np64 = P.npad[l] * 64;
      wide_stage(din * 64, din, [&](int c, int k) { return __bfloat162float(t[(k >> 6) * np64 + c * 64 + (k & 63)]); },
                 [&](int c, int k) { return k * WS + c; }, s);
    } else {
      const int dout = m.dout[l];
      const float* f = W.f32 + W.pk->woff[l] + 64 * h;
      wide_stage_flat(din * 64, [&](int i) { return f[(i >> 6) * dout + (i & 63)]; }, s);
    }
    if (threadIdx.x < 64) s[din * WS + threadIdx.x] = W.b(l, 64 * h + threadIdx.x);
  }
  // Wc[o][c] = W_l[o][64 h + c] (o < dout, c < 64) at s[o * WS + c]
  MLPS_DEV void dgrad_half(int l, int h) const {
    const int dout = m.dout[l];
    if constexpr (BF16) {
      const __nv_bfloat16* t = W.tile(l) + (size_t)h * P.npad[l] * 64;
      wide_stage(dout * 64, 64, [&](int o, int c) { return __bfloat162float(t[o * 64 + c]); },
                 [&](int o, int c) { return o * WS + c; }, s);
    } else {
      const float* f = W.f32 + W.pk->woff[l] + (size_t)64 * h * dout;
      wide_stage_flat(dout * 64, [&](int i) { return f[(i & 63) * dout + (i >> 6)]; }, s);
    }
  }
  // the head, compact: Wt[k][o] at s[k * dout + o], then dout biases
  MLPS_DEV void head(int l) const {
    const int din = m.din[l], dout = m.dout[l];
    if constexpr (BF16) {
      const __nv_bfloat16* t = W.tile(l);
      const int np64 = P.npad[l] * 64;
      wide_stage(din * dout, din, [&](int o, int k) { return __bfloat162float(t[(k >> 6) * np64 + o * 64 + (k & 63)]); },
                 [&](int o, int k) { return k * dout + o; }, s);
    } else {
      const float* f = W.f32 + W.pk->woff[l];
      wide_stage_flat(din * dout, [&](int i) { return f[i]; }, s);
    }
    if (threadIdx.x < dout) s[din * dout + threadIdx.x] = W.b(l, threadIdx.x);
  }
  // layer 0's columns of the encoded position features: Wc[o][f] = W_0[o][x0 + f] at s[o * nx + f]
  MLPS_DEV void input_cols() const {
    const int dout = m.dout[0], nx = P.nx, x0 = P.x0;
    if constexpr (BF16) {
      const __nv_bfloat16* t = W.tile(0);
      const int np64 = P.npad[0] * 64;
      wide_stage(dout * nx, nx, [&](int o, int f) { const int k = x0 + f;
                                                    return __bfloat162float(t[(k >> 6) * np64 + o * 64 + (k & 63)]); },
                 [&](int o, int f) { return o * nx + f; }, s);
    } else {
      const float* f = W.f32 + W.pk->woff[0] + (size_t)x0 * dout;
      wide_stage_flat(dout * nx, [&](int i) { const int o = i / nx; return f[(i - o * nx) * dout + o]; }, s);
    }
  }
};

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_bwd_simt_wide(Work w, MlpArgs a, WidePlan P) {
  constexpr int WS = WideStager<BF16>::WS;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const Model& m = a.m;
  const int S = m.S, F = m.F, nl = m.nl;
  const int ipcb = kRB / S;
  float* sStage = smem;
  float* sAct = sStage + P.stage_floats;     // input of layer l >= 1 at (l - 1) * 128 rows
  float* sG = sAct + P.act_floats;           // X, then dL/dZ, then X, then dL/dx
  float* sZ = sG + P.gbuf_rows * kRS;
  float* sGeo = sZ + P.zrows * kRS;
  float4* sGrad = reinterpret_cast<float4*>(sGeo + 16);
  IntervalInfo* sI = reinterpret_cast<IntervalInfo*>(sGrad + ipcb);
  float* sGF = reinterpret_cast<float*>(sI + ipcb);
  auto act = [&](int l) { return sAct + (size_t)(l - 1) * m.width * kRS; };

  const int total = walk_chunk_count(w);
  const int* const bmap = walk_map(w);  // list position -> forward position
  const int cb = (int)((long long)total * blockIdx.x / gridDim.x);
  const int ce = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  if (cb >= ce) return;
  float* dwb = w.dwb + (size_t)blockIdx.x * m.P;  // this block's dW copy (canonical layout)
  float bacc[kMaxBias];
  for (int j = 0; j < kMaxBias; ++j) bacc[j] = 0.f;
  if (threadIdx.x < 16) sGeo[threadIdx.x] = 0.f;
  const int wstride = (int)(a.pk.stride / 4);
  int prim = find_prim(w, cb);
  int loaded = -1;
  WideWeights W{nullptr, nullptr, &a.pk, &P};
  const WideStager<BF16> stage{W, m, P, sStage};

  auto flush = [&](int p) {
    float* dW = a.d_weights + (size_t)p * m.Prow;
    __syncthreads();
    for (int i = threadIdx.x; i < m.P; i += kThreads) {
      const float v = dwb[i];
      if (v != 0.f) {
        atomicAdd(&dW[i], v);
        dwb[i] = 0.f;
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxBias; ++j) {
      const int bi = threadIdx.x + j * kThreads;
      if (bi < P.bias_base[nl] && bacc[j] != 0.f) {
        int l = 0;
        while (bi >= P.bias_base[l + 1]) ++l;
        atomicAdd(&dW[m.boff[l] + (bi - P.bias_base[l])], bacc[j]);
      }
      bacc[j] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
      const float v = sGeo[threadIdx.x];
      if (v != 0.f) atomicAdd(&w.dgeo[12 * (size_t)p + threadIdx.x], v);
      sGeo[threadIdx.x] = 0.f;
    }
  };
  // wgrad of layer l (D: dL/dZ_l rows, H: input rows) over the first `rows` rows of the
  // sub-chunk into dwb, and biases. The tile's dwb entries are read before the FMA loop so that
  // their latency hides under it.
  auto wgrad = [&](int l, const float* D, const float* H, int rows) {
    const int ni = P.ni[l], din = m.din[l], dout = m.dout[l];
    const int n_t = P.tile_base[l + 1] - P.tile_base[l];
    float* dwl = dwb + m.woff[l];
    for (int t = threadIdx.x; t < n_t; t += kThreads) {
      const int o0 = (t / ni) * 4, it = t % ni;
      float acc[16], cur[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int o = o0 + (e >> 2), i = it + ni * (e & 3);
        cur[e] = (o < dout && i < din) ? dwl[o * din + i] : 0.f;
        acc[e] = 0.f;
      }
      for (int r = 0; r < rows; r += 4) {
        float4 dv[4], av[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          dv[u] = *reinterpret_cast<const float4*>(&D[(o0 + u) * kRS + r]);
          av[u] = *reinterpret_cast<const float4*>(&H[(it + ni * u) * kRS + r]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float s_ = acc[u * 4 + v];
            s_ = fmaf(dv[u].x, av[v].x, s_);
            s_ = fmaf(dv[u].y, av[v].y, s_);
            s_ = fmaf(dv[u].z, av[v].z, s_);
            s_ = fmaf(dv[u].w, av[v].w, s_);
            acc[u * 4 + v] = s_;
          }
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int o = o0 + (e >> 2), i = it + ni * (e & 3);
        if (o < dout && i < din && acc[e] != 0.f) dwl[o * din + i] = cur[e] + acc[e];
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxBias; ++j) {
      const int bi = threadIdx.x + j * kThreads - P.bias_base[l];
      if (bi >= 0 && bi < dout) {
        float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int r = 0; r < rows; r += 4) {
          const float4 d = *reinterpret_cast<const float4*>(&D[bi * kRS + r]);
          s4.x += d.x; s4.y += d.y; s4.z += d.z; s4.w += d.w;
        }
        bacc[j] += (s4.x + s4.y) + (s4.z + s4.w);
      }
    }
  };
  // the encoded input of the sub-chunk's rows into sG (rows nin..gbuf_rows zero)
  auto encode = [&](int nint, const PrimGeo& G) {
    if (threadIdx.x < kRB) {
      const int row = threadIdx.x, i = row / S, k = row - i * S;
      if (i < nint) {
        const IntervalInfo& I = sI[i];
        const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
        float xl[3];
        if (m.contact) contact_residual(G, I.p, I.tmid, I.d, xl);
        else for (int q = 0; q < 3; ++q) xl[q] = fmaf(tr, I.dp[q], I.p[q]);
        encode_row(m, xl, I.d, sG, row, kRS);
        for (int f = m.nin; f < P.gbuf_rows; ++f) sG[f * kRS + row] = 0.f;
      } else {
        for (int f = 0; f < P.gbuf_rows; ++f) sG[f * kRS + row] = 0.f;
      }
    }
  };

  for (int c = cb; c < ce; ++c) {
    while (c >= w.chunk_start[prim + 1]) ++prim;
    const int first = (c - w.chunk_start[prim]) * w.ipc;
    const int nint_c = min(w.ipc, w.prim_count[prim] - first);
    if (prim != loaded) {
      if (loaded >= 0) flush(loaded);
      loaded = prim;
    }
    W.blob = a.weights + (size_t)prim * a.pk.stride;
    W.f32 = reinterpret_cast<const float*>(a.weights) + (size_t)prim * wstride;
    const PrimGeo& G = w.geo[prim];
    for (int sub = 0; sub * ipcb < nint_c; ++sub) {
      const int i0 = sub * ipcb;
      const int nint = min(ipcb, nint_c - i0);
      const int rows = round4(nint * S);  // rows past nint * S carry zero dL/dZ
      __syncthreads();
      if (threadIdx.x < nint) {
        const int slot = walk_slot(bmap, w.prim_start[prim] + first + i0 + threadIdx.x);
        load_interval(w, m, slot, sI[threadIdx.x]);
        sGrad[threadIdx.x] = w.hit_grad[slot];
        for (int f = 0; f < F; ++f) sGF[threadIdx.x * F + f] = w.hit_gfeat[(size_t)slot * F + f];
      }
      __syncthreads();
      encode(nint, G);
      // forward recompute, hidden layers in two 64-column halves, then the head
      for (int l = 0; l < nl - 1; ++l) {
        const float* X = l == 0 ? sG : act(l);
        const int din = m.din[l];
        for (int h = 0; h < 2; ++h) {
          __syncthreads();
          stage.fwd_half(l, h);
          __syncthreads();
          fwd_layer<8, WS>(X, din, sStage, sStage + din * WS, act(l + 1) + (size_t)64 * h * kRS, true);
        }
      }
      {
        const int l = nl - 1, din = m.din[l], dout = m.dout[l];
        __syncthreads();
        stage.head(l);
        __syncthreads();
        fwd_small(act(l), din, sStage, sStage + din * dout, dout, sZ);
        __syncthreads();
      }
      // reverse of the interval composite: dL/dZ into sG (the encoded input is rebuilt later)
      reverse_composite(m, S, F, nint, sI, sGrad, sGF, sZ, sG, P.zrows);
      __syncthreads();
      // layers, last to first: wgrad, then dgrad over H_l in place (two 64-column halves)
      for (int l = nl - 1; l >= 1; --l) {
        const float* D = l == nl - 1 ? sG : act(l + 1);
        float* H = act(l);
        const int dout = m.dout[l];
        wgrad(l, D, H, rows);
        for (int h = 0; h < 2; ++h) {
          __syncthreads();
          stage.dgrad_half(l, h);
          __syncthreads();
          dgrad_layer<8, WS>(D, dout, sStage, H + (size_t)64 * h * kRS, H + (size_t)64 * h * kRS);
        }
        __syncthreads();
      }
      // layer 0: rebuild X, wgrad, then dL/dx of the encoded position (or residual) features
      encode(nint, G);
      __syncthreads();
      wgrad(0, act(1), sG, rows);
      __syncthreads();
      stage.input_cols();
      __syncthreads();
      dgrad_input(act(1), m.dout[0], sStage, P.nx, 0, P.nx, sG);
      __syncthreads();
      pose_step(m, S, nint, sI, sGrad, sG, G, sGeo);
    }
  }
  if (loaded >= 0) flush(loaded);
}

bool simt_bwd_wide_supported(const MlpArgs& a) {
  const Model& m = a.m;
  if (m.width != 128 || m.S > kRB || m.nl < 2) return false;
  if (m.nin > 64 || m.nout > 64 || m.F > kMaxFeat) return false;
  WidePlan P = make_wide_plan(a, nullptr);
  if (P.bias_base[m.nl] > kMaxBias * kThreads || P.nx > 64) return false;
  return wide_smem(a, P) <= 227 * 1024;
}

cudaError_t launch_mlp_bwd_simt_wide(const Work& w, const MlpArgs& a, const TcPlan* tp, int n_sm, cudaStream_t st) {
  if (!simt_bwd_wide_supported(a) || !w.dwb) return cudaErrorNotSupported;
  const WidePlan P = make_wide_plan(a, tp);
  const size_t smem = wide_smem(a, P);
  auto kern = P.bf16 ? k_mlp_bwd_simt_wide<true> : k_mlp_bwd_simt_wide<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_sm, kThreads, smem, st>>>(w, a, P);
  return cudaGetLastError();
}

bool simt_bwd_supported(const MlpArgs& a) {
  const Model& m = a.m;
  if (m.S > kRB || (m.width != 32 && m.width != 64)) return false;
  BwdPlan P = make_plan(a);
  if (P.tiles > kMaxTiles * kThreads || P.bias_base[m.nl] > kMaxBias * kThreads) return false;
  for (int l = 0; l < m.nl; ++l)
    if (m.dout[l] % 4 != 0 && l < m.nl - 1) return false;
  return bwd_smem(a, P) <= 227 * 1024;
}

template <int TN, int MT>
static cudaError_t launch_bwd_mt(const Work& w, const MlpArgs& a, const BwdPlan& P, size_t smem, int n_sm,
                                 cudaStream_t st) {
  auto kern = k_mlp_bwd_simt<TN, MT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  kern<<<n_sm * per_sm, kThreads, smem, st>>>(w, a, P);
  return cudaGetLastError();
}

template <int TN>
static cudaError_t launch_bwd_width(const Work& w, const MlpArgs& a, const BwdPlan& P, size_t smem, int n_sm,
                                    cudaStream_t st) {
  if (P.tiles <= kThreads) return launch_bwd_mt<TN, 1>(w, a, P, smem, n_sm, st);
  if (P.tiles <= 2 * kThreads) return launch_bwd_mt<TN, 2>(w, a, P, smem, n_sm, st);
  return launch_bwd_mt<TN, kMaxTiles>(w, a, P, smem, n_sm, st);
}

cudaError_t launch_mlp_bwd_simt(const Work& w, const MlpArgs& a, int n_sm, cudaStream_t st) {
  const Model& m = a.m;
  if (!simt_bwd_supported(a)) return cudaErrorNotSupported;
  BwdPlan P = make_plan(a);
  const size_t smem = bwd_smem(a, P);
  switch (m.width) {
    case 32:
      return launch_bwd_width<4>(w, a, P, smem, n_sm, st);
    case 64:
      return launch_bwd_width<8>(w, a, P, smem, n_sm, st);
    default:
      return cudaErrorNotSupported;
  }
}

}  // namespace mlps
