// simt_common.cuh -- helpers shared by the FP32 (SIMT) MLP forward and backward kernels:
// chunk bookkeeping, interval tables, sample encoding and the register-tiled FP32 layers.
#pragma once

#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

namespace mlps {
namespace simt {

constexpr int kThreads = 256;
constexpr int kRows = 128;

MLPS_HD int round4(int x) { return (x + 3) & ~3; }

struct IntervalInfo {
  int h;
  float p[3];
  float r0, dt;
  float dp[3];
  float d[3];
  float tmid, r1;
};

MLPS_DEV void stage_f4(float* dst, const float* src, int count) {
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < count / 4; i += blockDim.x) d[i] = __ldg(s + i);
}

// Y[c][r] = act(b[c] + sum_k X[k][r] Wt[k][c]) for dout = 8 * TN columns, 128 rows.
template <int TN>
MLPS_DEV void dense_layer(const float* __restrict__ X, int din, const float* __restrict__ Wt,
                          const float* __restrict__ b, float* __restrict__ Y, bool relu) {
  constexpr int DOUT = 8 * TN;
  const int cg = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = cg * TN, r0 = lane * 4;
  float acc[4][TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const float bj = b[c0 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][j] = bj;
  }
#pragma unroll 2
  for (int k = 0; k < din; ++k) {
    const float4 xv = *reinterpret_cast<const float4*>(&X[k * kRows + r0]);
    const float xr[4] = {xv.x, xv.y, xv.z, xv.w};
    float wr[TN];
#pragma unroll
    for (int j4 = 0; j4 < TN / 4; ++j4) {
      const float4 wv = *reinterpret_cast<const float4*>(&Wt[k * DOUT + c0 + 4 * j4]);
      wr[4 * j4] = wv.x; wr[4 * j4 + 1] = wv.y; wr[4 * j4 + 2] = wv.z; wr[4 * j4 + 3] = wv.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(xr[i], wr[j], acc[i][j]);
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    float4 o = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
    if (relu) { o.x = fmaxf(o.x, 0.f); o.y = fmaxf(o.y, 0.f); o.z = fmaxf(o.z, 0.f); o.w = fmaxf(o.w, 0.f); }
    *reinterpret_cast<float4*>(&Y[(c0 + j) * kRows + r0]) = o;
  }
}

// Small output layer (dout not a multiple of 8): one dot product per (row, column).
MLPS_DEV void dense_small(const float* __restrict__ X, int din, const float* __restrict__ Wt,
                          const float* __restrict__ b, int dout, float* __restrict__ Y) {
  for (int i = threadIdx.x; i < kRows * dout; i += blockDim.x) {
    const int r = i % kRows, o = i / kRows;
    float acc = b[o];
    for (int k = 0; k < din; ++k) acc = fmaf(X[k * kRows + r], Wt[k * dout + o], acc);
    Y[o * kRows + r] = acc;
  }
}

template <int TN>
MLPS_DEV void run_layer(const Model& m, int l, const float* X, const float* Wt, const float* b,
                        float* Y) {
  if (l < m.nl - 1) dense_layer<TN>(X, m.din[l], Wt, b, Y, true);
  else dense_small(X, m.din[l], Wt, b, m.dout[l], Y);
}

// gamma (Eq. 5) of one 3-vector with L frequencies (raw when L = 0) into rows f.. of column
// `row` of X ([feature][stride]); returns the next free feature row.
MLPS_DEV int encode_vec(int L, const float v[3], float* X, int row, int stride, int f) {
  if (L == 0) {
    for (int c = 0; c < 3; ++c) X[(f++) * stride + row] = v[c];
    return f;
  }
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < L; ++l) {
      float s, co;
      sincospif(ldexpf(v[c], l), &s, &co);
      X[(f++) * stride + row] = s;
      X[(f++) * stride + row] = co;
    }
  return f;
}

// Encoding of one sample into column `row` of X ([feature][stride]): gamma(x') then gamma(d)
// (Eq. 5), or in contact-point mode gamma(d) then gamma(delta) (Eq. 4), `xl` holding delta.
MLPS_DEV void encode_row(const Model& m, const float xl[3], const float d[3], float* X, int row,
                         int stride = kRows) {
  if (m.contact) {
    const int f = m.dirL > 0 ? encode_vec(m.dirL, d, X, row, stride, 0) : 0;
    encode_vec(m.xyzL, xl, X, row, stride, f);
    return;
  }
  const int f = encode_vec(m.xyzL, xl, X, row, stride, 0);
  if (m.dirL > 0) encode_vec(m.dirL, d, X, row, stride, f);
}

// Contact-point residual delta = mu - p* with p* = o + max(0, t_mid) d (Eq. 3), from the
// interval's closest point p = M (o + t_mid d - mu) in the normalised frame: R S p is the world
// offset o + t_mid d - mu, so delta = -R S p + min(t_mid, 0) d, free of the cancellation of
// mu - o - t* d.
MLPS_DEV void contact_residual(const PrimGeo& G, const float p[3], float tmid, const float d[3],
                               float delta[3]) {
  const float tn = fminf(tmid, 0.f);
  for (int q = 0; q < 3; ++q) {
    const float y = G.R[q * 3] * G.s[0] * p[0] + G.R[q * 3 + 1] * G.s[1] * p[1] + G.R[q * 3 + 2] * G.s[2] * p[2];
    delta[q] = fmaf(tn, d[q], -y);
  }
}

MLPS_DEV float sigmoidf_acc(float z) { return 1.0f / (1.0f + expf(-z)); }
MLPS_DEV float softplusf_acc(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// Fill one entry of a chunk's interval table from its record (slot in primitive order).
MLPS_DEV void load_interval(const Work& w, const Model& m, int slot, IntervalInfo& I) {
  (void)m;
  const IntervalRec& r = w.rec[slot];
  I.h = r.h;
  for (int i = 0; i < 3; ++i) {
    I.d[i] = r.d[i];
    I.dp[i] = r.dp[i];
    I.p[i] = r.p[i];
  }
  I.tmid = r.tmid;
  I.r0 = r.r0;
  I.r1 = r.r1;
  I.dt = r.dt;
}

MLPS_DEV int find_prim(const Work& w, int c) {
  int lo = 0, hi = w.K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.chunk_start[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}


}  // namespace simt
}  // namespace mlps
