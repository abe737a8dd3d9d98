// k_mlp_simt.cu -- FP32 path of the grouped per-primitive MLP (true FP32 FMA, no TF32).
//
// Work unit: one "chunk" = up to `ipc` hit intervals of ONE primitive, expanded into ipc * S
// sample rows (S midpoint samples per interval, App. D.1), 128 rows per chunk. Persistent
// blocks take contiguous ranges of the global chunk list (primitive-major), so a block keeps
// the same primitive's weights in shared memory over many chunks.
//
// Per chunk:
//  1. sample placement: x'_k = p + (r0 + (k + 1/2) Delta) d' in the primitive's normalised
//     frame (p = closest point o' + t_mid d', r0 = t0 - t_mid, Delta = (t1 - t0) / S);
//  2. encoding gamma of Eq. 5 (sin/cos of 2^l pi p, per scalar) into shared memory;
//  3. the MLP: register-tiled FP32 GEMMs (4 rows x dout/8 columns per thread), ReLU between;
//  4. activations (sigmoid colour, softplus density) and the front-to-back composite of the
//     interval's S samples (Eq. 6): the interval's partial colour C_j = sum_k T_k alpha_k c_k
//     (T_k within the interval) and its optical depth a_j = sum_k sigma_k Delta. The per-ray
//     composite over intervals happens in k_composite.cu; because an interval's samples are
//     contiguous in the ray's order, this split is exact.
// The backward kernel recomputes the forward (no stored activations), reverses the interval
// composite, back-propagates through the MLP (dgrad + wgrad with per-thread register
// accumulators flushed by atomics once per primitive segment) and chains the sample positions
// back to the primitive's pose.
#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

namespace mlps {

constexpr int kThreads = 256;
constexpr int kRows = 128;

struct IntervalInfo {
  int h;
  float p[3];
  float r0, dt;
  float dp[3];
  float d[3];
  float tmid, r1;
};

struct SimtLayout {
  int wfloats, maxdim;
};

MLPS_HD int round4(int x) { return (x + 3) & ~3; }

static SimtLayout simt_layout(const MlpArgs& a) {
  SimtLayout L;
  const Model& m = a.m;
  int maxl = 0;
  for (int l = 0; l < m.nl; ++l) maxl = max(maxl, round4(m.din[l] * m.dout[l]) + round4(m.dout[l]));
  int total = a.pk.boff[m.nl - 1] + round4(m.dout[m.nl - 1]);
  L.wfloats = a.resident ? total : maxl;
  L.maxdim = max(max(m.nin, m.width), m.nout);
  return L;
}

size_t mlp_simt_smem(const MlpArgs& a, bool backward) {
  SimtLayout L = simt_layout(a);
  size_t f = (size_t)L.wfloats + 2 * (size_t)kRows * L.maxdim;
  if (backward) {
    // activations of every layer + one more gradient buffer + per-row scalars
    size_t acts = 0;
    for (int l = 0; l < a.m.nl; ++l) acts += (size_t)a.m.din[l] * kRows;
    f = (size_t)L.wfloats + acts + 2 * (size_t)kRows * L.maxdim + 8 * kRows;
  }
  return f * sizeof(float) + sizeof(IntervalInfo) * kRows + 64 * sizeof(float);
}

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

// Encoding gamma (Eq. 5) of one sample into column `row` of X ([feature][kRows]).
MLPS_DEV void encode_row(const Model& m, const float xl[3], const float d[3], float* X, int row) {
  int f = 0;
  if (m.xyzL == 0) {
    for (int c = 0; c < 3; ++c) X[(f++) * kRows + row] = xl[c];
  } else {
    for (int c = 0; c < 3; ++c)
      for (int l = 0; l < m.xyzL; ++l) {
        float s, co;
        sincospif(ldexpf(xl[c], l), &s, &co);
        X[(f++) * kRows + row] = s;
        X[(f++) * kRows + row] = co;
      }
  }
  if (m.dirL > 0)
    for (int c = 0; c < 3; ++c)
      for (int l = 0; l < m.dirL; ++l) {
        float s, co;
        sincospif(ldexpf(d[c], l), &s, &co);
        X[(f++) * kRows + row] = s;
        X[(f++) * kRows + row] = co;
      }
}

MLPS_DEV float sigmoidf_acc(float z) { return 1.0f / (1.0f + expf(-z)); }
MLPS_DEV float softplusf_acc(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// Fill the chunk's interval table (one thread per interval).
MLPS_DEV void load_interval(const Work& w, const Model& m, int prim, int h, IntervalInfo& I) {
  const int ray = w.hit_ray[h];
  const int hw = w.H * w.W;
  const int v = ray / hw, pix = ray - v * hw;
  const int y = pix / w.W, x = pix - y * w.W;
  float d[3];
  ray_dir_f(w.views[v], x, y, d);
  const PrimGeo& g = w.geo[prim];
  I.h = h;
  for (int i = 0; i < 3; ++i) {
    I.d[i] = d[i];
    I.dp[i] = g.Mhi[i * 3] * d[0] + g.Mhi[i * 3 + 1] * d[1] + g.Mhi[i * 3 + 2] * d[2];
    I.p[i] = w.hit_p[(size_t)i * w.hit_cap + h];
  }
  I.tmid = w.hit_tmid[h];
  I.r0 = w.hit_r0[h];
  I.r1 = w.hit_r1[h];
  I.dt = (I.r1 - I.r0) / (float)m.S;
}

MLPS_DEV int find_prim(const Work& w, int c) {
  int lo = 0, hi = w.K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.chunk_start[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------------------------------
// Forward

template <int TN>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_fwd_simt(Work w, MlpArgs a) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const Model& m = a.m;
  const SimtLayout L = {a.resident ? a.pk.boff[m.nl - 1] + round4(m.dout[m.nl - 1]) : 0, max(max(m.nin, m.width), m.nout)};
  int wfl = L.wfloats;
  if (!a.resident)
    for (int l = 0; l < m.nl; ++l) wfl = max(wfl, round4(m.din[l] * m.dout[l]) + round4(m.dout[l]));
  float* sW = smem;
  float* sA = sW + wfl;
  float* sB = sA + kRows * L.maxdim;
  IntervalInfo* sI = reinterpret_cast<IntervalInfo*>(sB + kRows * L.maxdim);

  const int total = w.saved_hdr[2];
  const int cb = (int)((long long)total * blockIdx.x / gridDim.x);
  const int ce = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  if (cb >= ce) return;
  int prim = find_prim(w, cb);
  int loaded = -1;
  const int S = m.S;
  const float* wbase = reinterpret_cast<const float*>(a.weights);
  const int wstride = (int)(a.pk.stride / 4);
  for (int c = cb; c < ce; ++c) {
    while (c >= w.chunk_start[prim + 1]) ++prim;
    const int first = (c - w.chunk_start[prim]) * w.ipc;
    const int nint = min(w.ipc, w.prim_count[prim] - first);
    __syncthreads();
    if (a.resident && prim != loaded) {
      stage_f4(sW, wbase + (size_t)prim * wstride, wfl);
      loaded = prim;
    }
    if (threadIdx.x < nint)
      load_interval(w, m, prim, w.prim_list[w.prim_start[prim] + first + threadIdx.x], sI[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x < kRows) {
      const int row = threadIdx.x, i = row / S, k = row - i * S;
      if (i < nint) {
        const IntervalInfo& I = sI[i];
        const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
        float xl[3];
        for (int q = 0; q < 3; ++q) xl[q] = fmaf(tr, I.dp[q], I.p[q]);
        encode_row(m, xl, I.d, sA, row);
      } else {
        for (int f = 0; f < m.nin; ++f) sA[f * kRows + row] = 0.f;
      }
    }
    __syncthreads();
    float* X = sA;
    float* Y = sB;
    for (int l = 0; l < m.nl; ++l) {
      const float* Wt;
      const float* bb;
      if (a.resident) {
        Wt = sW + a.pk.woff[l];
        bb = sW + a.pk.boff[l];
      } else {
        const int n = a.pk.boff[l] + round4(m.dout[l]) - a.pk.woff[l];
        stage_f4(sW, wbase + (size_t)prim * wstride + a.pk.woff[l], n);
        __syncthreads();
        Wt = sW;
        bb = sW + (a.pk.boff[l] - a.pk.woff[l]);
      }
      run_layer<TN>(m, l, X, Wt, bb, Y);
      __syncthreads();
      float* t = X; X = Y; Y = t;
    }
    if (threadIdx.x < nint) {
      const IntervalInfo& I = sI[threadIdx.x];
      const int r0 = threadIdx.x * S;
      float A = 0.f, C[3] = {0.f, 0.f, 0.f};
      float Fv[kMaxFeat];
      for (int f = 0; f < m.F; ++f) Fv[f] = 0.f;
      for (int k = 0; k < S; ++k) {
        const int row = r0 + k;
        const float sig = softplusf_acc(X[3 * kRows + row]);
        const float aa = sig * I.dt;
        const float wgt = expf(-A) * -expm1f(-aa);
        for (int q = 0; q < 3; ++q) C[q] = fmaf(wgt, sigmoidf_acc(X[q * kRows + row]), C[q]);
        for (int f = 0; f < m.F; ++f) Fv[f] = fmaf(wgt, X[(4 + f) * kRows + row], Fv[f]);
        A += aa;
      }
      w.hit_out[I.h] = make_float4(C[0], C[1], C[2], A);
      for (int f = 0; f < m.F; ++f) w.hit_feat[(size_t)I.h * m.F + f] = Fv[f];
    }
  }
}

cudaError_t launch_mlp_fwd_simt(const Work& w, const MlpArgs& a, int n_sm, cudaStream_t st) {
  const size_t smem = mlp_simt_smem(a, false);
  const int grid = n_sm;
  switch (a.m.width) {
#define MLPS_CASE(WID)                                                                      \
  case WID: {                                                                               \
    auto kern = k_mlp_fwd_simt<WID / 8>;                                                    \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                        \
    if (e != cudaSuccess) return e;                                                         \
    kern<<<grid, kThreads, smem, st>>>(w, a);                                               \
    return cudaGetLastError();                                                              \
  }
    MLPS_CASE(32)
    MLPS_CASE(64)
    MLPS_CASE(128)
#undef MLPS_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mlp_bwd_simt(const Work& w, const MlpArgs& a, int n_sm, cudaStream_t st) {
  (void)w; (void)a; (void)n_sm; (void)st;
  return cudaErrorNotSupported;
}

}  // namespace mlps
