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
#include "simt_common.cuh"

namespace mlps {

using namespace simt;

struct SimtLayout {
  int wfloats, maxdim;
};

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

  const int total = walk_chunk_count(w);  // (a depth wave's lists, or every chunk)
  const int* const bmap = walk_map(w);    // list position -> primitive-major position
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
      load_interval(w, m, walk_slot(bmap, w.prim_start[prim] + first + threadIdx.x), sI[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x < kRows) {
      const int row = threadIdx.x, i = row / S, k = row - i * S;
      if (i < nint) {
        const IntervalInfo& I = sI[i];
        const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
        float xl[3];
        if (m.contact) contact_residual(w.geo[prim], I.p, I.tmid, I.d, xl);
        else for (int q = 0; q < 3; ++q) xl[q] = fmaf(tr, I.dp[q], I.p[q]);
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

}  // namespace mlps
