// k_pack.cu -- conversion of canonical FP32 weights [K, P] into the packed per-primitive blob
// that the MLP kernels stage into shared memory.
//
// FP32 blob: per layer W^T as [din][dout] (so one input feature's weights to all outputs are
// contiguous for the register-tiled FMA loop), then the bias; each block 16-byte aligned.
// Tensor-core blobs (BF16 / FP8) are written by the tensor-core packer in k_mlp_tc.cu.
#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

namespace mlps {

__global__ void k_pack_fp32(Model m, Packed pk, int K, const float* __restrict__ src,
                            float* __restrict__ dst) {
  const int p = blockIdx.y;
  if (p >= K) return;
  const float* s = src + (size_t)p * m.Prow;
  float* d = dst + (size_t)p * (pk.stride / 4);
  const int slot0 = (int)(pk.slot_byte / 4);
  const int total = (int)(pk.stride / 4);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int l = 0; l < m.nl; ++l) {
      const int din = m.din[l], dout = m.dout[l];
      if (i >= pk.woff[l] && i < pk.woff[l] + din * dout) {
        const int r = i - pk.woff[l];
        const int k = r / dout, o = r - k * dout;  // W^T[k][o] = W[o][k]
        v = s[m.woff[l] + o * din + k];
      } else if (i >= pk.boff[l] && i < pk.boff[l] + dout) {
        v = s[m.boff[l] + (i - pk.boff[l])];
      }
    }
    if (m.C > 0 && i >= slot0 && i < slot0 + 4 * m.C) v = s[m.P + (i - slot0)];
    d[i] = v;
  }
}

void launch_pack_fp32(const Model& m, const Packed& pk, int K, const float* w, void* out,
                      cudaStream_t st) {
  if (K == 0) return;
  dim3 grid(8, K);
  k_pack_fp32<<<grid, 256, 0, st>>>(m, pk, K, w, static_cast<float*>(out));
}

}  // namespace mlps
