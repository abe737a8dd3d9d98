// mlps_kernels.h -- host-side launchers of the MLP-Splatting kernels (one per translation unit).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mlps_common.cuh"

namespace mlps {

// Packed weight blob description (per primitive, bytes from the primitive's base).
struct Packed {
  int precision;       // mlps_precision
  long long stride;    // bytes per primitive (multiple of 256)
  // FP32: per layer W^T [din][dout] then b [dout], each block starting on 16 bytes
  int woff[kMaxLayers], boff[kMaxLayers];  // float offsets (FP32 layout)
  int tc_scale;              // FP8: float scales [2 * nl] (forward tile, transposed tile)
  int din_pad[kMaxLayers], dout_pad[kMaxLayers];
  long long slot_byte;       // the four FP32 slot embeddings [4][C] (16-byte aligned), if C > 0
};

struct MlpArgs {
  Model m;
  Packed pk;
  const unsigned char* weights;  // packed blob [K, stride]
  float* d_weights;              // backward: canonical FP32 gradient [K, Prow]
  int resident;                  // FP32: all layers in shared memory at once
  int rows;                      // sample rows per chunk
  int groups;                    // forward tensor-core MLP: chunks in flight per CTA (0 = default)
};

// Input column of the canonical weights that column k of layer l's tensor-core tile holds. The
// tiles keep the canonical order except for the first layer of the contact-point model, whose
// encoded input [gamma(d); gamma(delta)] (Eq. 4) is stored as [gamma(delta); gamma(d)]: the
// backward pass then finds every input the pose gradient needs (gamma(delta)) in the first
// 64-column slab.
MLPS_HD int tc_in_col(const Model& m, int l, int k) {
  if (l != 0 || !m.contact) return k;
  const int nd = m.dirL > 0 ? 6 * m.dirL : 0, nx = m.xyzL > 0 ? 6 * m.xyzL : 3;
  return k < nx ? nd + k : k - nx;
}

// Tensor-core plan: per-layer padded shapes and where the operand tiles live.
struct TcPlan {
  int nl;
  int kpad[kMaxLayers], npad[kMaxLayers];  // K (inputs) and N (outputs) padded per layer
  int sw_off[kMaxLayers];                  // shared-memory byte offset of layer l's W tile
  int gw_row[kMaxLayers];                  // first 128-byte row of layer l's tile in a blob
  int w_bytes;                             // all forward W tiles
  // bias folding of the BF16 forward (0 = none): the biases of layers 0 .. fold-1 are a K-major
  // B tile of 64 rows and 64-column slabs (layer l's bias in slab l / 4, column 16 (l % 4)),
  // multiplied by a constant "ones" A tile in one extra K step per layer, so the epilogue adds
  // no bias
  int fold;
  int gbt_row;                             // first 128-byte row of the bias tile in a blob
  int sbt_off;                             // its shared-memory byte offset (after the W tiles)
  int bt_bytes;                            // 8192 per slab when fold > 0
  // E4M3 copy (FP8 precision only; w8_bytes = 0 otherwise): layer l's tile W [npad][kpad] / c_l
  // as one 128-byte row per output (kpad <= 128); then a bias tile for the hidden layers (rows =
  // hidden width, 64-column slabs: layer l's bias b / s_{l+1} as two E4M3 bytes hi + lo in
  // columns 32 (l % 4) and 32 (l % 4) + 1 of slab l / 4), added by one more K step against a
  // constant-1 operand; then FP32 mul_n / add_n of the last layer's epilogue (z = acc * mul + add,
  // bias_off indexing) and the input multiplier 1 / s_0. k_pack_e4m3 chooses the scales.
  int g8_row[kMaxLayers];                  // first 128-byte row of layer l's E4M3 tile in a blob
  int s8_off[kMaxLayers];                  // shared-memory byte offset of layer l's E4M3 tile
  int g8b_row;                             // first 128-byte row of the E4M3 bias tile
  int s8b_off;                             // its shared-memory byte offset
  int w8_bytes;                            // all E4M3 tiles, the bias tile included
  int gmul_byte;                           // byte offset of the FP32 multipliers (bias_off indexing)
  int gadd_byte;                           // byte offset of the FP32 offsets (bias_off indexing)
  int gin_byte;                            // byte offset of the FP32 input multiplier 1 / s_0
  int bias_off[kMaxLayers];                // float offset of layer l's bias
  int bias_floats;
  int gbias_byte;                          // byte offset of the FP32 biases in a blob
  int slot_byte;                           // byte offset of the FP32 slot embeddings (C > 0)
  int rows_per_prim;                       // blob stride / 128
  int kmax;                                // widest A tile (elements)
  int a_bytes;                             // one A tile: 128 rows x kmax BF16
};

// k_geometry.cu
void launch_store_views(const Work& w, const ViewArray& va, cudaStream_t st);
// View records from a device item table (checked against the caps; bases as running sums).
void launch_views_from_items(const Work& w, const mlps_batch_item* items, int max_w, int max_h, int max_p,
                             cudaStream_t st);
// returns the number of kernels launched
int launch_prim_setup(const Work& w, const float* c, const float* s, const float* q,
                      cudaStream_t st);
void launch_tile_lists(const Work& w, cudaStream_t st);
bool launch_intersect(const Work& w, cudaStream_t st);
void launch_prim_scan(const Work& w, cudaStream_t st);
void launch_scatter(const Work& w, int n_sm, cudaStream_t st);
void launch_export_hits(const Work& w, int max_out, int* count, int* prim, float* t0, float* t1,
                        float* tmid, cudaStream_t st);
void launch_export_tiles(const Work& w, int* count, int* list, cudaStream_t st);

// k_slots.cu (feature slots, Sec. 3.4)
void launch_slots_fwd(const Work& w, const Model& m, const Packed& pk, const unsigned char* weights,
                      float* feat, int row_stride, cudaStream_t st);
void launch_slots_bwd_ray(const Work& w, const Model& m, const Packed& pk, const unsigned char* weights,
                          const float* d_feat, int row_stride, cudaStream_t st);
void launch_slots_bwd_prim(const Work& w, const Model& m, const Packed& pk, const unsigned char* weights,
                           const float* d_feat, int row_stride, float* d_weights, int n_sm, cudaStream_t st);

// k_train.cu (training objective and optimizer, Sec. 3.5)
constexpr int kMaxAdamGroups = 8;
struct AdamGroupDev {
  float* param;
  const float* grad;
  float* m;
  float* v;
  float* aux;      // kind 1: x = exp(param), read for the chain rule and rewritten
  long long n;
  float lr;
  int kind;        // 0: plain, 1: log-parameter
};
// abc: 9 floats per pixel workspace; sums: 4 doubles
void launch_loss(int V, int H, int W, const float* rgb, const float* rgb_t, const uint8_t* tile_mask,
                 int tile, float lam, int C, const float* feat, const float* feat_t, float* d_rgb,
                 float* d_feat, float* abc, double* sums, float* loss_out, cudaStream_t st);
void launch_adam(const AdamGroupDev* groups, int n, float beta1, float beta2, float eps, int step,
                 int n_sm, cudaStream_t st);

// k_mlp_simt.cu (FP32 path)
size_t mlp_simt_smem(const MlpArgs& a, bool backward);
cudaError_t launch_mlp_fwd_simt(const Work& w, const MlpArgs& a, int n_sm, cudaStream_t st);
bool simt_bwd_supported(const MlpArgs& a);
cudaError_t launch_mlp_bwd_simt(const Work& w, const MlpArgs& a, int n_sm, cudaStream_t st);
// hidden width 128 (weights streamed, weight gradients in per-block global copies w.dwb);
// tp = the tensor-core plan when the blob holds BF16 tiles, else nullptr (FP32 blob)
bool simt_bwd_wide_supported(const MlpArgs& a);
cudaError_t launch_mlp_bwd_simt_wide(const Work& w, const MlpArgs& a, const TcPlan* tp, int n_sm, cudaStream_t st);

// k_mlp_tc.cu (BF16 tensor-core path)
bool tc_plan(const Model& m, TcPlan* P, long long* stride, bool e4m3 = false);
size_t tc_smem_bytes(const TcPlan& P, int F, int groups, int S);
// forward tensor-core MLP: the groups a configuration runs with (0 if `groups` is not allowed)
int tc_fwd_groups(int width, int F, int groups, bool e4m3);
void launch_pack_bf16(const Model& m, const TcPlan& P, long long stride, int K, const float* w,
                      void* out, cudaStream_t st);
cudaError_t launch_mlp_fwd_tc(const Work& w, const MlpArgs& a, const TcPlan& P, int n_sm,
                              cudaStream_t st);
// k_mlp_tc_bwd.cu (BF16 tensor-core backward)
bool tc_bwd_supported(const Model& m, const TcPlan& P);
// The model as the tensor-core kernels see it: 32-wide hidden layers padded to 64.
Model tc_model(const Model& m);
// BF16 tensor-core backward at hidden width 128 (weight gradients flushed per chunk into w.dwb,
// activations recomputed on demand).
bool tc_bwd_wide_supported(const Model& m, const TcPlan& P);
cudaError_t launch_mlp_bwd_tc_wide(const Work& w, const MlpArgs& a, const TcPlan& P, int n_sm,
                                   cudaStream_t st);
cudaError_t launch_mlp_bwd_tc(const Work& w, const MlpArgs& a, const TcPlan& P, int n_sm,
                              cudaStream_t st);

// k_composite.cu
// F MLP feature channels in rows of FT floats (FT = F + slot channels)
void launch_composite_fwd(const Work& w, int F, int FT, float* rgb, float* trans, float* feat,
                          cudaStream_t st);
// Interval lists (a selection of the primitive-major order, kept in that order) into w.live_*;
// chunk total in scratch header word 1, interval total in word 2 (4 launches). mode 0: the
// intervals with a nonzero gradient (the backward); 1: each ray's first k1 hits; 2: the later
// hits of the rays w.ray_alive marks (the forward's depth waves, whose intervals are also added
// up in word 3).
void launch_live_lists(const Work& w, int F, int mode, int k1, cudaStream_t st);
// After the first depth wave: w.ray_alive[r] = ray r has hits past its first k1 and its
// composite does not stop within them.
void launch_wave_alive(const Work& w, int k1, cudaStream_t st);
void launch_composite_bwd(const Work& w, int F, int FT, const float* d_rgb, const float* d_trans,
                          const float* d_feat, const float* slot_ga, cudaStream_t st);
void launch_pose_bwd(const Work& w, float* d_centers, float* d_scales, float* d_quats,
                     cudaStream_t st);

// k_pack.cu
void launch_pack_fp32(const Model& m, const Packed& pk, int K, const float* w_fp32, void* out,
                      cudaStream_t st);

}  // namespace mlps
