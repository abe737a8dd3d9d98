// k_mlp_tc_bwd_wide.cu -- BF16 tensor-core (tcgen05) backward of the grouped per-primitive MLP
// at hidden width 128 (the stress configuration: 60 -> 128 x 4 -> 4 + 16).
//
// What does not fit on chip at this width, and how the kernel gets around it:
//  * Weight gradients: four 128 x 128 layers and the head need 544 TMEM columns, more than the
//    512 of an SM. Each layer's gradient is accumulated in one TMEM region for one chunk only
//    and then added into the block's FP32 copy in global memory (L2-resident, laid out as
//    [out / 4][in][4] per layer, so that one vector reduction instruction of a warp covers four
//    outputs of 32 consecutive inputs, 512 contiguous bytes); the copy goes into d_weights when
//    the block's primitive changes.
//  * Activations: the resident weights take 120 KB of shared memory, so only one H tile, one
//    delta tile and the encoded input fit next to them. The last hidden activation H_L stays
//    in the H tile (it is also the head's A operand); H_{L-1} and H_{L-2} stay in TMEM (BF16
//    pairs, 64 columns each) and are copied into the H tile when their wgrad comes; an earlier
//    one (H_1 of a four-hidden-layer network) is recomputed from the input at that point. Each
//    delta takes the TMEM slot its phase has freed.
//  * Bias gradients: every input row of the wgrad accumulator is a feature, so the sum of
//    delta_l over the rows is one more MMA: A = delta_l read as an MN-major operand (M = the
//    outputs), B = a constant K-major operand whose first row is all ones (N = 16).
// Sixteen warps per SM: thread (row, part) owns TMEM lane `row` (the chunk's sample row) and
// the columns [32 part, 32 part + 32) of every 128-wide activation, gradient and weight-gradient
// row; the per-sample scalar work (the encoding, the pose chain) runs in part 0, the reverse
// scan of the composite is shared out over the parts, and part 1 copies the next chunk's
// interval tables with cp.async meanwhile. Per chunk: encode X; forward to the head; reverse of
// the interval composite (Eq. 6) into delta of the head; then for l = L .. 1:
// delta_{l-1} = G_l * [H_l > 0], dgrad_{l-1}, H_{l-1} into the H tile, wgrad_{l-1} and its bias
// sum, with dW_l read out of TMEM before that batch is issued and added into the copy after
// it; finally the encoding derivative and the pose chain (as in k_mlp_tc_bwd.cu). Every wait
// is bounded by wall time;
// after a timeout the kernel runs out its chunks without issuing MMAs, frees TMEM and reports
// MLPS_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "mlps_common.cuh"
#include "mlps_kernels.h"
#include "simt_common.cuh"
#include "tc_bwd_common.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace mlps {
namespace tc {

namespace {

constexpr int kParts = 4;                      // threads per TMEM lane (column quarters)
constexpr int kWThreads = kParts * kEGThreads;
constexpr int kPartCols = 128 / kParts;        // FP32 columns of a 128-wide row per thread
constexpr int kScanPart = 4 * 8;               // scan scratch floats per part (4 warps x 8 values)
constexpr uint32_t kSlab = kM * 128;           // one 64-column slab of 128 rows (16 KB)
constexpr uint32_t kOnesMN = 2048;             // 16 rows of the MN-major ones atom (one K step)
constexpr uint32_t kOnesK = 2048;              // K-major ones operand: 16 rows, the first all ones
constexpr uint64_t kWaitNsW = 2000000000ull;
// TMEM columns: accumulator (forward / dgrad), three 64-column slots of BF16 pairs (activations
// H_{L-2} in Sa and H_{L-1} in Sb, deltas as dgrad A operands), weight gradient, bias sums
constexpr uint32_t kColD = 0, kColSa = 128, kColSb = 192, kColSc = 256, kColR = 320, kColRb = 448;
constexpr uint32_t kTmemColsW = 512;

struct WideSmem {
  // tab: two buffers (tab_stride apart) of the chunk tables, each holding the interval records
  // (itab), their gradients (giv) and feature gradients (gf) at these offsets
  uint32_t w, xt, ht, dt, ones_mn, ones_k, bias, tab, tab_stride, itab, giv, gf, ddel, pose, scan, share, geo, pgeo,
      bars, misc, total;
};

MLPS_HD uint32_t alw(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

MLPS_HD WideSmem wide_layout(const TcPlan& P, int F, int ipc) {
  WideSmem L;
  uint32_t o = 0;
  L.w = o;
  o = alw(o + P.w_bytes, 1024);
  L.xt = o;  // encoded input X: one slab (kpad0 = 64)
  o += kSlab;
  L.ht = o;  // H_l: two slabs
  o += 2 * kSlab;
  L.dt = o;  // delta_l: two slabs
  o += 2 * kSlab;
  L.ones_mn = o;  // after the X tile's reach: wgrad_0 finds it at a positive offset
  o = alw(o + kOnesMN, 1024);
  L.ones_k = o;
  o = alw(o + kOnesK, 1024);
  L.bias = o;
  o = alw(o + 4 * P.bias_floats, 16);
  L.tab = o;
  uint32_t q = 0;
  L.itab = q;
  q = alw(q + (uint32_t)sizeof(IntervalRec) * ipc, 16);
  L.giv = q;
  q = alw(q + 16 * ipc, 16);
  L.gf = q;
  q = alw(q + 4 * ipc * (F > 0 ? F : 1), 16);
  L.tab_stride = q;
  o += 2 * q;
  L.ddel = o;
  o = alw(o + 4 * ipc, 16);
  L.pose = o;  // per interval: the six sums of the pose chain
  o = alw(o + 4 * 6 * ipc, 16);
  L.scan = o;  // per part: 4 warps x the widest segmented scan of that part (at most 8 values)
  o = alw(o + 4 * kParts * kScanPart, 16);
  L.share = o;  // parts 1-3: their shares of dL/d alpha per row
  o = alw(o + 4 * (kParts - 1) * kM, 16);
  L.geo = o;
  o = alw(o + 4 * 16, 16);
  L.pgeo = o;
  o = alw(o + (uint32_t)sizeof(PrimGeo), 16);
  L.bars = o;
  o = alw(o + 8 * 4, 16);
  L.misc = o;
  o = alw(o + 16, 16);
  L.total = o;
  return L;
}

// dgrad G = delta W_l (M = rows, N = nin inputs, K = nout outputs): A = delta in TMEM (8 columns
// per K = 16 step), B = the forward W_l tile read MN-major, its 64-input slabs `slab` bytes apart.
MLPS_DEV void issue_dgrad_w(uint32_t At, uint32_t wtile, uint32_t d, int nin, int nout, uint32_t slab) {
  const uint32_t id = idesc_bf16(kM, nin) | (1u << 16);
  const uint64_t db = sw128_desc_mn(wtile, slab);
  const int nk = nout / 16;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    if (kk >= nk) break;
    mma_bf16_ta(d, At + 8u * (uint32_t)kk, db + (uint64_t)(kk * 128), id, kk > 0 ? 1u : 0u);
  }
}

// wgrad dW_l^T [inputs][outputs] = H_l^T delta_l over the chunk's 128 rows (K), overwriting the
// region: A = H_l (M = 128 inputs, two slabs), B = delta_l (N = nout, slabs 16 KB apart), both
// MN-major views of the row-major tiles.
MLPS_DEV void issue_wgrad_w(uint32_t H, uint32_t Dt, uint32_t R, int nout) {
  const uint32_t id = idesc_bf16(kM, nout) | (1u << 15) | (1u << 16);
  const uint64_t da = sw128_desc_mn(H, kSlab), db = sw128_desc_mn(Dt, kSlab);
#pragma unroll
  for (int kk = 0; kk < kM / 16; ++kk) mma_bf16(R, da + (uint64_t)(kk * 128), db + (uint64_t)(kk * 128), id, kk > 0);
}

// wgrad of the first layer (64 inputs): A = [X | ones atom] (row 64 of the accumulator is the
// bias gradient; the ones atom's offset shrinks by one K step per step, so one 16-row block
// serves them all), B = delta_0 as above.
MLPS_DEV void issue_wgrad_w0(uint32_t X, uint32_t Dt, uint32_t R, uint32_t ones, int nout) {
  const uint32_t id = idesc_bf16(kM, nout) | (1u << 15) | (1u << 16);
  const uint64_t da = sw128_desc_mn(X, ones - X), db = sw128_desc_mn(Dt, kSlab);
#pragma unroll
  for (int kk = 0; kk < kM / 16; ++kk) {
    const uint64_t step = (uint64_t)(kk * 128);
    mma_bf16(R, da + step - (step << 16), db + step, id, kk > 0);
  }
}

// Bias sums: Rb[out][0] = sum over the rows of delta[row][out]: A = delta (M = 128 outputs,
// MN-major, two slabs), B = the K-major ones operand (N = 16, its first row all ones; the same
// 16 K values serve every step, so its descriptor does not move).
MLPS_DEV void issue_bias_w(uint32_t Dt, uint32_t onesK, uint32_t Rb) {
  const uint32_t id = idesc_bf16(kM, 16) | (1u << 15);
  const uint64_t da = sw128_desc_mn(Dt, kSlab), db = sw128_desc(onesK);
#pragma unroll
  for (int kk = 0; kk < kM / 16; ++kk) mma_bf16(Rb, da + (uint64_t)(kk * 128), db, id, kk > 0);
}

// Part P's share of the reverse of the interval composite (Eq. 6) for one sample row: of the
// 3 + NF weighted head outputs w_k c_k (colours) and w_k f_k (features), the values
// [P kHeadPer, (P + 1) kHeadPer), reverse-scanned over the interval with the part's scratch and
// named barrier, and their terms of dL/d alpha_k: g (tau_k e^{-alpha_k} c_k - (suffix - w_k c_k)).
// `gf` is the row's feature gradient (nullptr: zero); outputs past 3 + F are zero.
template <int NF>
constexpr int head_per() { return (3 + NF + kParts - 1) / kParts; }

template <int NF, int P>
MLPS_DEV float head_share(const float (&z)[4 + NF], const float (&cq)[3], const float (&gcs)[3], const float* gf, int F,
                          float wk, float te, int row, int S, float* scratch, int bar_id) {
  constexpr int kPer = head_per<NF>(), v0 = P * kPer;
  float sv[kPer], val[kPer], g[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int v = v0 + j;
    if (v < 3) {
      val[j] = cq[v < 3 ? v : 0];
      g[j] = gcs[v < 3 ? v : 0];
    } else if (v < 3 + NF && v - 3 < F) {
      val[j] = z[v < 3 + NF ? v + 1 : 0];
      g[j] = gf ? gf[v - 3] : 0.f;
    } else {
      val[j] = 0.f;
      g[j] = 0.f;
    }
    sv[j] = wk * val[j];
  }
  const int nv = min(kPer, 3 + F - v0);  // the same for the whole part
  if (nv > 0) seg_scan_rev<kPer>(sv, nv, row, S, scratch, bar_id);
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kPer; ++j) acc += g[j] * (te * val[j] - (sv[j] - wk * val[j]));
  return acc;
}

// Four floats added to global memory without return (16-byte aligned address).
MLPS_DEV void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

}  // namespace

template <int NF, int XL, int DL>
__global__ void __launch_bounds__(kWThreads, 1)
    k_mlp_bwd_tc_wide(Work w, MlpArgs a, TcPlan P, const __grid_constant__ CUtensorMap tmap) {
  static_assert(4 + NF <= 32 && NF % 2 == 0, "the head's outputs lie in the first 32 columns");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* gb = smem_raw + (sbase - raw);
  const Model& m = a.m;
  const int F = m.F, nl = m.nl, S = m.S, L = m.nl - 1;  // L: the head layer
  const WideSmem Lw = wide_layout(P, 32, w.ipc);  // the host sizes the same layout
  float* sBias = reinterpret_cast<float*>(gb + Lw.bias);
  float* sScan = reinterpret_cast<float*>(gb + Lw.scan);
  float* sShare = reinterpret_cast<float*>(gb + Lw.share);
  float* sGeo = reinterpret_cast<float*>(gb + Lw.geo);
  // barriers: weights (TMA), MMA chain (forward layers, dgrads), weight gradients (wgrad and
  // bias sums), teardown
  const uint32_t bar_w = sbase + Lw.bars, bar_m = bar_w + 8u, bar_e = bar_w + 16u, bar_g = bar_w + 24u;
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(gb + Lw.misc);
  volatile int* sAbort = reinterpret_cast<volatile int*>(gb + Lw.misc + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = threadIdx.x & (kM - 1);  // sample row of the chunk, TMEM lane
  const int part = threadIdx.x >> 7;       // column quarter (warp-uniform)
  const bool lead = part == 0;             // the per-sample scalar work
  const bool issuer = threadIdx.x == 0;
  const uint32_t xt = sbase + Lw.xt, ht = sbase + Lw.ht, dt = sbase + Lw.dt;
  // this thread's columns in a two-slab row-major tile: slab, first 16-byte chunk of the row
  const uint32_t hs = (uint32_t)(part * kPartCols / 64) * kSlab;
  const int hch = (part * kPartCols % 64) / 8;
  const uint32_t ones_mn = sbase + Lw.ones_mn, ones_k = sbase + Lw.ones_k;
  auto wt = [&](int l) { return sbase + Lw.w + (uint32_t)P.sw_off[l]; };

  if (threadIdx.x == 0) {
    mbar_init(bar_w, 1);
    mbar_init(bar_m, 1);
    mbar_init(bar_e, 1);
    mbar_init(bar_g, 1);
    *sAbort = 0;
    fence_mbar_init();
  }
  // MN-major ones atom: element 0 of every row is 1.0 (BF16 0x3F80); K-major ones operand: the
  // first of its 16 rows is all ones (the swizzle leaves row 0 in place)
  for (int i = threadIdx.x; i < (int)(kOnesMN / 16); i += kWThreads) {
    const int r = i >> 3, ch = i & 7;
    st_shared_v4(ones_mn + (uint32_t)i * 16, ((ch ^ (r & 7)) == 0) ? 0x3F80u : 0u, 0u, 0u, 0u);
    const uint32_t o = r == 0 ? 0x3F803F80u : 0u;
    st_shared_v4(ones_k + (uint32_t)i * 16, o, o, o, o);
  }
  if (threadIdx.x < 16) sGeo[threadIdx.x] = 0.f;
  fence_proxy_async_smem();
  if (warp == 0) {
    tmem_alloc(sbase + Lw.misc, kTmemColsW);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
  // MMA operand / accumulator addresses (lane 0) and this thread's row of them
  const uint32_t mD = tmem + kColD, mR = tmem + kColR, mRb = tmem + kColRb;
  const uint32_t mSa = tmem + kColSa, mSb = tmem + kColSb, mSc = tmem + kColSc;
  const uint32_t rD = mD + lanes, rR = mR + lanes, rRb = mRb + lanes;
  const uint32_t hc = (uint32_t)(kPartCols * part);  // first FP32 column of this thread's part
  const uint32_t hp = hc / 2;                        // first BF16-pair column of this thread's part
  // this thread's 32 columns (16 BF16 pairs) of row `row` of a two-slab tile
  auto store_part = [&](uint32_t tile, const uint32_t(&pk)[16]) {
    const RowSw sw(row);
#pragma unroll
    for (int ch = 0; ch < 4; ++ch)
      st_shared_v4(tile + hs + sw.off(hch + ch), pk[4 * ch], pk[4 * ch + 1], pk[4 * ch + 2], pk[4 * ch + 3]);
  };

  const int total = walk_chunk_count(w);
  const int* const bmap = walk_map(w);  // list position -> forward position
  const int cb = (int)((long long)total * blockIdx.x / gridDim.x);
  const int ce = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  float* dwb = w.dwb + (size_t)blockIdx.x * m.P;  // this block's dW copy, per layer [out / 4][in][4]
  uint32_t ph_w = 0, ph_m = 0, ph_g = 0;
  float geo_acc = 0.f;  // pose output `lane` (< 12) of the current primitive, this warp's share
  const float invS = 1.f / (float)S;
  int loaded = -1;

  // the next completion of the issuer's MMAs (every thread waits: tcgen05.ld is warp-wide)
  auto wait_m = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_m, ph_m, sAbort, kWaitNsW));
    ph_m ^= 1u;
    tc_fence_after();
    return ok;
  };
  auto commit_m = [&]() {
    if (issuer) mma_commit(bar_m);
  };
  // the next completion of the weight-gradient MMAs (wgrad and bias sum of a layer)
  auto wait_g = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_g, ph_g, sAbort, kWaitNsW));
    ph_g ^= 1u;
    tc_fence_after();
    return ok;
  };
  // the block's copy of primitive p's gradients into d_weights (canonical layout), then zeroed
  auto flush_prim = [&](int p) {
    __threadfence_block();  // the block's reductions into its copy before the reads below
    __syncthreads();
    float* dW = a.d_weights + (size_t)p * m.Prow;
    for (int l = 0; l < nl; ++l) {
      const int din = m.din[l], dout = m.dout[l];
      // (the copy is updated by reductions at L2: read and clear it there, past the L1; its
      // layout is [out / 4][in][4], d_weights' is [out][in])
      for (int i = threadIdx.x; i < din * dout; i += kWThreads) {
        const float v = __ldcg(dwb + m.woff[l] + i);
        if (v != 0.f) {
          const int g4 = i / (4 * din), r = i - g4 * 4 * din, k = r >> 2, n = 4 * g4 + (r & 3);
          atomicAdd(&dW[m.woff[l] + n * din + k], v);
          __stcg(dwb + m.woff[l] + i, 0.f);
        }
      }
      for (int n = threadIdx.x; n < dout; n += kWThreads) {
        const float v = __ldcg(dwb + m.boff[l] + n);
        if (v != 0.f) {
          atomicAdd(&dW[m.boff[l] + n], v);
          __stcg(dwb + m.boff[l] + n, 0.f);
        }
      }
    }
    if (geo_acc != 0.f) atomicAdd(&sGeo[lane], geo_acc);
    geo_acc = 0.f;
    __syncthreads();
    if (threadIdx.x < 12) {
      const float v = sGeo[threadIdx.x];
      if (v != 0.f) atomicAdd(&w.dgeo[12 * (size_t)p + threadIdx.x], v);
      sGeo[threadIdx.x] = 0.f;
    }
    __syncthreads();
  };
  // chunk gradient of layer l (region R: input row = lane, outputs along the columns, this
  // thread's part of them; layer 0's bias gradient in row 64, other layers' in Rb) into the
  // block's copy, in two steps: flush_take reads R and Rb into registers (before the barrier
  // after which the next wgrad overwrites them), flush_put adds them to the copy. The
  // reductions go out after that barrier: a barrier waits until the earlier global memory
  // operations of its threads are performed, so reductions issued before it would put their
  // whole round trip to the L2 on the chunk's serial chain.
  auto flush_take = [&](int l, uint32_t(&v)[32], float& b) {
    uint32_t bb = 0u;
    tmem_ld32(rR + hc, v);  // (R has 128 columns; only the head's first 32 are used below)
    if (l > 0 && lead) bb = tmem_ld1(rRb);
    tmem_wait_ld();
    b = __uint_as_float(bb);
  };
  auto flush_put = [&](int l, const uint32_t(&v)[32], float b) {
    if (*sAbort) return;
    const int din = m.din[l], dout = m.dout[l];
    const int c0 = (int)hc;
    if (c0 < P.npad[l]) {
      if (row < din) {
        // copy layout [out / 4][in][4]: the four outputs 4g .. 4g + 3 of input `row` are one
        // 16-byte vector, and the warp's 32 consecutive inputs make one 512-byte run
        float* cp = dwb + m.woff[l] + ((size_t)(c0 / 4) * din + row) * 4;
        const int nj = min(32, dout - c0);
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          if (j < nj)
            red_add_v4(cp, __uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                       __uint_as_float(v[j + 3]));
          cp += 4 * din;
        }
      } else if (l == 0 && row == 64) {
        for (int j = 0; j < 32; ++j)
          if (c0 + j < dout) atomicAdd(&dwb[m.boff[0] + c0 + j], __uint_as_float(v[j]));
      }
    }
    if (l > 0 && lead && row < dout) atomicAdd(&dwb[m.boff[l] + row], b);
  };
  // epilogue of hidden layer l, this thread's part: H_{l+1} = ReLU(Z_l + b_l) from the
  // accumulator row `src` as BF16 pairs, into the TMEM slot row `dst` or the H tile
  auto hidden_epilogue = [&](int l, uint32_t src, bool to_tile, uint32_t dst) {
    const float4* b4 = reinterpret_cast<const float4*>(sBias + P.bias_off[l] + hc);
    uint32_t pk[16];
    {
      uint32_t v[32];
      tmem_ld32(src + hc, v);
      tmem_wait_ld();
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float4 bq = b4[e];
        float x0 = __uint_as_float(v[4 * e]), x1 = __uint_as_float(v[4 * e + 1]);
        float x2 = __uint_as_float(v[4 * e + 2]), x3 = __uint_as_float(v[4 * e + 3]);
        add2_f32(x0, x1, bq.x, bq.y);
        add2_f32(x2, x3, bq.z, bq.w);
        pk[2 * e] = pack_bf16_relu(x0, x1);
        pk[2 * e + 1] = pack_bf16_relu(x2, x3);
      }
    }
    tc_fence_before();
    if (to_tile) {
      store_part(ht, pk);
      fence_proxy_async_smem();
    } else {
      tmem_st16(dst + hp, pk);
      tmem_wait_st();
    }
  };
  // TMEM slot of H_j (1 <= j < L) during the forward: H_{L-1} in Sb, H_{L-2} in Sa, an earlier
  // one in Sa until the next overwrites it
  auto fwd_slot = [&](int j) { return j == L - 1 ? mSb : mSa; };
  // TMEM slot that receives delta_{l-1} in phase l (free by then: its activation has been
  // copied to the H tile, or its delta consumed by an earlier dgrad)
  auto delta_slot = [&](int l) { return (l == L || l == L - 3) ? mSc : (l == L - 1 ? mSb : mSa); };

  float* DD = reinterpret_cast<float*>(gb + Lw.ddel);
  float* sPose = reinterpret_cast<float*>(gb + Lw.pose);
  // Chunk c's tables are in buffer (c - cb) & 1. From the block's second chunk on, part 1 copies
  // them with cp.async while part 0 reverses the previous chunk's composite.
  auto tab = [&](int cc) { return gb + Lw.tab + (uint32_t)((cc - cb) & 1) * Lw.tab_stride; };
  auto prefetch_tab = [&](int cn, int pc) {
    int pn = pc;
    while (cn >= w.chunk_start[pn + 1]) ++pn;
    const int fst = (cn - w.chunk_start[pn]) * w.ipc;
    const int i = threadIdx.x - kEGThreads;  // part 1's thread i copies interval i
    if (i < 0 || i >= min(w.ipc, w.prim_count[pn] - fst)) return;
    const int slot = walk_slot(bmap, w.prim_start[pn] + fst + i);
    const uint32_t t = smem_u32(tab(cn));
    // (F is a multiple of 4 on this path: the head's output count is)
    for (int f = 0; f < F; f += 4) cp_async16(t + Lw.gf + 4u * (uint32_t)(i * F + f), w.hit_gfeat + (size_t)slot * F + f);
    rec_copy_async(w, slot, t + Lw.itab + 64u * (uint32_t)i, t + Lw.giv + 16u * (uint32_t)i);
  };
  const PrimGeo& Gp = *reinterpret_cast<const PrimGeo*>(gb + Lw.pgeo);
  int prim = cb < ce ? simt::find_prim(w, cb) : 0;

  // Layer 0's gradient of the previous chunk stays in R until the next chunk has issued its
  // first layer (R is next written by that chunk's wgrad of the head), so that its reductions
  // overlap the first forward layer instead of the next barrier; earlier on a primitive change
  bool pend0 = false;
  auto flush0 = [&]() {
    uint32_t rv[32];
    float rb;
    flush_take(0, rv, rb);
    tc_fence_before();
    flush_put(0, rv, rb);
    pend0 = false;
  };
  for (int c = cb; c < ce; ++c) {
    while (c >= w.chunk_start[prim + 1]) ++prim;
    if (prim != loaded) {
      if (pend0) flush0();
      if (loaded >= 0) flush_prim(loaded);
      if (threadIdx.x == 0 && !*sAbort) {
        mbar_arrive_expect_tx(bar_w, (uint32_t)P.w_bytes);
        const int row0 = prim * P.rows_per_prim;
        for (int l = 0; l < nl; ++l)
          for (int sl = 0; sl < P.kpad[l] / 64; ++sl)
            for (int j = 0; j < P.npad[l] / 16; ++j)
              tma_load_2d(wt(l) + sl * P.npad[l] * 128 + j * 2048, &tmap, 0,
                          row0 + P.gw_row[l] + sl * P.npad[l] + j * 16, bar_w);
      }
      const float* gbias = reinterpret_cast<const float*>(a.weights + (size_t)prim * a.pk.stride + P.gbias_byte);
      for (int i = threadIdx.x; i < P.bias_floats; i += kWThreads) sBias[i] = gbias[i];
      {
        const int* src = reinterpret_cast<const int*>(w.geo + prim);
        int* dst = reinterpret_cast<int*>(gb + Lw.pgeo);
        for (int i = threadIdx.x; i < (int)(sizeof(PrimGeo) / 4); i += kWThreads) dst[i] = src[i];
      }
      mbar_wait(bar_w, ph_w, sAbort, kWaitNsW);
      ph_w ^= 1;
      __syncthreads();
      loaded = prim;
    }
    // ---------------- the chunk's interval records and their gradients
    const int first = (c - w.chunk_start[prim]) * w.ipc;
    const int nint = min(w.ipc, w.prim_count[prim] - first);
    IntervalRec* T = reinterpret_cast<IntervalRec*>(tab(c) + Lw.itab);
    float4* GI = reinterpret_cast<float4*>(tab(c) + Lw.giv);
    float* GF = reinterpret_cast<float*>(tab(c) + Lw.gf);
    if (c == cb) {
      for (int i = threadIdx.x; i < nint; i += kWThreads) {
        const size_t slot = walk_slot(bmap, w.prim_start[prim] + first + i);
        T[i] = w.rec[slot];
        GI[i] = w.hit_grad[slot];
        for (int f = 0; f < F; ++f) GF[i * F + f] = w.hit_gfeat[slot * F + f];
      }
    } else {
      cp_async_wait_all();  // this thread's copies of the chunk's tables (if any) have landed
    }
    __syncthreads();
    const int iv = row / S, k = row - iv * S;
    const bool valid = iv < nint;
    const uint32_t vmask = valid ? 0xFFFFFFFFu : 0u;

    // ---------------- X into its tile; forward to the head: H_1 .. H_{L-1} in TMEM slots, H_L
    // in the H tile (the head's A operand)
    if (lead) {
      uint32_t pk[32];
      encode_row64<XL, DL>(T, nint, S, row, pk);
      store_row64(xt, row, pk);
      fence_proxy_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    if (issuer) {
      tc_fence_after();
      if (!*sAbort) issue_fwd_layer(xt, wt(0), mD, P.kpad[0], P.npad[0]);
    }
    commit_m();
    if (pend0) flush0();
    for (int l = 0; l < L; ++l) {
      const int j = l + 1;  // H_j
      (void)wait_m();
      hidden_epilogue(l, rD, j == L, fwd_slot(j) + lanes);
      tc_fence_before();
      __syncthreads();
      if (issuer) {
        tc_fence_after();
        if (!*sAbort) {
          if (j == L) issue_fwd_layer(ht, wt(L), mD, P.kpad[L], P.npad[L]);
          else issue_fwd_layer_ta(fwd_slot(j), wt(j), mD, P.kpad[j], P.npad[j]);
        }
      }
      commit_m();
    }
    // ---------------- heads and reverse of the interval composite (Eq. 6) -> delta_L. Every part
    // evaluates the head of its row and the interval's transmittance; the reverse scan of the
    // 3 + F weighted outputs is shared out, kHeadPer values per part, and part 0 gathers the
    // parts' contributions to dL/d alpha and writes delta_L.
    (void)wait_m();
    {
      float z[4 + NF];
      {
        uint32_t r32[32];
        tmem_ld32(rD, r32);
        tmem_wait_ld();
        const float* bias = sBias + P.bias_off[L];
#pragma unroll
        for (int j = 0; j < 4 + NF; ++j) z[j] = j < m.nout ? __uint_as_float(r32[j]) + bias[j] : 0.f;
      }
      tc_fence_before();
      float* scr = sScan + part * kScanPart;  // this part's scan scratch and named barrier
      const int pbar = 1 + part;
      const IntervalRec& I = T[valid ? iv : 0];
      const float dtv = valid ? I.dt : 0.f;
      const float sig = softplus_fast(z[3]);
      const float ak = valid ? sig * dtv : 0.f;
      float sc1[1] = {ak};
      seg_scan<1>(sc1, 1, row, S, scr, pbar);
      const float Aex = sc1[0] - ak;
      const float tau = __expf(-Aex), ea = __expf(-ak);
      const float wk = valid ? tau * (1.f - ea) : 0.f;
      float cq[3];
      for (int u = 0; u < 3; ++u) cq[u] = sigmoid_fast(z[u]);
      const float4 gI = valid ? GI[iv] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float gcs[3] = {gI.x, gI.y, gI.z};
      const float* gfr = valid ? GF + iv * F : nullptr;
      float share = 0.f;
      switch (part) {
        case 0: share = head_share<NF, 0>(z, cq, gcs, gfr, F, wk, tau * ea, row, S, scr, pbar); break;
        case 1: share = head_share<NF, 1>(z, cq, gcs, gfr, F, wk, tau * ea, row, S, scr, pbar); break;
        case 2: share = head_share<NF, 2>(z, cq, gcs, gfr, F, wk, tau * ea, row, S, scr, pbar); break;
        default: share = head_share<NF, 3>(z, cq, gcs, gfr, F, wk, tau * ea, row, S, scr, pbar); break;
      }
      if (!lead) sShare[(part - 1) * kM + row] = share;
      __syncthreads();
      if (lead) {
        const float dLda = gI.w + share + sShare[row] + sShare[kM + row] + sShare[2 * kM + row];
        float dz[4 + NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) dz[4 + f] = (valid && f < F) ? wk * gfr[f] : 0.f;
#pragma unroll
        for (int u = 0; u < 3; ++u) dz[u] = wk * gcs[u] * cq[u] * (1.f - cq[u]);
        dz[3] = valid ? dLda * dtv * sigmoid_fast(z[3]) : 0.f;
        float dd[1] = {valid ? sig * dLda : 0.f};
        seg_scan<1>(dd, 1, row, S, scr, pbar);
        if (valid && k == S - 1) DD[iv] = dd[0];
        uint32_t pk[16];
#pragma unroll
        for (int e = 0; e < 16; ++e)
          pk[e] = (2 * e < 4 + NF) ? pack_bf16(2 * e < m.nout ? dz[2 * e] : 0.f, 2 * e + 1 < m.nout ? dz[2 * e + 1] : 0.f)
                                   : 0u;
        // delta_L (32 columns): A operand of dgrad_L in slot Sc; B of wgrad_L and A of its bias
        // sum in the delta tile (chunks 0-3 of slab 0; the rest is never flushed)
        tmem_st16(mSc + lanes, pk);
        const RowSw sw(row);
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) st_shared_v4(dt + sw.off(ch), pk[4 * ch], pk[4 * ch + 1], pk[4 * ch + 2], pk[4 * ch + 3]);
        tmem_wait_st();
        fence_proxy_async_smem();
      } else if (part == 1 && c + 1 < ce) {
        prefetch_tab(c + 1, prim);  // the next chunk's tables, into the other buffer
      }
    }
    tc_fence_before();
    __syncthreads();
    if (issuer) {
      tc_fence_after();
      if (!*sAbort) issue_dgrad_w(mSc, wt(L), mD, P.kpad[L], P.npad[L], (uint32_t)P.npad[L] * 128u);
      mma_commit(bar_m);
      if (!*sAbort) {
        issue_wgrad_w(ht, dt, mR, P.npad[L]);
        issue_bias_w(dt, ones_k, mRb);
      }
      mma_commit(bar_g);
    }
    // ---------------- backward phases l = L .. 1: each starts when dgrad_l is done (bar_m),
    // reads G_l and masks it while wgrad_l and its bias sum run, waits for them (bar_g), flushes
    // them, and issues dgrad_{l-1} (bar_m) and wgrad_{l-1} with its bias sum (bar_g)
    bool dgrad_waited = false;  // (the recompute step has already waited for dgrad_1)
    for (int l = L; l >= 1; --l) {
      if (!dgrad_waited) (void)wait_m();
      dgrad_waited = false;
      uint32_t G[16];  // this thread's part of G_l = dL/dH_l (unmasked) as BF16 pairs
      {
        uint32_t v[32];
        tmem_ld32(rD + hc, v);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) G[e] = pack_bf16(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]));
      }
      // delta_{l-1} = G_l * [H_l > 0] (H_l in the H tile, still read by wgrad_l), into its TMEM
      // slot now and into the delta tile once wgrad_l is done
      {
        const RowSw sw(row);
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          uint32_t hq[4];
          ld_shared_v4(ht + hs + sw.off(hch + ch), hq[0], hq[1], hq[2], hq[3]);
#pragma unroll
          for (int e = 0; e < 4; ++e) G[4 * ch + e] &= bf16x2_nonzero(hq[e]) & vmask;
        }
      }
      const uint32_t ds = delta_slot(l);
      tmem_st16(ds + lanes + hp, G);
      // H_{l-1} into the H tile from its TMEM slot (the mask above has read H_l: same thread,
      // same row), or recomputed from X below
      const bool from_slot = l - 1 >= 1 && l - 1 >= L - 2;
      const bool recompute = l - 1 >= 1 && !from_slot;
      uint32_t h[16];
      if (from_slot) {
        tmem_ld16(fwd_slot(l - 1) + lanes + hp, h);
        tmem_wait_ld();
      }
      (void)wait_g();  // wgrad_l and its bias sum: R, Rb final; the H and delta tiles free
      store_part(dt, G);
      if (from_slot) store_part(ht, h);
      uint32_t rv[32];
      float rb;
      flush_take(l, rv, rb);
      tmem_wait_st();
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      if (issuer) {
        tc_fence_after();
        if (!*sAbort)
          issue_dgrad_w(ds, wt(l - 1), mD, P.kpad[l - 1], P.npad[l - 1], (uint32_t)P.npad[l - 1] * 128u);
        if (recompute) {
          if (!*sAbort) issue_fwd_layer(xt, wt(0), mR, P.kpad[0], P.npad[0]);  // Z_0 into R
          mma_commit(bar_m);  // dgrad_{l-1} and Z_0
        } else {
          mma_commit(bar_m);
          if (!*sAbort) {
            if (l == 1) {
              issue_wgrad_w0(xt, dt, mR, ones_mn, P.npad[0]);  // bias gradient in row 64
            } else {
              issue_wgrad_w(ht, dt, mR, P.npad[l - 1]);
              issue_bias_w(dt, ones_k, mRb);
            }
          }
          mma_commit(bar_g);
        }
      }
      flush_put(l, rv, rb);
      if (recompute) {
        // H_1 = ReLU(Z_0 + b_0) into the H tile, then wgrad_1 and its bias sum
        (void)wait_m();
        dgrad_waited = true;
        hidden_epilogue(0, rR, true, 0u);
        tc_fence_before();
        __syncthreads();
        if (issuer) {
          tc_fence_after();
          if (!*sAbort) {
            issue_wgrad_w(ht, dt, mR, P.npad[1]);
            issue_bias_w(dt, ones_k, mRb);
          }
          mma_commit(bar_g);
        }
      }
    }
    // ---------------- encoding derivative and pose chain (midpoint samples), as in the 64-wide
    // kernel: the per-interval sums A = sum_k gx_k and B = sum_k c_k gx_k, coordinate u of
    // both in part u (u < 3); part 0 then runs the per-interval tail
    (void)wait_m();  // dgrad_0 (wgrad_0 may still run)
    if (part < 3) {
      uint32_t v0[32], v1[32];
      tmem_ld32(rD, v0);
      tmem_ld32(rD + 32, v1);
      tmem_wait_ld();
      const IntervalRec& I = T[valid ? iv : 0];
      const float ck = ((float)k + 0.5f) * invS - 0.5f;
      float gxu = 0.f;
      if (valid) {
        const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
        const float xu = fmaf(tr, I.dp[part], I.p[part]);
        gxu = part == 0 ? enc_grad_coord<XL, 0>(xu, v0, v1)
            : part == 1 ? enc_grad_coord<XL, 1>(xu, v0, v1)
                        : enc_grad_coord<XL, 2>(xu, v0, v1);
      }
      float red[2] = {gxu, ck * gxu};
      seg_scan<2>(red, 2, row, S, sScan + part * kScanPart, 1 + part);
      if (valid && k == S - 1) {  // the interval's totals
        sPose[6 * iv + part] = red[0];
        sPose[6 * iv + 3 + part] = red[1];
      }
    }
    __syncthreads();
    if (lead) {
      const int wrow0 = row - lane;
      for (int r_end = (wrow0 / S + 1) * S - 1; r_end < wrow0 + 32; r_end += S) {
        const int ive = r_end / S;
        if (ive >= nint) break;  // warp-uniform
        float rr[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) rr[j] = sPose[6 * ive + j];
        if (lane < 12) {
          const IntervalRec& Ie = T[ive];
          const float span = Ie.r1 - Ie.r0, tm = Ie.r0 + 0.5f * span;
          const float dA = rr[0] * Ie.dp[0] + rr[1] * Ie.dp[1] + rr[2] * Ie.dp[2];
          const float dB = rr[3] * Ie.dp[0] + rr[4] * Ie.dp[1] + rr[5] * Ie.dp[2];
          const float dDelta = DD[ive];
          const float gt0 = 0.5f * dA - dB - dDelta * invS, gt1 = 0.5f * dA + dB + dDelta * invS;
          const bool clamped = Ie.r0 != -Ie.r1;
          const float gtm = gt1 + (clamped ? 0.f : gt0);
          const float gh = gt1 - (clamped ? 0.f : gt0);
          const float aa = Ie.dp[0] * Ie.dp[0] + Ie.dp[1] * Ie.dp[1] + Ie.dp[2] * Ie.dp[2];
          const float inv_a = 1.f / aa;
          const float hh = Ie.r1;
          const float gh_ah = hh > 0.f ? gh * inv_a / hh : 0.f;
          if (lane < 9) {
            const int u = lane / 3, e = lane - 3 * u;
            const float ru = u == 0 ? rr[0] : (u == 1 ? rr[1] : rr[2]);
            const float rbu = u == 0 ? rr[3] : (u == 1 ? rr[4] : rr[5]);
            const float pu = Ie.p[u], dpu = Ie.dp[u];
            const float go_u = -gtm * dpu * inv_a - gh_ah * pu;
            const float cd_u = -(gtm * pu + gh * hh * dpu) * inv_a;
            const float ta = tm * ru + span * rbu;
            float gy = 0.f, ym = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const float rsj = Gp.R[e * 3 + j] * Gp.s[j];
              gy = fmaf(rsj, ru * Ie.p[j] + ta * Ie.dp[j], gy);
              ym = fmaf(rsj, Ie.p[j], ym);
            }
            geo_acc += gy + go_u * ym + cd_u * Ie.d[e];
          } else {
            const int e = lane - 9;
            float acc2 = 0.f;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              const float go_u = -gtm * Ie.dp[u] * inv_a - gh_ah * Ie.p[u];
              acc2 = fmaf(Gp.Mhi[u * 3 + e], rr[u] + go_u, acc2);
            }
            geo_acc -= acc2;
          }
        }
      }
    }
    (void)wait_g();  // wgrad_0 (also before the next chunk writes X)
    pend0 = true;
  }
  if (pend0) flush0();
  // teardown: no MMA may still write TMEM; the last primitive's gradients; TMEM freed
  if (issuer) {
    mma_commit(bar_e);
    mbar_wait_limit(bar_e, 0, kWaitNsW);
  }
  tc_fence_before();
  __syncthreads();
  if (loaded >= 0) flush_prim(loaded);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemColsW);
  }
  if (threadIdx.x == 0 && *sAbort) set_status(w.scr_hdr, MLPS_ERR_TIMEOUT);
}

}  // namespace tc

// ------------------------------------------------------------------------------------------
// Host side

// The tensor-core backward at hidden width 128 (tc model `m`): midpoint samples with the
// configurations' encodings (xyz L = 6, direction L = 4: 60 inputs in one slab), up to 16
// feature outputs, every output count and weight offset a multiple of 4 (the weight-gradient
// copy's 16-byte vectors), and its shared memory within the SM's.
bool tc_bwd_wide_supported(const Model& m, const TcPlan& P) {
  if (m.width != 128 || m.nl < 2 || m.nl > 5 || m.contact) return false;
  if (m.xyzL != 6 || m.dirL != 4 || P.kpad[0] != 64) return false;
  if (m.F > 16 || m.nout > 32) return false;
  if (m.P % 4 != 0) return false;
  for (int l = 0; l < m.nl; ++l)
    if (m.dout[l] % 4 != 0 || m.woff[l] % 4 != 0) return false;
  const int ipc = m.S <= 128 ? 128 / m.S : 1;
  return tc::wide_layout(P, 32, ipc).total + 1024 <= 227 * 1024;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode_w() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

cudaError_t launch_mlp_bwd_tc_wide(const Work& w, const MlpArgs& a, const TcPlan& P, int n_sm,
                                   cudaStream_t st) {
  if (!tc_bwd_wide_supported(a.m, P) || !w.dwb) return cudaErrorNotSupported;
  auto encode = get_encode_w();
  if (!encode) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t dims[2] = {64, (cuuint64_t)w.K * (cuuint64_t)P.rows_per_prim};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {64, 16};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<unsigned char*>(a.weights),
                      dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = tc::wide_layout(P, 32, w.ipc).total + 1024;
  auto kern = a.m.F > 0 ? tc::k_mlp_bwd_tc_wide<16, 6, 4> : tc::k_mlp_bwd_tc_wide<0, 6, 4>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_sm, tc::kWThreads, smem, st>>>(w, a, P, tmap);
  return cudaGetLastError();
}

}  // namespace mlps
