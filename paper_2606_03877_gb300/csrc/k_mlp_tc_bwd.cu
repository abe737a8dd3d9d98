// k_mlp_tc_bwd.cu -- BF16 tensor-core (tcgen05) backward of the grouped per-primitive MLP stage.
//
// Per chunk of 128 sample rows of one primitive (same chunks as the forward pass), one epilogue
// group (4 warps, thread = sample row; three groups, i.e. three chunks in flight per SM) runs
// 2 * nl phases:
//   F_l  (l = 0 .. nl-1): Z_l = H_l W_l^T recomputes the forward; the epilogue writes
//        H_{l+1} = ReLU(Z_l + b_l) as BF16 into the group's tile T_{l+1};
//   B_l  (l = nl-1 .. 0): dgrad  G = delta_l W_l          (A = delta_l, K-major; B = the forward
//                                W_l tile read MN-major)
//                         wgrad  dW_l^T += H_l^T delta_l  (A = H_l, B = delta_l, both read as
//                                MN-major views of the same swizzled tiles; M = 128: the 64
//                                input features of H_l plus a constant "ones" atom, so that
//                                row 64 of the accumulator collects the bias gradient
//                                sum_rows delta_l); the epilogue forms
//                                delta_{l-1} = G * [H_l > 0] in place of H_l.
// The MMAs of a phase are issued by the group's first thread right after a group-local barrier.
// dgrad and wgrad complete on separate mbarriers: the epilogue of B_l starts once its dgrad is
// done and waits for the wgrad (which still reads H_l) only before delta_{l-1} overwrites H_l.
// delta_{nl-1} = dL/dZ comes from the last forward epilogue: the reverse of the interval
// composite of Eq. 6 with segmented suffix scans (see k_mlp_simt_bwd.cu for the formulas).
// The input-encoding gradient G_enc = delta_0 W_0 feeds the encoding derivative and the pose
// chain (closest-point form, no cancellation), reduced per interval and per block.
// The weight-gradient accumulators live in TMEM for the whole primitive segment of the block and
// are shared by the groups: they are cleared with tcgen05.st when the block starts a primitive,
// every wgrad MMA accumulates into them, and they are flushed to global memory with one
// atomicAdd per entry when the primitive changes.
// Tiles per group (nl of them, so that three chunks fit in shared memory): T_0 = H_0 (the
// encoded input), then dL/dZ once the forward is done, then H_0 again (rebuilt for the last
// wgrad once dL/dZ has been consumed); T_l = H_l, then delta_{l-1}. The per-interval sums of the
// pose chain reduce to two 3-vectors per interval, because the sample positions are affine in
// the sample index.
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

using simt::IntervalInfo;

namespace {

// Epilogue groups (chunks in flight per SM): 3 where their tiles fit in shared memory and their
// accumulators next to the weight gradients in TMEM, else 2 (template parameter NG).
constexpr int kGThreads = kEGThreads;               // 4 warps, one per TMEM lane quarter
constexpr uint32_t kTmemColsB = 512;  // per group kGColsB, per layer 64 of weight gradients (16
                                      // for the head layer)
constexpr uint32_t kGColsB = 96;      // per group: accumulator (64) + A operand (32 columns of BF16 pairs)

// TMEM columns of the weight gradients: 64 per layer, the head layer (npad <= 16) last with 16.
MLPS_HD int dw_cols(int nl) { return (nl - 1) * 64 + 16; }
constexpr uint64_t kWaitNsB = 2000000000ull;
constexpr uint32_t kTile = kM * 128;                // one [128 x 64] BF16 tile
constexpr uint32_t kOnes = 2048;                    // 16 rows of the MN-major ones atom (one K step)

// Byte offsets in dynamic shared memory; per-group regions are base + g * stride. The group's
// interval tables hold ipc = 128 / S entries.
struct BwdSmem {
  uint32_t w, tiles0, tiles_stride, ones, bias, grp0, grp_stride, tab_stride, itab, giv, ddel, gf, scan, geo,
      pgeo, bars, misc, total;  // itab/giv/ddel/gf: offsets inside one group's block
};

MLPS_HD uint32_t al(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Values per warp of the widest segmented scan (pose chain: 6; reverse composite: 3 + NF).
MLPS_HD int scan_vals(int F) { return F > 0 ? 3 + 12 : 6; }

MLPS_HD BwdSmem bwd_layout(const TcPlan& P, int F, int ipc, int kNG) {
  BwdSmem L;
  uint32_t o = 0;
  L.w = o;
  o = al(o + P.w_bytes, 1024);
  L.tiles0 = o;
  // T_0 (kpad0 / 64 slabs: the encoded input) .. T_{nl-1}
  L.tiles_stride = al((uint32_t)(P.kpad[0] / 64 + P.nl - 1) * kTile, 1024);
  o += L.tiles_stride * kNG;
  L.ones = o;  // above every group tile: the wgrad descriptors reach it with a positive offset
  o = al(o + kOnes, 1024);
  L.bias = o;
  o = al(o + 4 * P.bias_floats, 16);
  // per group: two buffers (tab_stride apart) of the chunk's interval records (itab),
  // gradients (giv) and feature gradients (gf), then the per-interval dL/d delta (ddel)
  uint32_t q = 0;
  L.itab = q;
  q = al(q + (uint32_t)sizeof(IntervalRec) * ipc, 16);
  L.giv = q;
  q = al(q + 16 * ipc, 16);
  L.gf = q;
  q = al(q + 4 * ipc * (F > 0 ? F : 1), 16);
  L.tab_stride = q;
  q += q;
  L.ddel = q;
  q = al(q + 4 * ipc, 16);
  L.grp0 = o;
  L.grp_stride = q;
  o += q * kNG;
  L.scan = o;  // per group and warp, the widest scan of the kernel: 6 values, or 3 + 12 with features
  o = al(o + 4 * kNG * 4 * scan_vals(F), 16);
  L.geo = o;
  o = al(o + 4 * 16, 16);
  L.pgeo = o;  // the current primitive's geometry (staged at every primitive change)
  o = al(o + (uint32_t)sizeof(PrimGeo), 16);
  L.bars = o;
  o = al(o + 8 * (2 + 3 * kNG), 16);
  L.misc = o;
  o = al(o + 16, 16);
  L.total = o;
  return L;
}

// dgrad of phase B_l, issued by one thread of the group: G = delta_l W_l into the group's
// accumulator, K = npad (outputs of layer l), N = kpad (its inputs). A = delta_l in tensor memory
// (`At`: lane = sample row, BF16 pairs along the columns, 8 columns per K = 16 step); B = the
// forward W_l tile read as an MN-major operand (inputs contiguous, outputs = K rows).
MLPS_DEV void issue_dgrad_ta(uint32_t At, uint32_t wtile, uint32_t acc, int kpad, int npad) {
  const uint32_t id = idesc_bf16(kM, kpad) | (1u << 16);
  const uint64_t db = sw128_desc_mn(wtile, 16);
  const int nk = npad / 16;  // npad <= 64
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    if (kk >= nk) break;
    mma_bf16_ta(acc, At + 8u * (uint32_t)kk, db + (uint64_t)(kk * 128), id, kk > 0 ? 1u : 0u);
  }
}

// wgrad of phase B_l: dW_l^T[in (+ones)][out] += H_l^T delta_l over the 128 rows (K = rows).
// A = [H_l | ones] as MN-major atoms (the ones atom's offset is given per K step, so a single
// 16-row ones block serves every step); B = delta_l MN-major, N = npad (outputs of layer l).
// Always accumulates: the accumulator is cleared when the block starts a primitive. Stepping K
// moves A's start address up and its atom offset (LBO, descriptor bits 16..29) down by 2 KB.
MLPS_DEV void issue_wgrad(uint32_t Hl, uint32_t Dl, uint32_t dw_l, uint32_t ones, int npad) {
  const uint32_t id = idesc_bf16(kM, npad) | (1u << 15) | (1u << 16);
  const uint64_t da = sw128_desc_mn(Hl, ones - Hl), db = sw128_desc_mn(Dl, 16);
#pragma unroll
  for (int kk = 0; kk < kM / 16; ++kk) {
    const uint64_t step = (uint64_t)(kk * 128);
    mma_bf16(dw_l, da + step - (step << 16), db + step, id, 1u);
  }
}

}  // namespace

// Contact-point input row (Eq. 4) of one hit into the two-slab tile `A`, in the tensor-core
// blob's column order gamma(delta), gamma(d) (tc_in_col), then a constant 1 in the first padding
// column `nin`: multiplied by nothing in the forward pass (the weights there are zero), it makes
// row nin of wgrad_0's accumulator the bias gradient of the first layer.
MLPS_DEV void build_row_contact(const Model& m, const PrimGeo& G, const IntervalRec* T, int nint, int row,
                                uint32_t A) {
  RowWriter rw{A, row, 0, 0.f};
  if (row < nint) {
    const IntervalRec& I = T[row];
    float del[3];
    contact_delta(G, I, del);
    if (m.xyzL == 0) {
      for (int u = 0; u < 3; ++u) rw.put(del[u]);
    } else {
      for (int u = 0; u < 3; ++u) put_gamma(rw, del[u], m.xyzL);
    }
    if (m.dirL > 0)
      for (int u = 0; u < 3; ++u) put_gamma(rw, I.d[u], m.dirL);
    rw.put(1.f);
  }
  rw.pad_to(128);
}

// wgrad of the first layer with a two-slab input (kpad0 = 128): A = [X slab 0 | X slab 1] as two
// MN-major atoms 16 KB apart (M = 128 inputs, the constant-1 column giving the bias gradient),
// B = delta_0 MN-major, N = npad; K = the 128 rows.
MLPS_DEV void issue_wgrad2(uint32_t X, uint32_t Dl, uint32_t dw, int npad) {
  const uint32_t id = idesc_bf16(kM, npad) | (1u << 15) | (1u << 16);
  const uint64_t da = sw128_desc_mn(X, kTile), db = sw128_desc_mn(Dl, 16);
#pragma unroll
  for (int kk = 0; kk < kM / 16; ++kk) mma_bf16(dw, da + (uint64_t)(kk * 128), db + (uint64_t)(kk * 128), id, 1u);
}

// CT: the contact-point model (Sec. 3.2): one sample per hit (S = 1), input [gamma(delta);
// gamma(d)] over two 64-column slabs with XL, DL their frequencies, the pose chain of Eq. 3.
template <int NF, int XL, int DL, int kNG, bool CT = false>
__global__ void __launch_bounds__(kGThreads * kNG, 1)
    k_mlp_bwd_tc(Work w, MlpArgs a, TcPlan P, const __grid_constant__ CUtensorMap tmap) {
  constexpr int kThreadsB = kGThreads * kNG;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* gb = smem_raw + (sbase - raw);
  const Model& m = a.m;
  const int F = m.F;
  static_assert(14 <= kMaxScanVals && 3 + NF <= kMaxScanVals, "scan scratch holds kMaxScanVals values per warp");
  static_assert(4 + NF <= 16 && NF % 2 == 0, "the head's outputs lie in the first 16 columns");
  constexpr int kScanNV = NF > 0 ? 3 + 12 : 6;  // = scan_vals(F) of the layout
  static_assert(NF == 0 || NF == 12, "feature heads are instantiated with NF = 12");
  const BwdSmem L = bwd_layout(P, F, w.ipc, kNG);
  float* sBias = reinterpret_cast<float*>(gb + L.bias);
  float* sScan = reinterpret_cast<float*>(gb + L.scan);
  float* sGeo = reinterpret_cast<float*>(gb + L.geo);
  const uint32_t bar_w = sbase + L.bars;
#define bar_end(G) (bar_w + 16u + 8u * (uint32_t)(G))
#define bar_done(G) (bar_w + 16u + 8u * (uint32_t)(kNG) + 8u * (uint32_t)(G))
#define bar_wg(G) (bar_w + 16u + 16u * (uint32_t)(kNG) + 8u * (uint32_t)(G))
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(gb + L.misc);
  volatile int* sAbort = reinterpret_cast<volatile int*>(gb + L.misc + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = m.nl, S = m.S;
  const int g = warp >> 2, q = warp & 3;          // group, TMEM lane quarter
  const int row = q * 32 + lane;                  // sample row within the chunk
  const int gbar = 1 + g;                         // the group's named barrier
  const bool issuer = row == 0;                   // issues the group's MMAs

  if (threadIdx.x == 0) {
    mbar_init(bar_w, 1);
    for (int gg = 0; gg < kNG; ++gg) {
      mbar_init(bar_done(gg), 1);
      mbar_init(bar_wg(gg), 1);
      mbar_init(bar_end(gg), 1);
    }
    *sAbort = 0;
    fence_mbar_init();
  }
  // constant ones atom: element 0 of every row is 1.0 (BF16 0x3F80)
  for (int i = threadIdx.x; i < (int)(kOnes / 16); i += kThreadsB) {
    const int r = i >> 3, ch = i & 7;
    const uint32_t one = ((ch ^ (r & 7)) == 0) ? 0x3F80u : 0u;  // chunk 0 of row r lands at r & 7
    st_shared_v4(sbase + L.ones + (uint32_t)i * 16, one, 0u, 0u, 0u);
  }
  if (threadIdx.x < 16) sGeo[threadIdx.x] = 0.f;
  fence_proxy_async_smem();
  if (warp == 0) {
    tmem_alloc(sbase + L.misc, kTmemColsB);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t tm_dw = tmem + kGColsB * kNG;  // weight-gradient accumulators: 64 columns per layer

  const int total = walk_chunk_count(w);
  const int* const bmap = walk_map(w);  // list position -> forward position
  const int cb = (int)((long long)total * blockIdx.x / gridDim.x);
  const int ce = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  // phase parities of bar_w and of this group's bar_done (forward layers and dgrad) and bar_wg
  // (wgrad). Each barrier gets its next commit only after its previous phase was waited for, so
  // it is never two phases ahead of its waiters (a parity wait could not tell those apart).
  uint32_t ph_w = 0, ph = 0, ph_g = 0;
  float geo_acc = 0.f;  // pose-chain output `lane` (< 12) of the current primitive, this warp's share
  const float invS = 1.f / (float)S;
  int loaded = -1;
  int prim = cb < ce ? simt::find_prim(w, cb) : 0;

  // the next completion of the group's MMAs (warp-uniform: tcgen05.ld is a warp instruction)
  auto wait_mma = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_done(g), ph, sAbort, kWaitNsB));
    ph ^= 1u;
    tc_fence_after();
    return ok;
  };
  auto wait_wgrad = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_wg(g), ph_g, sAbort, kWaitNsB));
    ph_g ^= 1u;
    tc_fence_after();
    return ok;
  };
  // wgrad_0 of the group's last chunk may still read T_0 and T_1: waited for before the next
  // write of either tile, before a flush of the weight gradients, and at teardown
  bool wg_pending = false;

  // flush of the block's accumulated gradients of primitive p (all threads call it)
  auto flush = [&](int p) {
    if (warp < 4) {
      tc_fence_after();
      float* dW = a.d_weights + (size_t)p * m.Prow;
      const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
      const int frow = warp * 32 + lane;
      for (int l = 0; l < nl; ++l) {
        const int din = m.din[l], dout = m.dout[l];
        for (int c0 = 0; c0 < (l == nl - 1 ? 16 : 64); c0 += 32) {
          uint32_t v[32];
          if (l == nl - 1) {  // the head layer's 16 columns
            uint32_t v16[16];
            tmem_ld16(tm_dw + (uint32_t)(l * 64) + lanebase, v16);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = j < 16 ? v16[j & 15] : 0u;
          } else {
            tmem_ld32(tm_dw + (uint32_t)(l * 64 + c0) + lanebase, v);
          }
          tmem_wait_ld();
          if (*sAbort) continue;
          // accumulator row of the bias gradient: the ones atom's (64), or for a two-slab input
          // the constant-1 column after the encoded input (build_row_contact)
          const int brow = (l == 0 && P.kpad[0] > 64) ? din : 64;
          const int col = tc_in_col(m, l, frow);
          for (int j = 0; j < 32; ++j) {
            const int n = c0 + j;
            const float val = __uint_as_float(v[j]);
            if (n >= dout || val == 0.f) continue;
            if (frow < din) atomicAdd(&dW[m.woff[l] + n * din + col], val);
            else if (frow == brow) atomicAdd(&dW[m.boff[l] + n], val);
          }
        }
      }
      tc_fence_before();
    }
    if (threadIdx.x < 12) {
      const float v = sGeo[threadIdx.x];
      if (v != 0.f) atomicAdd(&w.dgeo[12 * (size_t)p + threadIdx.x], v);
      sGeo[threadIdx.x] = 0.f;
    }
  };
  // the next chunk's interval records and interval gradients, one step ahead, copied with
  // cp.async into the group's pending table buffer `pb` (no registers held across the chunk)
  uint8_t* grp = gb + L.grp0 + (uint32_t)g * L.grp_stride;
  int pb = 0;
  auto prefetch = [&](const ChunkStep<kNG>& st, int c) {
    const int f = (c - w.chunk_start[st.prim]) * w.ipc;
    if (row < min(w.ipc, w.prim_count[st.prim] - f)) {
      const uint32_t t = smem_u32(grp) + (uint32_t)pb * L.tab_stride;
      rec_copy_async(w, walk_slot(bmap, w.prim_start[st.prim] + f + row), t + L.itab + 64u * (uint32_t)row,
                     t + L.giv + 16u * (uint32_t)row);
    }
  };

  ChunkStep<kNG> cur = chunk_step<kNG>(w, cb, ce, prim);
  const int my_first = step_chunk(cur, g);
  if (cur.n > 0 && my_first >= 0) prefetch(cur, my_first);
  while (cur.c0 < ce) {
    prim = cur.prim;
    const ChunkStep<kNG> nxt = chunk_step<kNG>(w, cur.c0 + cur.n, ce, prim);
    const int my_cc = step_chunk(cur, g);  // this group's chunk this step and the next
    const int my_nx = step_chunk(nxt, g);
    if (prim != loaded) {
      if (wg_pending) {  // the flush reads the accumulators that wgrad_0 adds to
        (void)wait_wgrad();
        wg_pending = false;
      }
      if (geo_acc != 0.f) atomicAdd(&sGeo[lane], geo_acc);  // nonzero only on lanes < 12
      geo_acc = 0.f;
      tc_fence_before();
      __syncthreads();
      if (loaded >= 0) flush(loaded);
      if (warp < 4) {  // clear the weight-gradient accumulators for the new primitive
        const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
        for (int c0 = 0; c0 < (nl - 1) * 64; c0 += 32) tmem_st32_zero(tm_dw + (uint32_t)c0 + lanebase);
        tmem_st16_zero(tm_dw + (uint32_t)((nl - 1) * 64) + lanebase);
        tmem_wait_st();
      }
      tc_fence_before();
      __syncthreads();
      if (threadIdx.x == 0 && !*sAbort) {
        mbar_arrive_expect_tx(bar_w, (uint32_t)P.w_bytes);
        const int row0 = prim * P.rows_per_prim;
        for (int l = 0; l < nl; ++l)
          for (int sl = 0; sl < P.kpad[l] / 64; ++sl)
            for (int j = 0; j < P.npad[l] / 16; ++j)
              tma_load_2d(sbase + L.w + P.sw_off[l] + sl * P.npad[l] * 128 + j * 2048, &tmap, 0,
                          row0 + P.gw_row[l] + sl * P.npad[l] + j * 16, bar_w);
      }
      const float* gbias = reinterpret_cast<const float*>(a.weights + (size_t)prim * a.pk.stride + P.gbias_byte);
      for (int i = threadIdx.x; i < P.bias_floats; i += kThreadsB) sBias[i] = gbias[i];
      {
        const int* src = reinterpret_cast<const int*>(w.geo + prim);
        int* dst = reinterpret_cast<int*>(gb + L.pgeo);
        for (int i = threadIdx.x; i < (int)(sizeof(PrimGeo) / 4); i += kThreadsB) dst[i] = src[i];
      }
      mbar_wait(bar_w, ph_w, sAbort, kWaitNsB);
      ph_w ^= 1;
      __syncthreads();
      loaded = prim;
    }

    if (my_cc < 0) {
      if (nxt.n > 0 && my_nx >= 0) prefetch(nxt, my_nx);  // idle this step: still prefetch
      cur = nxt;
      continue;
    }
    // ============================================================ epilogue group g
    const int first = (my_cc - w.chunk_start[prim]) * w.ipc;
    const int nint = min(w.ipc, w.prim_count[prim] - first);
    // this chunk's tables are in buffer pb (copied during the previous step); the other buffer
    // was last read by the chunk before the previous one, so no barrier is needed before it is
    // refilled
    uint8_t* tb = grp + (uint32_t)pb * L.tab_stride;
    IntervalRec* T = reinterpret_cast<IntervalRec*>(tb + L.itab);
    float4* GI = reinterpret_cast<float4*>(tb + L.giv);
    float* DD = reinterpret_cast<float*>(grp + L.ddel);
    float* GF = reinterpret_cast<float*>(tb + L.gf);
    cp_async_wait_all();  // this thread's copies of the chunk's records and gradients landed
    if (F > 0 && row < nint) {
      const size_t slot = walk_slot(bmap, w.prim_start[prim] + first + row);
      for (int f = 0; f < F; ++f) GF[row * F + f] = w.hit_gfeat[slot * F + f];
    }
    named_bar_sync(gbar, kGThreads);  // everyone's did
    pb ^= 1;
    if (nxt.n > 0 && my_nx >= 0) prefetch(nxt, my_nx);  // start loading the next chunk now
    const uint32_t tiles = sbase + L.tiles0 + (uint32_t)g * L.tiles_stride;
    const int t0s = P.kpad[0] / 64;  // slabs of T_0
#define tileaddr(I) (tiles + (uint32_t)((I) == 0 ? 0 : (CT ? t0s + (I) - 1 : (I))) * kTile)
    const int iv = row / S, k = row - iv * S;
    const bool valid = iv < nint;
    const uint32_t acc = tmem + (uint32_t)g * kGColsB;  // this group's dgrad / forward accumulator
    const uint32_t trow = acc + ((uint32_t)(q * 32) << 16);

    const uint32_t aT = acc + 64u;  // A operand in TMEM: 32 columns of BF16 pairs
    const uint32_t arow = aT + ((uint32_t)(q * 32) << 16);
    if constexpr (CT) {  // contact-point input (two slabs) through the shared-memory tile T_0
      if (wg_pending) {
        (void)wait_wgrad();
        wg_pending = false;
      }
      build_row_contact(m, *reinterpret_cast<const PrimGeo*>(gb + L.pgeo), T, nint, row, tileaddr(0));
      fence_proxy_async_smem();
    } else if (DL >= 0) {  // encoded input straight into the A operand in TMEM
      uint32_t pk[32];
      encode_row64<XL, (DL > 0 ? DL : 0)>(T, nint, S, row, pk);
      tmem_st32(arow, pk);
      tmem_wait_st();
    } else {  // generic encodings: through the shared-memory tile T_0 (free once wgrad_0 is done)
      if (wg_pending) {
        (void)wait_wgrad();
        wg_pending = false;
      }
      build_row(m, T, nint, row, tileaddr(0), P.kpad[0]);
      fence_proxy_async_smem();
    }
    tc_fence_before();
    named_bar_sync(gbar, kGThreads);
    if (issuer) {
      tc_fence_after();
      if (!*sAbort) {
        if (DL >= 0 && !CT) issue_fwd_layer_ta(aT, sbase + L.w + P.sw_off[0], acc, P.kpad[0], P.npad[0]);
        else issue_fwd_layer(tileaddr(0), sbase + L.w + P.sw_off[0], acc, P.kpad[0], P.npad[0]);
      }
      mma_commit(bar_done(g));
    }

    // ---------------- forward recompute
    // (after a wait that gave up, the kernel still walks its chunks with whatever TMEM holds,
    // issuing no MMA: the outputs are then void and the status word says MLPS_ERR_TIMEOUT)
    for (int l = 0; l < nl; ++l) {
      (void)wait_mma();
      const float* bias = sBias + P.bias_off[l];
      if (l < nl - 1) {
        uint32_t pk[32];
        {
          uint32_t v0[32], v1[32];
          tmem_ld32(trow, v0);
          tmem_ld32(trow + 32, v1);
          tmem_wait_ld();
          const float4* b4 = reinterpret_cast<const float4*>(bias);
#pragma unroll
          for (int e4 = 0; e4 < 16; ++e4) {
            const float4 bq = b4[e4];
            const int c0 = 4 * e4;
            float x0 = __uint_as_float(c0 < 32 ? v0[c0] : v1[c0 - 32]);
            float x1 = __uint_as_float(c0 + 1 < 32 ? v0[c0 + 1] : v1[c0 + 1 - 32]);
            float x2 = __uint_as_float(c0 + 2 < 32 ? v0[c0 + 2] : v1[c0 + 2 - 32]);
            float x3 = __uint_as_float(c0 + 3 < 32 ? v0[c0 + 3] : v1[c0 + 3 - 32]);
            add2_f32(x0, x1, bq.x, bq.y);
            add2_f32(x2, x3, bq.z, bq.w);
            pk[2 * e4] = pack_bf16_relu(x0, x1);
            pk[2 * e4 + 1] = pack_bf16_relu(x2, x3);
          }
        }
        tmem_st32(arow, pk);  // H_{l+1}: A operand of the next layer
        tmem_wait_st();
        tc_fence_before();
        named_bar_sync(gbar, kGThreads);
        if (issuer) {
          tc_fence_after();
          if (!*sAbort)
            issue_fwd_layer_ta(aT, sbase + L.w + P.sw_off[l + 1], acc, P.kpad[l + 1], P.npad[l + 1]);
          mma_commit(bar_done(g));
        }
        if (wg_pending) {  // the previous chunk's wgrad_0 reads T_0 and T_1
          (void)wait_wgrad();
          wg_pending = false;
        }
        // H_{l+1} also goes to T_{l+1}: the ReLU mask of B_{l+1} and the A operand of wgrad_{l+1}
        // (made visible to the tensor core by the proxy fence before the head's barrier). It is
        // read back from TMEM (the MMA only reads it too), so pk need not live across the issue.
        {
          uint32_t hv[32];
          tmem_ld32(arow, hv);
          tmem_wait_ld();
          store_row64(tileaddr(l + 1), row, hv);
        }
      } else {
        // ---------------- heads and reverse of the interval composite -> dL/dZ into T_0
        float z[4 + NF];
        {
          uint32_t r16[16];
          tmem_ld16(trow, r16);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 4 + NF; ++j) z[j] = j < m.nout ? __uint_as_float(r16[j]) + bias[j] : 0.f;
        }
        tc_fence_before();
        const IntervalRec& I = T[valid ? iv : 0];
        const float dt = valid ? I.dt : 0.f;
        const float sig = softplus_fast(z[3]);
        const float ak = valid ? sig * dt : 0.f;
        float sc1[1] = {ak};
        seg_scan<1>(sc1, 1, row, S, sScan + g * 4 * kScanNV, gbar);
        const float Aex = sc1[0] - ak;
        const float tau = __expf(-Aex), ea = __expf(-ak);
        const float wk = valid ? tau * (1.f - ea) : 0.f;
        float cq[3];
        for (int u = 0; u < 3; ++u) cq[u] = sigmoid_fast(z[u]);
        float sv[3 + NF];
#pragma unroll
        for (int u = 0; u < 3; ++u) sv[u] = wk * cq[u];
#pragma unroll
        for (int f = 0; f < NF; ++f) sv[3 + f] = f < F ? wk * z[4 + f] : 0.f;
        seg_scan_rev<3 + NF>(sv, 3 + F, row, S, sScan + g * 4 * kScanNV, gbar);
        const float4 gI = valid ? GI[iv] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float gcs[3] = {gI.x, gI.y, gI.z};
        float dLda = gI.w;
#pragma unroll
        for (int u = 0; u < 3; ++u) dLda += gcs[u] * (tau * ea * cq[u] - (sv[u] - wk * cq[u]));
        float dz[4 + NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const float gf = (valid && f < F) ? GF[iv * F + f] : 0.f;
          const float fk = z[4 + f];
          dLda += gf * (tau * ea * fk - (sv[3 + f] - wk * fk));
          dz[4 + f] = wk * gf;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) dz[u] = wk * gcs[u] * cq[u] * (1.f - cq[u]);
        dz[3] = valid ? dLda * dt * sigmoid_fast(z[3]) : 0.f;
        float dd[1] = {valid ? sig * dLda : 0.f};
        seg_scan<1>(dd, 1, row, S, sScan + g * 4 * kScanNV, gbar);
        if (valid && k == S - 1) DD[iv] = dd[0];
        uint32_t pk[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) pk[e] = 0u;
#pragma unroll
        for (int e = 0; e < (4 + NF) / 2; ++e)
          pk[e] = pack_bf16(2 * e < m.nout ? dz[2 * e] : 0.f, 2 * e + 1 < m.nout ? dz[2 * e + 1] : 0.f);
        // delta_{nl-1} (16 columns): A operand of dgrad_{nl-1} in TMEM, and B operand of
        // wgrad_{nl-1} in T_0 (X is dead there: F_0 is done; it is rebuilt for wgrad_0)
        tmem_st16(arow, pk);
        st_shared_v4(tileaddr(0) + sw128_off(row, 0), pk[0], pk[1], pk[2], pk[3]);
        st_shared_v4(tileaddr(0) + sw128_off(row, 1), pk[4], pk[5], pk[6], pk[7]);
        tmem_wait_st();
        fence_proxy_async_smem();  // also covers the H tiles written during the recompute
        tc_fence_before();
        named_bar_sync(gbar, kGThreads);
        if (issuer) {  // B_{nl-1}: dgrad, then wgrad (complete once the next dgrad is)
          tc_fence_after();
          if (!*sAbort) issue_dgrad_ta(aT, sbase + L.w + P.sw_off[nl - 1], acc, P.kpad[nl - 1], P.npad[nl - 1]);
          mma_commit(bar_done(g));
          if (!*sAbort)
            issue_wgrad(tileaddr(nl - 1), tileaddr(0), tm_dw + (uint32_t)((nl - 1) * 64), sbase + L.ones, P.npad[nl - 1]);
        }
      }
    }
    // ---------------- backward phases B_{nl-1} .. B_0
    // On entry to B_l, dgrad_l is issued with A = delta_l in TMEM; B_l issues dgrad_{l-1} and then
    // wgrad_l, whose B operand is delta_l's copy in shared memory, tile D(l) (below). A commit
    // arrives once every earlier MMA of its thread is complete, so when dgrad_l is done, every
    // wgrad issued before it (wgrad_m for m >= l + 2, and wgrad_{nl-1}) is done too, and their
    // tiles are free: D(nl-1) = D(nl-2) = T_0, D(l) = T_{l+2} for l <= nl-3. No B phase waits for
    // a wgrad, except B_0 with three layers (X then needs T_1, still read by wgrad_1).
#define dtile(I) ((I) >= nl - 2 ? tileaddr(0) : tileaddr((I) + 2))
    for (int l = nl - 1; l >= 0; --l) {
      (void)wait_mma();  // dgrad of B_l (and every wgrad issued before it)
      if (l > 0 && l < nl - 1) {
        // delta_l (A operand of dgrad_l, done) from TMEM to its tile D(l), 16 columns at a time
        uint32_t dl[32];
        tmem_ld32(arow, dl);
        tmem_wait_ld();
        store_row64(dtile(l), row, dl);
      }
      if (l > 0) {
        // delta_{l-1} = G * [H_l > 0] (H_l from T_l; wgrad_l, which reads it, is issued below),
        // 32 columns of G at a time
        const uint32_t Tl = tileaddr(l);
        const uint32_t vmask = valid ? 0xFFFFFFFFu : 0u;
        const RowSw sw(row);
        uint32_t pk[32];
        uint32_t v2[2][32];
        tmem_ld32(trow, v2[0]);
        tmem_ld32(trow + 32u, v2[1]);
        tmem_wait_ld();
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const uint32_t (&v)[32] = v2[hf];
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) {
            uint32_t hq[4];
            ld_shared_v4(Tl + sw.off(4 * hf + ch), hq[0], hq[1], hq[2], hq[3]);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c0 = ch * 8 + 2 * e;
              // H_l was written by the ReLU pack, so each BF16 half is +0 or positive: H > 0 iff
              // the half is nonzero (one packed compare for both halves)
              pk[(4 * hf + ch) * 4 + e] =
                  pack_bf16(__uint_as_float(v[c0]), __uint_as_float(v[c0 + 1])) & bf16x2_nonzero(hq[e]) & vmask;
            }
          }
        }
        tc_fence_before();
        tmem_st32(arow, pk);  // delta_{l-1}: A operand of dgrad_{l-1}
        tmem_wait_st();
        fence_proxy_async_smem();
        tc_fence_before();
        named_bar_sync(gbar, kGThreads);
        if (issuer) {
          tc_fence_after();
          // into the first layer only its first input slab: every input the pose chain needs
          // (the contact model's gamma(delta) comes first there)
          if (!*sAbort)
            issue_dgrad_ta(aT, sbase + L.w + P.sw_off[l - 1], acc, l == 1 ? 64 : P.kpad[l - 1], P.npad[l - 1]);
          mma_commit(bar_done(g));
          if (l < nl - 1) {
            if (!*sAbort) issue_wgrad(Tl, dtile(l), tm_dw + (uint32_t)(l * 64), sbase + L.ones, P.npad[l]);
            if (nl == 3 && l == 1) mma_commit(bar_wg(g));  // B_0 waits for it before writing X into T_1
          }
        }
      } else {
        uint32_t v0[32], v1[32];
        tmem_ld32(trow, v0);
        tmem_ld32(trow + 32, v1);
        tmem_wait_ld();
        tc_fence_before();
        if constexpr (CT) {
          // ---------------- contact-point chain (Eq. 3-4), one hit per row: dL/d delta from
          // gamma(delta)'s derivative (the first 6 XL columns), then the pose contributions of
          // the hit (see chain_pose of the FP32 path for the formulas), summed over the warp;
          // lane j < 12 keeps output j
          const PrimGeo& Gp = *reinterpret_cast<const PrimGeo*>(gb + L.pgeo);
          float out[12];
#pragma unroll
          for (int j = 0; j < 12; ++j) out[j] = 0.f;
          if (valid) {
            const IntervalRec& I = T[iv];
            float del[3], gd[3];
            contact_delta(Gp, I, del);
            enc_grad64<XL>(del, v0, v1, gd);
            const float dDelta = DD[iv];
            const bool clamped = I.r0 != -I.r1;
            const float gtd = I.tmid > 0.f ? -(gd[0] * I.d[0] + gd[1] * I.d[1] + gd[2] * I.d[2]) : 0.f;
            const float gtm = dDelta + (clamped ? 0.f : -dDelta) + gtd;
            const float gh = dDelta - (clamped ? 0.f : -dDelta);
            const float aa = I.dp[0] * I.dp[0] + I.dp[1] * I.dp[1] + I.dp[2] * I.dp[2];
            const float inv_a = 1.f / aa;
            const float hh = I.r1;
            const float gh_ah = hh > 0.f ? gh * inv_a / hh : 0.f;
            float go[3], cd[3], ym[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
              go[u] = -gtm * I.dp[u] * inv_a - gh_ah * I.p[u];
              cd[u] = -(gtm * I.p[u] + gh * hh * I.dp[u]) * inv_a;
              ym[u] = Gp.R[u * 3] * Gp.s[0] * I.p[0] + Gp.R[u * 3 + 1] * Gp.s[1] * I.p[1] +
                      Gp.R[u * 3 + 2] * Gp.s[2] * I.p[2];
            }
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
              for (int e = 0; e < 3; ++e) out[u * 3 + e] = go[u] * ym[e] + cd[u] * I.d[e];
#pragma unroll
            for (int e = 0; e < 3; ++e)
              out[9 + e] = gd[e] - (Gp.Mhi[e] * go[0] + Gp.Mhi[3 + e] * go[1] + Gp.Mhi[6 + e] * go[2]);
          }
#pragma unroll
          for (int j = 0; j < 12; ++j) {
            float v = out[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == j) geo_acc += v;
          }
        } else {
        // ---------------- encoding derivative and pose chain
          // With x_k = p + t_k dp and t_k = tm + c_k (r1 - r0), c_k = (k + 1/2) / S - 1/2, every
          // per-interval sum the chain needs follows from A = sum_k gx_k and B = sum_k c_k gx_k.
          float gx[3] = {0.f, 0.f, 0.f};
          const IntervalRec& I = T[valid ? iv : 0];
          const float ck = ((float)k + 0.5f) * invS - 0.5f;
          if (valid) {
            const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
            float xl[3];
            for (int u = 0; u < 3; ++u) xl[u] = fmaf(tr, I.dp[u], I.p[u]);
            enc_grad64<XL>(xl, v0, v1, gx);
          }
          float red[6] = {gx[0], gx[1], gx[2], ck * gx[0], ck * gx[1], ck * gx[2]};
          seg_scan<6>(red, 6, row, S, sScan + g * 4 * kScanNV, gbar);
          // Tail of the chain, per interval ending in this warp: the segment totals are
          // broadcast from the interval's last row and lane j < 12 computes output j (dL/dM_{u,e}
          // for j = 3u + e < 9, dL/dmu_{j-9} otherwise), accumulated in a register until the
          // block's primitive changes (no shared-memory atomics per interval).
          const int wrow0 = row - lane;
          for (int r_end = (wrow0 / S + 1) * S - 1; r_end < wrow0 + 32; r_end += S) {
            const int ive = r_end / S;
            if (ive >= nint) break;  // warp-uniform
            float rr[6];
  #pragma unroll
            for (int j = 0; j < 6; ++j) rr[j] = __shfl_sync(0xffffffffu, red[j], r_end - wrow0);
            if (lane < 12) {
              const IntervalRec& Ie = T[ive];
              const PrimGeo& Gp = *reinterpret_cast<const PrimGeo*>(gb + L.pgeo);
              const float span = Ie.r1 - Ie.r0, tm = Ie.r0 + 0.5f * span;
              const float dA = rr[0] * Ie.dp[0] + rr[1] * Ie.dp[1] + rr[2] * Ie.dp[2];
              const float dB = rr[3] * Ie.dp[0] + rr[4] * Ie.dp[1] + rr[5] * Ie.dp[2];
              const float dDelta = DD[ive];
              // end-point gradients: sum_k gt_k (1 - u_k), sum_k gt_k u_k, plus the width term
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
                const float ta = tm * ru + span * rbu;  // sum_k t_k gx_k[u]
                float gy = 0.f, ym = 0.f;               // y = R diag(s) x
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
        // wgrad_0: delta_0 copied to D(0) and X rebuilt in a free tile (T_0 with four or more
        // layers: its last reader wgrad_{nl-2} is done; T_1 with two, freed by wgrad_1; T_1 after
        // waiting for wgrad_1 with three). The group waits for this last wgrad only when the next
        // chunk writes these tiles.
        {
          uint32_t dl[32];
          tmem_ld32(arow, dl);
          tmem_wait_ld();
          tc_fence_before();
          store_row64(dtile(0), row, dl);
        }
        if (nl == 3) (void)wait_wgrad();
        // the two-slab input of the contact model only fits T_0
        const uint32_t xt = (nl >= 4 || CT) ? tileaddr(0) : tileaddr(1);
        if constexpr (CT) build_row_contact(m, *reinterpret_cast<const PrimGeo*>(gb + L.pgeo), T, nint, row, xt);
        else if (DL >= 0) build_row64<XL, (DL > 0 ? DL : 0)>(T, nint, S, row, xt);
        else build_row(m, T, nint, row, xt, P.kpad[0]);
        fence_proxy_async_smem();
        named_bar_sync(gbar, kGThreads);
        if (issuer) {
          tc_fence_after();
          if (!*sAbort) {
            if (CT) issue_wgrad2(xt, dtile(0), tm_dw, P.npad[0]);
            else issue_wgrad(xt, dtile(0), tm_dw, sbase + L.ones, P.npad[0]);
          }
          mma_commit(bar_wg(g));  // every wgrad of the chunk
        }
        wg_pending = true;
      }
    }
#undef dtile
#undef tileaddr
    cur = nxt;
  }
  cp_async_wait_all();  // (every prefetch is for a chunk this group consumes; kept for safety)
  // teardown: none of this group's MMAs may still write TMEM (after an abort a group may have
  // stopped waiting for them); then the final flush, and TMEM is freed
  if (issuer) {
    mma_commit(bar_end(g));
    mbar_wait_limit(bar_end(g), 0, kWaitNsB);
  }
  if (geo_acc != 0.f) atomicAdd(&sGeo[lane], geo_acc);
  tc_fence_before();
  __syncthreads();
  if (loaded >= 0) flush(loaded);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemColsB);
  }
  if (threadIdx.x == 0 && *sAbort) set_status(w.scr_hdr, MLPS_ERR_TIMEOUT);
#undef bar_done
#undef bar_wg
#undef bar_end
}

}  // namespace tc

// ------------------------------------------------------------------------------------------
// Groups of the backward kernel for this model: 3 when their tiles fit in shared memory and
// their accumulators in TMEM, else 2; 0 when not even 2 fit.
static int bwd_groups(const Model& m, const TcPlan& P) {
  const int ipc = m.S <= 128 ? 128 / m.S : 1;
  for (int ng = 3; ng >= 1; --ng) {  // one group: the deep networks (5 or 6 hidden layers)
    if ((int)tc::kGColsB * ng + tc::dw_cols(m.nl) > (int)tc::kTmemColsB) continue;  // TMEM: groups + weight gradients
    if (tc::bwd_layout(P, m.F, ipc, ng).total + 1024 <= 227 * 1024) return ng;
  }
  return 0;
}

// `m` is the tensor-core model (hidden layers of a 32-wide model padded to 64, tc_model).
bool tc_bwd_supported(const Model& m, const TcPlan& P) {
  if (m.width != 64 || m.nl < 2) return false;
  if (m.F > 12) return false;
  for (int l = 0; l < m.nl; ++l)
    if (P.npad[l] > 64) return false;
  if (m.contact) {
    // the paper's contact-point model: gamma(delta) and gamma(d) with L = 6 (72 inputs over two
    // slabs, the constant-1 column after them), one sample per hit, no feature head
    if (m.xyzL != 6 || m.dirL != 6 || m.F != 0 || m.S != 1 || m.nl < 3) return false;
    if (P.kpad[0] != 128 || m.nin >= 128) return false;
  } else {
    if (m.xyzL != 0 && m.xyzL != 6) return false;
    if (P.kpad[0] != 64) return false;
  }
  return bwd_groups(m, P) > 0;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode_b() {
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

cudaError_t launch_mlp_bwd_tc(const Work& w, const MlpArgs& a, const TcPlan& P, int n_sm,
                              cudaStream_t st) {
  if (!tc_bwd_supported(tc_model(a.m), P)) return cudaErrorNotSupported;
  auto encode = get_encode_b();
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
  const int ng = bwd_groups(a.m, P);
  const size_t smem = tc::bwd_layout(P, a.m.F, w.ipc, ng).total + 1024;
  // compile-time encodings for the configurations' shapes (xyz L = 6 with dir L = 4, raw xyz
  // without direction); anything else builds rows through the generic writer (DL = -1)
  const bool f = a.m.F > 0;
  const int xl = a.m.xyzL, dl = a.m.dirL;
#define MLPS_BWD_KERN(NG)                                                                        \
  ((xl == 6 && dl == 4)   ? (f ? tc::k_mlp_bwd_tc<12, 6, 4, NG> : tc::k_mlp_bwd_tc<0, 6, 4, NG>)   \
   : (xl == 0 && dl == 0) ? (f ? tc::k_mlp_bwd_tc<12, 0, 0, NG> : tc::k_mlp_bwd_tc<0, 0, 0, NG>)   \
   : (xl == 6)            ? (f ? tc::k_mlp_bwd_tc<12, 6, -1, NG> : tc::k_mlp_bwd_tc<0, 6, -1, NG>) \
                          : (f ? tc::k_mlp_bwd_tc<12, 0, -1, NG> : tc::k_mlp_bwd_tc<0, 0, -1, NG>))
  // the contact-point model runs two groups: its chunks hold 128 interval records each
  if (a.m.contact && ng != 2) return cudaErrorNotSupported;
  decltype(&tc::k_mlp_bwd_tc<0, 6, 4, 3>) kern =
      a.m.contact ? tc::k_mlp_bwd_tc<0, 6, 6, 2, true>
                  : (ng == 3 ? MLPS_BWD_KERN(3) : ng == 2 ? MLPS_BWD_KERN(2) : MLPS_BWD_KERN(1));
#undef MLPS_BWD_KERN
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_sm, tc::kGThreads * ng, smem, st>>>(w, a, P, tmap);
  return cudaGetLastError();
}

}  // namespace mlps
