// k_mlp_tc.cu -- grouped per-primitive MLP on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory (TMEM).
//
// Same work decomposition as the FP32 path: a chunk is up to ipc = 128 / S hit intervals of one
// primitive, i.e. one M = 128 tile of sample rows; persistent blocks walk a contiguous range
// of the primitive-major chunk list. Inside a block:
//  * warp 0 allocates tensor memory; thread 0 loads the primitive's weight tiles with TMA
//    tensor copies (cp.async.bulk.tensor, 128-byte swizzle) into shared memory whenever the
//    primitive changes;
//  * epilogue warpgroups (four for width 64, three with a feature head, two for width 128;
//    every warp of the block belongs to one) each own one chunk at a time,
//    its A-operand tile in shared memory and 128 TMEM columns. A group builds the sample
//    encodings (Eq. 5) as BF16 rows of the first A tile; its first thread issues the layer's
//    tcgen05.mma and commits them to the group's mbarrier; once they complete, the group reads
//    its accumulator rows from TMEM (thread = sample row), adds the bias, applies ReLU,
//    converts to BF16 and writes the next layer's A tile in place. Groups run independently,
//    so the tensor core works on one group's layer while the others run epilogues.
//  * the last layer's epilogue applies sigmoid / softplus and composites each interval's S
//    samples front to back (Eq. 6) with warp-level segmented scans, writing the interval's
//    (C_j, a_j) exactly like the FP32 path.
// Every wait is bounded by wall time; on a timeout the block raises an abort flag, finishes its
// loops without work, waits (bounded) for its MMAs in flight, frees TMEM and reports
// MLPS_ERR_TIMEOUT through the status word.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstring>

#include "mlps_common.cuh"
#include "mlps_kernels.h"
#include "simt_common.cuh"
#include "tc_ptx.cuh"
#include "tc_common.cuh"

namespace mlps {
namespace tc {

using simt::IntervalInfo;

constexpr int threads_tc(int neg) { return kEGThreads * neg; }
constexpr uint32_t kTmemCols = 512;             // WIDTH columns per group
constexpr uint64_t kWaitNs = 2000000000ull;     // 2 s
// Byte offsets in dynamic shared memory; per-group regions are base + g * stride (plain
// arithmetic, so that nothing is indexed at run time).
struct TcSmem {
  uint32_t w, ones, a0, a_stride, bias, itab0, itab_stride, scan, bars, misc, total;
};

MLPS_HD uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

MLPS_HD TcSmem tc_smem(const TcPlan& P, int kNEG, bool e4m3, int ipc) {
  TcSmem L;
  uint32_t off = 0;
  L.w = off;
  off = align_up(off + (e4m3 ? P.w8_bytes : P.w_bytes + P.bt_bytes), 1024);
  L.ones = off;  // folded bias: A tile whose every row is (1, 0, ..., 0)
  off += (!e4m3 && P.fold > 0) ? (uint32_t)kM * 128 : 0u;
  L.a0 = off;
  L.a_stride = align_up(P.a_bytes, 1024);
  off += L.a_stride * kNEG;
  L.bias = off;  // biases, then (E4M3) the per-output weight scales
  off = align_up(off + 4 * P.bias_floats * (e4m3 ? 3 : 1) + (e4m3 ? 16 : 0), 16);
  L.itab0 = off;
  // two buffers of ipc interval records: the current chunk's and the next chunk's (in flight)
  L.itab_stride = align_up(2 * (uint32_t)sizeof(IntervalRec) * ipc, 16);
  off += L.itab_stride * kNEG;
  L.scan = off;
  off = align_up(off + 4 * kNEG * 4 * kMaxScanVals, 16);
  L.bars = off;
  off = align_up(off + 8 * (2 + 2 * kNEG), 16);
  L.misc = off;
  off = align_up(off + 16, 16);
  L.total = off;
  return L;
}

// F8: E4M3 operands (kind::f8f6f4). Layer l's A operand holds its input divided by a static
// power-of-two scale s_l per (primitive, layer), the weights are stored divided by a power of two
// c_l chosen so that s_{l+1} = s_l c_l, and the bias is one more K step: a hidden layer's
// accumulator is the next A operand before ReLU and conversion (k_pack_e4m3).
template <int WIDTH, int XL, int DL, int NF, int kNEG, bool F8, int NL = 0>
__global__ void __launch_bounds__(kEGThreads * kNEG, 1)
    k_mlp_fwd_tc(Work w, MlpArgs a, TcPlan P, const __grid_constant__ CUtensorMap tmap) {
  constexpr int kThreadsTC = kEGThreads * kNEG;
  // Each group's TMEM holds its FP32 accumulator (WIDTH columns) and the next layer's A operand:
  // WIDTH / 2 columns of BF16 pairs, or WIDTH / 4 columns of E4M3 quadruples.
  constexpr bool kTA = true;
  constexpr uint32_t kGCols = (uint32_t)(WIDTH + (F8 ? WIDTH / 4 : WIDTH / 2));
  // the encoded input goes to TMEM too when it is built in registers (compile-time shapes)
  constexpr bool kA0T = kTA && XL >= 0;
  // BF16 at width 64: every hidden layer's bias is added by one more MMA step (the plan folds
  // all of them); width 128 adds them in the epilogue
  constexpr bool kFold = WIDTH == 64 && !F8;
  static_assert(kNEG >= 1 && kNEG <= 6 && kNEG * kGCols + (F8 ? 8 : 0) <= 512, "TMEM holds 512 columns");
  static_assert(4 + NF <= kMaxScanVals, "scan scratch holds kMaxScanVals values per warp");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (sbase - raw);
  const TcSmem L = tc_smem(P, kNEG, F8, w.ipc);
  const Model& m = a.m;
  float* sBias = reinterpret_cast<float*>(gbase + L.bias);
  float* sScan = reinterpret_cast<float*>(gbase + L.scan);
  const uint32_t bar_w = sbase + L.bars;
#define bar_end(G) (bar_w + 16u + 8u * (uint32_t)(G))
#define bar_done(G) (bar_w + 16u + 8u * (uint32_t)(kNEG) + 8u * (uint32_t)(G))
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(gbase + L.misc);
  volatile int* sAbort = reinterpret_cast<volatile int*>(gbase + L.misc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(bar_w, 1);
    for (int g = 0; g < kNEG; ++g) {
      mbar_init(bar_done(g), 1);
      mbar_init(bar_end(g), 1);
    }
    *sAbort = 0;
    fence_mbar_init();
  }
  if (!F8 && P.fold > 0) {  // ones tile of the folded bias: element 0 of every row is 1.0
    for (int i = threadIdx.x; i < kM * 8; i += kThreadsTC) {
      const int r = i >> 3, ch = i & 7;
      st_shared_v4(sbase + L.ones + (uint32_t)i * 16, ((ch ^ (r & 7)) == 0) ? 0x3F80u : 0u, 0u, 0u, 0u);
    }
    fence_proxy_async_smem();
  }
  if (warp == 0) {
    tmem_alloc(sbase + L.misc, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  // E4M3: a constant-1 A operand after the groups' columns (8 columns = one K = 32 step; the
  // first two elements of every row are 1.0, 0x38), shared by every group's bias step
  const uint32_t ones_t = tmem + (uint32_t)kNEG * kGCols;
  if (F8) {
    if (warp < 4) {
      const uint32_t o8[8] = {0x00003838u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
      tmem_st8(ones_t + ((uint32_t)(warp * 32) << 16), o8);
      tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }

  const int total = walk_chunk_count(w);  // (a depth wave's lists, or every chunk)
  const int* const bmap = walk_map(w);    // list position -> primitive-major position
  const int cb = (int)((long long)total * blockIdx.x / gridDim.x);
  const int ce = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  const int S = m.S;
  const int nl = NL > 0 ? NL : m.nl;  // (NL > 0: the layer count fixed at compile time)
  const int g = warp >> 2;               // epilogue group of this warp (< kNEG)
  const int q = warp & 3;                // TMEM lane quarter
  const int row = q * 32 + lane;         // sample row within the chunk
  // mbarrier phase parities, one bit per group (registers, no local memory)
  uint32_t ph_w = 0, ph_done = 0;
  int loaded = -1;
  int prim = cb < ce ? simt::find_prim(w, cb) : 0;

  // the next chunk's interval records, copied one step ahead (cp.async) into the group's
  // pending table buffer `pb`
  const uint32_t itab_s = sbase + L.itab0 + (uint32_t)g * L.itab_stride;
  int pb = 0;
  auto prefetch = [&](const ChunkStep<kNEG>& st, int c) {
    const int f = (c - w.chunk_start[st.prim]) * w.ipc;
    if (row < min(w.ipc, w.prim_count[st.prim] - f))
      rec_copy_async(w, walk_slot(bmap, w.prim_start[st.prim] + f + row),
                     itab_s + (uint32_t)((pb * w.ipc + row) * sizeof(IntervalRec)), 0u);
  };
  ChunkStep<kNEG> cur = chunk_step<kNEG>(w, cb, ce, prim);
  const int my_first = step_chunk(cur, g);
  if (cur.n > 0 && my_first >= 0) prefetch(cur, my_first);
  while (cur.c0 < ce) {
    prim = cur.prim;
    const ChunkStep<kNEG> nxt = chunk_step<kNEG>(w, cur.c0 + cur.n, ce, prim);
    const int my_cc = step_chunk(cur, g);  // this warp's chunk this step and the next
    const int my_nx = step_chunk(nxt, g);
    if (prim != loaded) {
      __syncthreads();  // every role is done with the previous primitive's tiles
      if (threadIdx.x == 0 && !*sAbort) {
        mbar_arrive_expect_tx(bar_w, (uint32_t)(F8 ? P.w8_bytes : P.w_bytes + P.bt_bytes));
        const int row0 = prim * P.rows_per_prim;
        for (int l = 0; l < nl; ++l) {
          if (F8) {
            for (int j = 0; j < P.npad[l] / 16; ++j)
              tma_load_2d(sbase + L.w + P.s8_off[l] + j * 2048, &tmap, 0, row0 + P.g8_row[l] + j * 16, bar_w);
            if (l == 0)  // the bias tile of the hidden layers
              for (int r = 0; r < ((nl - 1 + 3) / 4) * WIDTH; r += 16)
                tma_load_2d(sbase + L.w + P.s8b_off + r * 128, &tmap, 0, row0 + P.g8b_row + r, bar_w);
          } else {
            for (int sl = 0; sl < P.kpad[l] / 64; ++sl)
              for (int j = 0; j < P.npad[l] / 16; ++j)
                tma_load_2d(sbase + L.w + P.sw_off[l] + sl * P.npad[l] * 128 + j * 2048, &tmap, 0,
                            row0 + P.gw_row[l] + sl * P.npad[l] + j * 16, bar_w);
          }
        }
        if (!F8 && P.fold > 0)
          for (int sl = 0; sl < (P.fold + 3) / 4; ++sl)
            for (int j = 0; j < 4; ++j)
              tma_load_2d(sbase + L.w + P.sbt_off + sl * 8192 + j * 2048, &tmap, 0, row0 + P.gbt_row + sl * 64 + j * 16,
                          bar_w);
      }
      const unsigned char* blob = a.weights + (size_t)prim * a.pk.stride;
      const float* gb = reinterpret_cast<const float*>(blob + P.gbias_byte);
      for (int i = threadIdx.x; i < P.bias_floats; i += kThreadsTC) sBias[i] = gb[i];
      if (F8) {  // the last layer's multipliers and offsets, then the input multiplier
        const float* gm = reinterpret_cast<const float*>(blob + P.gmul_byte);
        for (int i = threadIdx.x; i <= 2 * P.bias_floats; i += kThreadsTC) sBias[P.bias_floats + i] = gm[i];
      }
      mbar_wait(bar_w, ph_w, sAbort, kWaitNs);
      ph_w ^= 1;
      __syncthreads();
      loaded = prim;
    }

    {
      // ------------------------------------------------------------ epilogue group g
      if (my_cc < 0 && nxt.n > 0 && my_nx >= 0) prefetch(nxt, my_nx);  // idle this step: still prefetch
      if (my_cc >= 0) {
        const int bar_id = 1 + g;
        const int first = (my_cc - w.chunk_start[prim]) * w.ipc;
        const int nint = min(w.ipc, w.prim_count[prim] - first);
        cp_async_wait_all();                  // this thread's copies of the chunk's records landed
        named_bar_sync(bar_id, kEGThreads);   // everyone's did; the other buffer is no longer read
        const IntervalRec* T = reinterpret_cast<const IntervalRec*>(
            gbase + L.itab0 + (uint32_t)g * L.itab_stride + pb * w.ipc * sizeof(IntervalRec));
        pb ^= 1;
        if (nxt.n > 0 && my_nx >= 0) prefetch(nxt, my_nx);  // start loading the next chunk now
        const uint32_t A = sbase + L.a0 + (uint32_t)g * L.a_stride;
        const int iv = row / S, k = row - iv * S;
        const bool valid = iv < nint;
        if (F8 && XL >= 0) {
          uint32_t pk[16];
          if (valid) {
            const IntervalRec& I = T[iv];
            const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
            float xl[3], dd[3];
            for (int u = 0; u < 3; ++u) { xl[u] = fmaf(tr, I.dp[u], I.p[u]); dd[u] = I.d[u]; }
            encode_e4m3_64<(XL > 0 ? XL : 0), (DL > 0 ? DL : 0)>(xl, dd, sBias[3 * P.bias_floats], pk);
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) pk[e] = 0u;
          }
          tmem_st16(tmem + (uint32_t)g * kGCols + WIDTH + ((uint32_t)(q * 32) << 16), pk);
          tmem_wait_st();
        } else if (F8) {
          RowWriter8 rw{A, row, 0, 0.f, sBias[3 * P.bias_floats]};
          if (valid && m.contact) {  // the tensor-core blob's order: gamma(delta), then gamma(d)
            const IntervalRec& I = T[iv];
            float del[3];
            contact_delta(w.geo[prim], I, del);
            if (m.xyzL == 0) {
              for (int u = 0; u < 3; ++u) rw.put(del[u]);
            } else {
              for (int u = 0; u < 3; ++u) put_gamma8(rw, del[u], m.xyzL);
            }
            if (m.dirL > 0)
              for (int u = 0; u < 3; ++u) put_gamma8(rw, I.d[u], m.dirL);
          } else if (valid) {
            const IntervalRec& I = T[iv];
            const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
            float xl[3];
            for (int u = 0; u < 3; ++u) xl[u] = fmaf(tr, I.dp[u], I.p[u]);
            if (m.xyzL == 0) {
              for (int u = 0; u < 3; ++u) rw.put(xl[u]);
            } else {
              for (int u = 0; u < 3; ++u) put_gamma8(rw, xl[u], m.xyzL);
            }
            if (m.dirL > 0)
              for (int u = 0; u < 3; ++u) put_gamma8(rw, I.d[u], m.dirL);
          }
          rw.pad_to(P.kpad[0]);
        } else if (XL >= 0) {
          // compile-time encoding (the configurations' shapes)
          uint32_t pk[32];
          if (valid) {
            const IntervalRec& I = T[iv];
            const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
            float xl[3], dd[3];
            for (int u = 0; u < 3; ++u) { xl[u] = fmaf(tr, I.dp[u], I.p[u]); dd[u] = I.d[u]; }
            encode_pairs64<(XL > 0 ? XL : 0), (DL > 0 ? DL : 0)>(xl, dd, pk);
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) pk[e] = 0u;
          }
          if (kA0T) {
            tmem_st32(tmem + (uint32_t)g * kGCols + WIDTH + ((uint32_t)(q * 32) << 16), pk);
            tmem_wait_st();
          } else {
#pragma unroll
            for (int ch = 0; ch < 8; ++ch)
              st_shared_v4(A + sw128_off(row, ch), pk[4 * ch], pk[4 * ch + 1], pk[4 * ch + 2], pk[4 * ch + 3]);
          }
        } else {
          RowWriter rw{A, row, 0, 0.f};
          if (valid && m.contact) {
            // contact-point input gamma([d; delta]) (Eq. 4), one sample per hit, in the tensor-core
            // blob's column order: gamma(delta) first (tc_in_col)
            const IntervalRec& I = T[iv];
            float del[3];
            contact_delta(w.geo[prim], I, del);
            if (m.xyzL == 0) {
              for (int u = 0; u < 3; ++u) rw.put(del[u]);
            } else {
              for (int u = 0; u < 3; ++u) put_gamma(rw, del[u], m.xyzL);
            }
            if (m.dirL > 0)
              for (int u = 0; u < 3; ++u) put_gamma(rw, I.d[u], m.dirL);
          } else if (valid) {
            const IntervalRec& I = T[iv];
            const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
            float xl[3];
            for (int u = 0; u < 3; ++u) xl[u] = fmaf(tr, I.dp[u], I.p[u]);
            if (m.xyzL == 0) {
              for (int u = 0; u < 3; ++u) rw.put(xl[u]);
            } else {
              for (int u = 0; u < 3; ++u) put_gamma(rw, xl[u], m.xyzL);
            }
            if (m.dirL > 0)
              for (int u = 0; u < 3; ++u) put_gamma(rw, I.d[u], m.dirL);
          }
          rw.pad_to(P.kpad[0]);
        }
        if (!kA0T) fence_proxy_async_smem();
        tc_fence_before();
        named_bar_sync(bar_id, kEGThreads);  // the whole A operand is written
        const uint32_t dacc = tmem + (uint32_t)g * kGCols;
        const uint32_t aT = dacc + WIDTH;  // A operand in TMEM (BF16)
        if (row == 0) {  // this group issues its own MMAs
          tc_fence_after();
          if (!*sAbort) {
            const uint32_t bt8 = nl > 1 ? sbase + L.w + P.s8b_off : 0u;  // E4M3 bias step of layer 0
            if (F8 && kA0T) issue_fwd_layer_e4m3_ta(aT, sbase + L.w + P.s8_off[0], dacc, P.kpad[0], P.npad[0], ones_t, bt8);
            else if (F8) issue_fwd_layer_e4m3(A, sbase + L.w + P.s8_off[0], dacc, P.kpad[0], P.npad[0], ones_t, bt8);
            else if (kA0T)
              issue_fwd_layer_ta(aT, sbase + L.w + P.sw_off[0], dacc, P.kpad[0], P.npad[0], sbase + L.ones,
                                 P.fold > 0 ? sbase + L.w + P.sbt_off : 0u);
            else issue_fwd_layer(A, sbase + L.w + P.sw_off[0], dacc, P.kpad[0], P.npad[0], sbase + L.ones,
                                 P.fold > 0 ? sbase + L.w + P.sbt_off : 0u);
          }
          mma_commit(bar_done(g));
        }
        const uint32_t trow = dacc + ((uint32_t)(q * 32) << 16);
        const uint32_t arow = aT + ((uint32_t)(q * 32) << 16);
#pragma unroll
        for (int l = 0; l < (NL > 0 ? NL : nl); ++l) {
          // warp-uniform: tcgen05.ld below is a .sync.aligned warp instruction
          const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_done(g), (ph_done >> g) & 1u, sAbort, kWaitNs));
          ph_done ^= 1u << g;
          tc_fence_after();
          const float* bias = sBias + P.bias_off[l];
          if (l < nl - 1) {
            if (ok && F8) {
              // E4M3: the accumulator already holds z / s_{l+1} (bias included, scales folded in
              // by the packing): ReLU and conversion (saturating) only, 32 columns at a time
#pragma unroll
              for (int h32 = 0; h32 < WIDTH / 32; ++h32) {
                uint32_t v[32];
                tmem_ld32(trow + h32 * 32, v);
                tmem_wait_ld();
                uint32_t pk[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                  pk[e] = pack_e4m3_relu(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1])) |
                          (pack_e4m3_relu(__uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3])) << 16);
                tmem_st8(arow + (uint32_t)(h32 * 8), pk);
              }
              tmem_wait_st();
            } else if (ok && kFold) {
              // bias added by the MMA: ReLU and BF16 pairs into the A operand in TMEM, 32 columns
              // at a time (fewer live registers, so more groups fit on the SM)
#pragma unroll
              for (int h32 = 0; h32 < WIDTH / 32; ++h32) {
                uint32_t v[32];
                tmem_ld32(trow + h32 * 32, v);
                tmem_wait_ld();
                uint32_t pk[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) pk[e] = pack_bf16_relu(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]));
                tmem_st16(arow + (uint32_t)(h32 * 16), pk);
              }
              tmem_wait_st();
            } else if (ok && !kFold && !F8) {
#pragma unroll
              for (int h32 = 0; h32 < WIDTH / 32; ++h32) {
                uint32_t v[32];
                tmem_ld32(trow + h32 * 32, v);
                tmem_wait_ld();
                const float4* b4 = reinterpret_cast<const float4*>(bias + h32 * 32);
                uint32_t pk[16];
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                  const float4 bq = b4[c4];
                  float x0 = __uint_as_float(v[4 * c4]), x1 = __uint_as_float(v[4 * c4 + 1]);
                  float x2 = __uint_as_float(v[4 * c4 + 2]), x3 = __uint_as_float(v[4 * c4 + 3]);
                  add2_f32(x0, x1, bq.x, bq.y);
                  add2_f32(x2, x3, bq.z, bq.w);
                  pk[2 * c4] = pack_bf16_relu(x0, x1);
                  pk[2 * c4 + 1] = pack_bf16_relu(x2, x3);
                }
                tmem_st16(arow + (uint32_t)(h32 * 16), pk);
              }
              tmem_wait_st();
            }
            tc_fence_before();
            named_bar_sync(bar_id, kEGThreads);
            if (row == 0) {
              tc_fence_after();
              if (!*sAbort) {
                if (F8)
                  issue_fwd_layer_e4m3_ta(aT, sbase + L.w + P.s8_off[l + 1], dacc, P.kpad[l + 1], P.npad[l + 1], ones_t,
                                          l + 2 < nl ? sbase + L.w + P.s8b_off + (uint32_t)(((l + 1) >> 2) * WIDTH * 128) +
                                                           32u * ((l + 1) & 3)
                                                     : 0u);
                else issue_fwd_layer_ta(aT, sbase + L.w + P.sw_off[l + 1], dacc, P.kpad[l + 1], P.npad[l + 1],
                                        sbase + L.ones,
                                        l + 1 < P.fold ? sbase + L.w + P.sbt_off + 8192u * ((l + 1) >> 2) + 32u * ((l + 1) & 3)
                                                       : 0u);
              }
              mma_commit(bar_done(g));
            }
          } else {
            // last layer: heads, then the interval composite (NF = largest feature count)
            constexpr int NZ = 4 + NF;
            float z[NZ];
            if (ok) {
              uint32_t r32[32], r16[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) r16[j] = 0u;
              if (P.npad[l] >= 32) {
                tmem_ld32(trow, r32);
                if (P.npad[l] == 48) tmem_ld16(trow + 32, r16);
              } else {
                tmem_ld16(trow, r16);
              }
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < NZ; ++j) {
                uint32_t bits;
                if (P.npad[l] >= 32) bits = j < 32 ? r32[j] : r16[(j - 32) & 15];
                else bits = j < 16 ? r16[j] : 0u;
                if (F8)
                  z[j] = (j < m.nout) ? fmaf(__uint_as_float(bits), sBias[P.bias_floats + P.bias_off[l] + j],
                                             sBias[2 * P.bias_floats + P.bias_off[l] + j])
                                      : 0.f;
                else z[j] = (j < m.nout) ? __uint_as_float(bits) + bias[j] : 0.f;
              }
            } else {
#pragma unroll
              for (int j = 0; j < NZ; ++j) z[j] = 0.f;
            }
            tc_fence_before();
            const float dt = valid ? T[iv].dt : 0.f;
            const float sig = softplus_fast(z[3]);
            float A1[1] = {valid ? sig * dt : 0.f};
            const float a_k = A1[0];
            seg_scan<1>(A1, 1, row, S, sScan + g * 4 * kMaxScanVals, bar_id);
            const float Aex = A1[0] - a_k;
            const float wk = valid ? __expf(-Aex) * (1.f - __expf(-a_k)) : 0.f;
            float vals[NZ];
            vals[0] = wk * sigmoid_fast(z[0]);
            vals[1] = wk * sigmoid_fast(z[1]);
            vals[2] = wk * sigmoid_fast(z[2]);
            vals[3] = a_k;
#pragma unroll
            for (int f = 0; f < NF; ++f) vals[4 + f] = f < m.F ? wk * z[4 + f] : 0.f;
            seg_sum<NZ>(vals, 4 + m.F, row, S, sScan + g * 4 * kMaxScanVals, bar_id);  // interval totals
            if (valid && k == S - 1 && ok) {
              const int h = T[iv].h;
              w.hit_out[h] = make_float4(vals[0], vals[1], vals[2], vals[3]);
#pragma unroll
              for (int f = 0; f < NF; ++f)
                if (f < m.F) w.hit_feat[(size_t)h * m.F + f] = vals[4 + f];
            }
          }
        }
      }
    }
    cur = nxt;
  }

  // teardown: no copy may still be in flight, and none of this group's MMAs may still write
  // TMEM (after an abort a group may have stopped waiting for them); then TMEM is freed
  cp_async_wait_all();
  if ((threadIdx.x & (kEGThreads - 1)) == 0) {
    mma_commit(bar_end(g));
    mbar_wait_limit(bar_end(g), 0, kWaitNs);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
  if (threadIdx.x == 0 && *sAbort) set_status(w.saved_hdr, MLPS_ERR_TIMEOUT);
#undef bar_done
#undef bar_end
}

// ------------------------------------------------------------------------------------------
// Packing of canonical FP32 weights into the BF16 tensor-core blob

__global__ void k_pack_bf16(Model m, TcPlan P, long long stride, int K, const float* __restrict__ src,
                            unsigned char* __restrict__ dst) {
  const int p = blockIdx.y;
  if (p >= K) return;
  const float* s = src + (size_t)p * m.Prow;
  unsigned char* d = dst + (size_t)p * stride;
  if (m.C > 0) {  // slot embeddings, unchanged
    float* e = reinterpret_cast<float*>(d + P.slot_byte);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * m.C; i += gridDim.x * blockDim.x) e[i] = s[m.P + i];
  }
  // weight tiles: element (n, k) of layer l at row gw_row + (k / 64) * npad + n, column k % 64
  for (int l = 0; l < m.nl; ++l) {
    const int np = P.npad[l], kp = P.kpad[l];
    __nv_bfloat16* t = reinterpret_cast<__nv_bfloat16*>(d + (size_t)P.gw_row[l] * 128);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np * kp; i += gridDim.x * blockDim.x) {
      const int n = i / kp, k = i - n * kp;
      const float v = (n < m.dout[l] && k < m.din[l]) ? s[m.woff[l] + n * m.din[l] + tc_in_col(m, l, k)] : 0.f;
      t[((k >> 6) * np + n) * 64 + (k & 63)] = __float2bfloat16_rn(v);
    }
  }
  float* b = reinterpret_cast<float*>(d + P.gbias_byte);
  for (int l = 0; l < m.nl; ++l)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.npad[l]; i += gridDim.x * blockDim.x)
      b[P.bias_off[l] + i] = i < m.dout[l] ? s[m.boff[l] + i] : 0.f;
  if (P.fold > 0) {  // bias tile: 64-column slabs; slab l / 4, row n, column 16 (l % 4) = bias n of layer l
    __nv_bfloat16* bt = reinterpret_cast<__nv_bfloat16*>(d + (size_t)P.gbt_row * 128);
    const int nsl = (P.fold + 3) / 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsl * 64 * 64; i += gridDim.x * blockDim.x) {
      const int sl = i >> 12, n = (i >> 6) & 63, k = i & 63, l = 4 * sl + (k >> 4);
      const float v = ((k & 15) == 0 && l < P.fold && n < m.dout[l]) ? s[m.boff[l] + n] : 0.f;
      bt[i] = __float2bfloat16_rn(v);
    }
  }
}

// E4M3 copy of the weights, bias tile and scales (FP8 precision), one block of 128 threads per
// primitive. Layer l's A operand holds its input divided by a power of two s_l; the stored weights
// are W_l / c_l with c_l a power of two, so the FP32 accumulator of layer l (the bias added by one
// more K step) holds z / (s_l c_l). The packing sets s_{l+1} = s_l c_l: the accumulator of a
// hidden layer is then the next layer's A operand as it stands, and the epilogue only applies
// ReLU and converts (no multiply, no bias). c_l is the smallest power of two with
//  * 4 a_{l+1} / (s_l c_l) <= 448, a_{l+1} the largest input of layer l + 1 met when the block
//    evaluates the primitive's FP32 MLP on 256 probe inputs (local positions uniform in
//    [-1, 1]^3, directions on the unit sphere, from a fixed integer hash): 4x headroom below the
//    largest finite E4M3 value, beyond which values saturate;
//  * max |W_l| / c_l <= 448 (every weight representable), and max |b_l| / s_{l+1} <= 224 (the
//    bias as hi + lo E4M3 bytes, hi = e4m3(v), lo = e4m3(v - hi)).
// s_0 = 1/32: the encoded inputs lie in [-1, 1]. The last layer keeps an FP32 epilogue:
// z = acc * (s_L c_L) + b, c_L = the smallest power of two with max |W_L| / c_L <= 448. Scaling by
// powers of two is exact, so the scales add no rounding of their own.
MLPS_DEV uint32_t probe_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return x;
}

MLPS_DEV float probe_unit(uint32_t& st) {  // uniform in [-1, 1)
  st = probe_hash(st + 0x9E3779B9u);
  return (float)(st >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

MLPS_DEV int probe_gamma(int L, const float v[3], float* x, int f) {
  if (L == 0) {
    for (int c = 0; c < 3; ++c) x[f++] = v[c];
    return f;
  }
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < L; ++l) {
      float sn, cs;
      sincospif(ldexpf(v[c], l), &sn, &cs);
      x[f++] = sn;
      x[f++] = cs;
    }
  return f;
}

MLPS_DEV float pow2_at_least(float q) {  // smallest power of two >= q (1 for q <= 0 or not finite)
  if (!(q > 1e-30f) || !(q < 1e30f)) return 1.0f;
  return __uint_as_float((__float_as_uint(q) + 0x007FFFFFu) & 0x7F800000u);
}

__global__ void __launch_bounds__(128) k_pack_e4m3(Model m, TcPlan P, long long stride, int K,
                                                   const float* __restrict__ src, unsigned char* __restrict__ dst) {
  const int p = blockIdx.x;
  if (p >= K) return;
  const float* s = src + (size_t)p * m.Prow;
  unsigned char* d = dst + (size_t)p * stride;
  __shared__ unsigned int amax[kMaxLayers + 1], wmax[kMaxLayers], bmax[kMaxLayers];
  __shared__ float sl[kMaxLayers + 1], cl[kMaxLayers];
  const int t = threadIdx.x;
  if (t <= kMaxLayers) amax[t] = 0u;
  if (t < kMaxLayers) wmax[t] = bmax[t] = 0u;
  __syncthreads();
  // largest |W_l| and |b_l| (non-negative floats order as their bits)
  for (int l = 0; l < m.nl; ++l) {
    const int din = m.din[l];
    for (int n = t; n < m.dout[l]; n += blockDim.x) {
      float am = 0.f;
      for (int k = 0; k < din; ++k) am = fmaxf(am, fabsf(s[m.woff[l] + n * din + k]));
      atomicMax(&wmax[l], __float_as_uint(am));
      atomicMax(&bmax[l], __float_as_uint(fabsf(s[m.boff[l] + n])));
    }
  }
  // calibration: the largest input of every hidden layer's successor on the probes
  float hin[128], hout[128];
  for (int probe = 0; probe < 2; ++probe) {
    uint32_t st = probe_hash(((uint32_t)p * 256u + (uint32_t)(2 * t + probe)) * 2654435761u + 12345u);
    float xl[3], dv[3];
    for (int c = 0; c < 3; ++c) xl[c] = probe_unit(st);
    float nn = 0.f;
    do {  // direction: rejection-sampled in the unit ball, then normalised
      nn = 0.f;
      for (int c = 0; c < 3; ++c) {
        dv[c] = probe_unit(st);
        nn += dv[c] * dv[c];
      }
    } while (!(nn > 1e-4f && nn <= 1.f));
    const float inv = rsqrtf(nn);
    for (int c = 0; c < 3; ++c) dv[c] *= inv;
    int f = 0;
    if (m.contact) {
      if (m.dirL > 0) f = probe_gamma(m.dirL, dv, hin, f);
      f = probe_gamma(m.xyzL, xl, hin, f);
    } else {
      f = probe_gamma(m.xyzL, xl, hin, f);
      if (m.dirL > 0) f = probe_gamma(m.dirL, dv, hin, f);
    }
    for (int l = 0; l + 1 < m.nl; ++l) {
      const int din = m.din[l], dout = m.dout[l];
      float mx = 0.f;
      for (int n = 0; n < dout; ++n) {
        float z = s[m.boff[l] + n];
        for (int k = 0; k < din; ++k) z = fmaf(s[m.woff[l] + n * din + k], hin[k], z);
        z = fmaxf(z, 0.f);
        hout[n] = z;
        mx = fmaxf(mx, z);
      }
      atomicMax(&amax[l + 1], __float_as_uint(mx));
      for (int n = 0; n < dout; ++n) hin[n] = hout[n];
    }
  }
  __syncthreads();
  if (t == 0) {  // the scale chain (sequential: s_{l+1} = s_l c_l)
    sl[0] = 1.0f / 32.0f;
    for (int l = 0; l < m.nl; ++l) {
      const float wm = __uint_as_float(wmax[l]);
      float c = pow2_at_least(wm / 448.0f);
      if (l + 1 < m.nl) {
        c = fmaxf(c, pow2_at_least(4.0f * __uint_as_float(amax[l + 1]) / (448.0f * sl[l])));
        const float bm = __uint_as_float(bmax[l]);
        for (int it = 0; it < 64 && bm / (sl[l] * c) > 224.0f; ++it) c *= 2.0f;
      }
      cl[l] = c;
      sl[l + 1] = sl[l] * c;
    }
  }
  __syncthreads();
  for (int l = 0; l < m.nl; ++l) {
    const int din = m.din[l];
    const float ic = 1.0f / cl[l];
    for (int n = t; n < P.npad[l]; n += blockDim.x) {
      const bool live = n < m.dout[l];
      unsigned char* r = d + (size_t)(P.g8_row[l] + n) * 128;
      for (int k = 0; k < 128; ++k)
        r[k] = (live && k < din)
                   ? __nv_cvt_float_to_fp8(s[m.woff[l] + n * din + tc_in_col(m, l, k)] * ic, __NV_SATFINITE, __NV_E4M3)
                   : 0;
    }
  }
  // bias tile of the hidden layers: rows n < the (padded) hidden width, slab l / 4, bytes
  // 32 (l % 4) and 32 (l % 4) + 1; rows of padded units stay zero
  const int nsl8 = (m.nl - 1 + 3) / 4, wrows = P.npad[0];
  for (int i = t; i < nsl8 * wrows; i += blockDim.x) {
    const int sl_ = i / wrows, n = i - sl_ * wrows;
    unsigned char* r = d + (size_t)(P.g8b_row + i) * 128;
    for (int k = 0; k < 128; ++k) r[k] = 0;
    for (int j = 0; j < 4; ++j) {
      const int l = 4 * sl_ + j;
      if (l + 1 >= m.nl || n >= m.dout[l]) continue;
      const float v = s[m.boff[l] + n] / sl[l + 1];
      const __nv_fp8_storage_t hi = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
      const float hv = __half2float(__half(__nv_cvt_fp8_to_halfraw(hi, __NV_E4M3)));
      r[32 * j] = hi;
      r[32 * j + 1] = __nv_cvt_float_to_fp8(v - hv, __NV_SATFINITE, __NV_E4M3);
    }
  }
  // last layer's FP32 epilogue, and the input multiplier
  float* mul = reinterpret_cast<float*>(d + P.gmul_byte);
  float* add = reinterpret_cast<float*>(d + P.gadd_byte);
  const int L = m.nl - 1;
  for (int n = t; n < P.bias_floats; n += blockDim.x) {
    mul[n] = 0.f;
    add[n] = 0.f;
  }
  __syncthreads();
  for (int n = t; n < m.dout[L]; n += blockDim.x) {
    mul[P.bias_off[L] + n] = sl[L] * cl[L];
    add[P.bias_off[L] + n] = s[m.boff[L] + n];
  }
  if (t == 0) *reinterpret_cast<float*>(d + P.gin_byte) = 1.0f / sl[0];
}

}  // namespace tc

// ------------------------------------------------------------------------------------------
// Host side

static int round_up_i(int x, int a) { return (x + a - 1) / a * a; }

bool tc_plan(const Model& m, TcPlan* P, long long* stride, bool e4m3) {
  std::memset(P, 0, sizeof(*P));
  if (m.width != 64 && m.width != 128) return false;
  if (m.nin > 128 || m.nout > 48 || m.S > 128) return false;
  P->nl = m.nl;
  int rows = 0, sw = 0, bias = 0, kmax = 0;
  for (int l = 0; l < m.nl; ++l) {
    P->kpad[l] = l == 0 ? round_up_i(m.nin, 64) : m.width;
    P->npad[l] = l == m.nl - 1 ? round_up_i(m.nout, 16) : m.width;
    P->gw_row[l] = rows;
    rows += (P->kpad[l] / 64) * P->npad[l];
    P->sw_off[l] = sw;
    sw += P->kpad[l] * P->npad[l] * 2;
    P->bias_off[l] = bias;
    bias += P->npad[l];
    kmax = kmax > P->kpad[l] ? kmax : P->kpad[l];
  }
  P->w_bytes = sw;
  // (the backward pass reads the same W tiles as MN-major operands: no transposed copies)
  if (m.width == 64 && m.nl - 1 >= 1) {  // every hidden-layer bias folded (BF16 forward at width 64)
    P->fold = m.nl - 1;  // <= kMaxLayers - 1 = 7: at most two 64-column slabs of bias columns
    const int nsl = (P->fold + 3) / 4;
    P->gbt_row = rows;
    rows += 64 * nsl;
    P->sbt_off = sw;
    P->bt_bytes = 64 * 128 * nsl;
  }
  P->bias_floats = bias;
  P->gbias_byte = rows * 128;
  long long bytes = (long long)rows * 128 + 4LL * bias;
  if (e4m3) {
    // E4M3 copy after the biases: one 128-byte row per output, then the FP32 multipliers and
    // offsets of the epilogue.
    // The BF16 tiles stay in the blob: the backward pass of the FP8 precision uses them.
    if (kmax > 128) return false;
    int r8 = (int)((bytes + 127) / 128), s8 = 0;
    for (int l = 0; l < m.nl; ++l) {
      P->g8_row[l] = r8;
      r8 += P->npad[l];
      P->s8_off[l] = s8;
      s8 += P->npad[l] * 128;
    }
    const int nsl8 = (m.nl - 1 + 3) / 4;  // bias slabs of the hidden layers
    P->g8b_row = r8;
    r8 += m.width * nsl8;
    P->s8b_off = s8;
    s8 += m.width * 128 * nsl8;
    P->w8_bytes = s8;
    P->gmul_byte = r8 * 128;
    P->gadd_byte = r8 * 128 + 4 * bias;
    P->gin_byte = r8 * 128 + 8 * bias;
    bytes = (long long)r8 * 128 + 8LL * bias + 16;
  }
  if (m.C > 0) {  // FP32 slot embeddings [4][C] after everything the MLP kernels read
    bytes = (bytes + 15) / 16 * 16;
    P->slot_byte = (int)bytes;
    bytes += 16LL * m.C;
  }
  *stride = (bytes + 1023) / 1024 * 1024;
  P->rows_per_prim = (int)(*stride / 128);
  P->kmax = kmax;
  P->a_bytes = tc::kM * kmax * 2;
  return true;
}

// Epilogue groups of the forward kernel (chunks of 128 sample rows in flight per CTA). Default:
// registers cap the feature-head variants at three groups (the head keeps 4 + 32 values per
// thread), TMEM and shared memory (a 32 KB operand tile per group) cap width 128 at two.
// Width 64 without a feature head runs with 2 to 5 in BF16 and 2 to 6 in E4M3 (the autotuner's
// choices).
int tc_fwd_groups(int width, int F, int groups, bool e4m3) {
  // BF16 at width 64 runs five groups in 96 registers (TMEM holds five groups' accumulators and
  // A operands); E4M3, with narrower A operands and a one-FMA epilogue, runs six
  const int def = width == 64 ? (F > 0 ? 3 : (e4m3 ? 6 : 5)) : 2;
  if (groups == 0) return def;
  // groups also hold their A operand in TMEM (96 columns each at width 64 in BF16, 80 in E4M3)
  if (width == 64 && F == 0) return (groups >= 2 && groups <= (e4m3 ? 6 : 5)) ? groups : 0;
  return groups == def ? groups : 0;
}

// The groups a plan runs with: an explicit choice as given; the default reduced (at width 64
// without features, where 2..6 are allowed) until the shared memory fits, e.g. for wide encoded
// inputs (two K atoms) with one sample per interval (128 interval records per chunk).
int tc_fwd_groups_for(const TcPlan& P, int F, int groups, int S) {
  const int width = P.npad[0];  // hidden width = N of layer 0
  const bool e4m3 = P.w8_bytes > 0;
  int g = tc_fwd_groups(width, F, groups, e4m3);
  const int ipc = S <= 128 ? 128 / S : 1;
  if (groups == 0 && width == 64 && F == 0)
    while (g > 2 && tc::tc_smem(P, g, e4m3, ipc).total + 1024 > 227 * 1024) --g;
  return g;
}

size_t tc_smem_bytes(const TcPlan& P, int F, int groups, int S) {
  const int neg = tc_fwd_groups_for(P, F, groups, S);
  return tc::tc_smem(P, neg > 0 ? neg : 5, P.w8_bytes > 0, S <= 128 ? 128 / S : 1).total + 1024;
}

void launch_pack_bf16(const Model& m, const TcPlan& P, long long stride, int K, const float* w,
                      void* out, cudaStream_t st) {
  if (K == 0) return;
  dim3 grid(8, K);
  tc::k_pack_bf16<<<grid, 256, 0, st>>>(m, P, stride, K, w, static_cast<unsigned char*>(out));
  if (P.w8_bytes > 0) tc::k_pack_e4m3<<<K, 128, 0, st>>>(m, P, stride, K, w, static_cast<unsigned char*>(out));
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

cudaError_t launch_mlp_fwd_tc(const Work& w, const MlpArgs& a, const TcPlan& P, int n_sm,
                              cudaStream_t st) {
  auto encode = get_encode();
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
  const int neg = tc_fwd_groups_for(P, a.m.F, a.groups, a.m.S);
  if (neg == 0) return cudaErrorNotSupported;
  const size_t smem = tc_smem_bytes(P, a.m.F, a.groups, a.m.S);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  const int xl = a.m.xyzL, dl = a.m.dirL;
  const bool fast64 = xl == 6 && dl == 4 && P.kpad[0] == 64 && !a.m.contact;
  const bool raw = xl == 0 && dl == 0 && P.kpad[0] == 64 && !a.m.contact;
  decltype(&tc::k_mlp_fwd_tc<64, 6, 4, 0, 4, false>) kern;
  const bool feat = a.m.F > 0;
#define MLPS_BY_GROUPS(W, XL, DL, F8) \
  (neg == 2 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 2, F8> : neg == 3 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 3, F8> \
            : neg == 4 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 4, F8> : neg == 5 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 5, F8> \
            : a.m.nl == 4 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 6, F8, 4> : tc::k_mlp_fwd_tc<W, XL, DL, 0, 6, F8>)
#define MLPS_BY_GROUPS5(W, XL, DL) \
  (neg == 2 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 2, false> : neg == 3 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 3, false> \
            : neg == 4 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 4, false> \
            : a.m.nl == 4 ? tc::k_mlp_fwd_tc<W, XL, DL, 0, 5, false, 4> : tc::k_mlp_fwd_tc<W, XL, DL, 0, 5, false>)
  if (P.w8_bytes > 0) {  // E4M3
    if (a.m.width == 64) {
      if (!feat) kern = fast64 ? MLPS_BY_GROUPS(64, 6, 4, true) : MLPS_BY_GROUPS(64, -1, -1, true);
      else kern = fast64 ? tc::k_mlp_fwd_tc<64, 6, 4, kMaxFeat, 3, true> : tc::k_mlp_fwd_tc<64, -1, -1, kMaxFeat, 3, true>;
    } else if (a.m.width == 128) {
      if (!feat) kern = fast64 ? tc::k_mlp_fwd_tc<128, 6, 4, 0, 2, true> : tc::k_mlp_fwd_tc<128, -1, -1, 0, 2, true>;
      else kern = !fast64 ? tc::k_mlp_fwd_tc<128, -1, -1, kMaxFeat, 2, true>
                  : (a.m.nl == 5 && a.m.F <= 16) ? tc::k_mlp_fwd_tc<128, 6, 4, 16, 2, true, 5>  // (the stress network)
                                : tc::k_mlp_fwd_tc<128, 6, 4, kMaxFeat, 2, true>;
    } else {
      return cudaErrorNotSupported;
    }
  } else if (a.m.width == 64) {
    if (!feat)
      kern = fast64 ? MLPS_BY_GROUPS5(64, 6, 4)
                    : (raw && neg == 4) ? tc::k_mlp_fwd_tc<64, 0, 0, 0, 4, false> : MLPS_BY_GROUPS5(64, -1, -1);
    else kern = fast64 ? tc::k_mlp_fwd_tc<64, 6, 4, kMaxFeat, 3, false> : tc::k_mlp_fwd_tc<64, -1, -1, kMaxFeat, 3, false>;
  } else if (a.m.width == 128) {
    if (!feat) kern = fast64 ? tc::k_mlp_fwd_tc<128, 6, 4, 0, 2, false> : tc::k_mlp_fwd_tc<128, -1, -1, 0, 2, false>;
    else kern = !fast64 ? tc::k_mlp_fwd_tc<128, -1, -1, kMaxFeat, 2, false>
                : (a.m.nl == 5 && a.m.F <= 16) ? tc::k_mlp_fwd_tc<128, 6, 4, 16, 2, false, 5>  // (the stress network)
                              : tc::k_mlp_fwd_tc<128, 6, 4, kMaxFeat, 2, false>;
  } else {
    return cudaErrorNotSupported;
  }
#undef MLPS_BY_GROUPS
#undef MLPS_BY_GROUPS5
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_sm, tc::threads_tc(neg), smem, st>>>(w, a, P, tmap);
  return cudaGetLastError();
}

}  // namespace mlps
