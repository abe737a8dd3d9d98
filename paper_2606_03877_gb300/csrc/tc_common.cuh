// tc_common.cuh -- device helpers shared by the tensor-core MLP kernels: segmented scans over
// a 128-row epilogue group, BF16 operand-row writers and the angle-doubling encoding.
#pragma once

#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "tc_ptx.cuh"

namespace mlps {
namespace tc {

constexpr int kM = 128;
constexpr int kEGThreads = 128;
constexpr int kMaxScanVals = 4 + kMaxFeat;

// Inclusive segmented scan of NV values over the 128 rows of one epilogue group. Segments
// are [j*S, (j+1)*S). `scratch` holds 4 warps x NV floats of this group.
template <int NV>
MLPS_DEV void seg_scan(float (&v)[NV], int nv, int row, int S, float* scratch, int bar_id) {
  const int lane = row & 31, wq = row >> 5;
  const int seg0 = (row / S) * S;
  const int lo = max(seg0, wq * 32) - wq * 32;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      if (j >= nv) break;
      const float y = __shfl_up_sync(0xffffffffu, v[j], o);
      if (lane - o >= lo) v[j] += y;
    }
  }
  if (S <= 32 && (32 % S) == 0) return;  // segments never cross a warp
  if (lane == 31) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < nv) scratch[wq * NV + j] = v[j];
  }
  named_bar_sync(bar_id, kEGThreads);
  if (seg0 < wq * 32)
    for (int w2 = seg0 / 32; w2 < wq; ++w2) {
#pragma unroll
      for (int j = 0; j < NV; ++j)
        if (j < nv) v[j] += scratch[w2 * NV + j];
    }
  named_bar_sync(bar_id, kEGThreads);
}

// Segmented sum of NV values over the 128 rows: the segment's last row gets its total. With S
// dividing 32 a segment lives inside one warp and the sum is a butterfly over its lanes (every
// row gets the total); otherwise it is the inclusive scan.
template <int NV>
MLPS_DEV void seg_sum(float (&v)[NV], int nv, int row, int S, float* scratch, int bar_id) {
  if (S <= 32 && (32 % S) == 0) {
    for (int o = 1; o < S; o <<= 1) {
#pragma unroll
      for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
    (void)nv;
    (void)row;
    (void)scratch;
    (void)bar_id;
    return;
  }
  seg_scan<NV>(v, nv, row, S, scratch, bar_id);
}

MLPS_DEV float sigmoid_fast(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
MLPS_DEV float softplus_fast(float z) { return fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z))); }

// Contact-point residual delta = mu - p* = -R S p + min(t_mid, 0) d (Eq. 3) of an interval,
// from its closest point p in the primitive's normalised frame.
MLPS_DEV void contact_delta(const PrimGeo& G, const IntervalRec& I, float del[3]) {
  const float tn = fminf(I.tmid, 0.f);
  for (int q = 0; q < 3; ++q) {
    const float y = G.R[q * 3] * G.s[0] * I.p[0] + G.R[q * 3 + 1] * G.s[1] * I.p[1] + G.R[q * 3 + 2] * G.s[2] * I.p[2];
    del[q] = fmaf(tn, I.d[q], -y);
  }
}

struct RowWriter {  // writes one sample row of a K-major swizzled BF16 A tile, two values at a time
  uint32_t base;
  int row, col;
  float pend;
  MLPS_DEV void put(float v) {
    if (col & 1) {
      const int c0 = col - 1;
      const uint32_t addr = base + (uint32_t)(c0 >> 6) * (kM * 128) + sw128_off(row, (c0 & 63) >> 3) +
                            (uint32_t)((c0 & 7) >> 1) * 4;
      st_shared_u32(addr, pack_bf16(pend, v));
    } else {
      pend = v;
    }
    ++col;
  }
  MLPS_DEV void pad_to(int n) {
    while (col < n) put(0.f);
  }
};

// Encoding gamma (Eq. 5) with one sincos per component and angle doubling
// (sin 2u = 2 sin u cos u, cos 2u = 1 - 2 sin^2 u); arguments pi * p lie in [-pi, pi].
MLPS_DEV void put_gamma(RowWriter& rw, float p, int L) {
  float s, c;
  __sincosf(3.14159265358979f * p, &s, &c);
  for (int l = 0; l < L; ++l) {
    rw.put(s);
    rw.put(c);
    const float s2 = 2.f * s * c;
    c = fmaf(-2.f * s, s, 1.f);
    s = s2;
  }
}


// Suffix (reverse) segmented scan: v[j] becomes the sum over rows r' >= row of the same segment.
template <int NV>
MLPS_DEV void seg_scan_rev(float (&v)[NV], int nv, int row, int S, float* scratch, int bar_id) {
  const int lane = row & 31, wq = row >> 5;
  const int seg0 = (row / S) * S;
  const int seg1 = seg0 + S - 1;                     // last row of the segment
  const int hi = min(seg1, wq * 32 + 31) - wq * 32;  // last lane of the segment in this warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      if (j >= nv) break;
      const float y = __shfl_down_sync(0xffffffffu, v[j], o);
      if (lane + o <= hi) v[j] += y;
    }
  }
  if (S <= 32 && (32 % S) == 0) return;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < nv) scratch[wq * NV + j] = v[j];
  }
  named_bar_sync(bar_id, kEGThreads);
  if (seg1 > wq * 32 + 31)
    for (int w2 = wq + 1; w2 <= seg1 / 32; ++w2) {
#pragma unroll
      for (int j = 0; j < NV; ++j)
        if (j < nv) v[j] += scratch[w2 * NV + j];
    }
  named_bar_sync(bar_id, kEGThreads);
}

// MMAs of one forward layer of a 128-row chunk: D[128 x npad] = A[128 x kpad] W^T, A and W in
// the K-major swizzled layout, K in 64-column slabs (kpad <= 128). Issued by one thread. The
// descriptors are built once; stepping K only moves their start-address field (address >> 4).
// With `bt` nonzero one more K step adds the bias: A = the `ones` tile (every row (1, 0, ...)),
// B = the K step of the bias tile that holds this layer's bias in its first column.
MLPS_DEV void issue_fwd_layer(uint32_t A, uint32_t W, uint32_t d, int kpad, int npad, uint32_t ones = 0u,
                              uint32_t bt = 0u) {
  const uint32_t idesc = idesc_bf16(kM, npad);
  const uint64_t da = sw128_desc(A), db = sw128_desc(W);
  const uint32_t wslab = (uint32_t)npad * 8;  // (npad * 128 bytes) >> 4: one 64-column slab of W
  const int nk = kpad / 16;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    if (kk >= nk) break;
    const uint32_t oa = (uint32_t)(kk >> 2) * (kM * 8) + (uint32_t)(kk & 3) * 2;
    const uint32_t ob = (uint32_t)(kk >> 2) * wslab + (uint32_t)(kk & 3) * 2;
    mma_bf16(d, da + oa, db + ob, idesc, kk > 0 ? 1u : 0u);
  }
  if (bt) mma_bf16(d, sw128_desc(ones), sw128_desc(bt), idesc, 1u);
}

// Forward layer with the A operand in tensor memory (`At`: lane = sample row, BF16 pairs along
// the columns, 8 columns per K = 16 step); W and the folded bias as in issue_fwd_layer.
MLPS_DEV void issue_fwd_layer_ta(uint32_t At, uint32_t W, uint32_t d, int kpad, int npad, uint32_t ones = 0u,
                                 uint32_t bt = 0u) {
  const uint32_t idesc = idesc_bf16(kM, npad);
  const uint64_t db = sw128_desc(W);
  const uint32_t wslab = (uint32_t)npad * 8;
  const int nk = kpad / 16;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    if (kk >= nk) break;
    const uint32_t ob = (uint32_t)(kk >> 2) * wslab + (uint32_t)(kk & 3) * 2;
    mma_bf16_ta(d, At + 8u * (uint32_t)kk, db + ob, idesc, kk > 0 ? 1u : 0u);
  }
  if (bt) mma_bf16(d, sw128_desc(ones), sw128_desc(bt), idesc, 1u);
}

// FP8 (E4M3) forward layer: same operand tiles (128-byte K-major swizzled rows, here holding up
// to 128 one-byte elements), K = 32 per instruction; kpad <= 128.
MLPS_DEV void issue_fwd_layer_e4m3(uint32_t A, uint32_t W, uint32_t d, int kpad, int npad, uint32_t ones = 0u,
                                   uint32_t bt = 0u) {
  const uint32_t idesc = idesc_e4m3(kM, npad);
  const uint64_t da = sw128_desc(A), db = sw128_desc(W);
  const int nk = kpad / 32;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    if (kk >= nk) break;
    mma_e4m3(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, kk > 0 ? 1u : 0u);
  }
  if (bt) mma_e4m3_ta(d, ones, sw128_desc(bt), idesc, 1u);
}

// E4M3 layer with the A operand in tensor memory (`At`: lane = sample row, four E4M3 values per
// column, 8 columns per K = 32 step).
// With `bt` nonzero one more K step adds the layer's bias: A = the constant-1 operand `ones` in
// TMEM (1.0 in the first two elements of every row), B = the K step of the bias tile that holds
// the layer's bias as hi and lo bytes in its first two columns.
MLPS_DEV void issue_fwd_layer_e4m3_ta(uint32_t At, uint32_t W, uint32_t d, int kpad, int npad, uint32_t ones = 0u,
                                      uint32_t bt = 0u) {
  const uint32_t idesc = idesc_e4m3(kM, npad);
  const uint64_t db = sw128_desc(W);
  const int nk = kpad / 32;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    if (kk >= nk) break;
    mma_e4m3_ta(d, At + 8u * (uint32_t)kk, db + (uint64_t)(kk * 2), idesc, kk > 0 ? 1u : 0u);
  }
  if (bt) mma_e4m3_ta(d, ones, sw128_desc(bt), idesc, 1u);
}

// Writes one sample row of an E4M3 A tile (one byte per column, 128-byte swizzled rows), two
// values at a time.
struct RowWriter8 {
  uint32_t base;
  int row, col;
  float pend, mul;
  MLPS_DEV void put(float v) {
    if (col & 1) {
      const int c0 = col - 1;
      st_shared_u16(base + sw128_off(row, c0 >> 4) + (uint32_t)(c0 & 15), pack_e4m3(pend * mul, v * mul));
    } else {
      pend = v;
    }
    ++col;
  }
  MLPS_DEV void pad_to(int n) {
    while (col < n) put(0.f);
  }
};

MLPS_DEV void put_gamma8(RowWriter8& rw, float p, int L) {
  float s, c;
  __sincosf(3.14159265358979f * p, &s, &c);
  for (int l = 0; l < L; ++l) {
    rw.put(s);
    rw.put(c);
    const float s2 = 2.f * s * c;
    c = fmaf(-2.f * s, s, 1.f);
    s = s2;
  }
}

// One step of a block's chunk schedule: up to NG consecutive chunks of the same primitive,
// one per epilogue group. Every role evaluates the same schedule.
template <int NG>
struct ChunkStep {
  int c0, prim, n;
  int c[6];  // chunk per group (-1: none); accessed with compile-time indices only
};

template <int NG>
MLPS_DEV ChunkStep<NG> chunk_step(const Work& w, int c, int ce, int prim) {
  static_assert(NG >= 1 && NG <= 6, "at most six epilogue groups");
  ChunkStep<NG> s;
  s.c0 = c;
  if (c < ce)
    while (c >= w.chunk_start[prim + 1]) ++prim;
  s.prim = prim;
  const int lim = min(ce, w.chunk_start[prim + 1]);
  s.c[0] = c < lim ? c : -1;
  s.c[1] = (NG > 1 && c + 1 < lim) ? c + 1 : -1;
  s.c[2] = (NG > 2 && c + 2 < lim) ? c + 2 : -1;
  s.c[3] = (NG > 3 && c + 3 < lim) ? c + 3 : -1;
  s.c[4] = (NG > 4 && c + 4 < lim) ? c + 4 : -1;
  s.c[5] = (NG > 5 && c + 5 < lim) ? c + 5 : -1;
  s.n = (s.c[0] >= 0) + (s.c[1] >= 0) + (s.c[2] >= 0) + (s.c[3] >= 0) + (s.c[4] >= 0) + (s.c[5] >= 0);
  return s;
}

// Chunk of group g in a step (register selects; no dynamic indexing).
template <int NG>
MLPS_DEV int step_chunk(const ChunkStep<NG>& s, int g) {
  return g == 0 ? s.c[0] : g == 1 ? s.c[1] : g == 2 ? s.c[2] : g == 3 ? s.c[3] : g == 4 ? s.c[4] : s.c[5];
}

// Asynchronous global -> shared copies (cp.async, 16 bytes each): the next chunk's interval
// records travel to shared memory while the current chunk is processed, holding no registers.
MLPS_DEV void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
MLPS_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
MLPS_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Start copying interval record `slot` (64 bytes) to shared address `dst_rec` and, when
// `dst_grad` is nonzero, its interval gradient (16 bytes) to `dst_grad`.
MLPS_DEV void rec_copy_async(const Work& w, int slot, uint32_t dst_rec, uint32_t dst_grad) {
  const char* src = reinterpret_cast<const char*>(w.rec + slot);
#pragma unroll
  for (int i = 0; i < 4; ++i) cp_async16(dst_rec + 16u * i, src + 16 * i);
  if (dst_grad) cp_async16(dst_grad, w.hit_grad + slot);
  cp_async_commit();
}

// Encoded input row (Eq. 5) with the frequency counts known at compile time: all values are
// produced in registers, packed to BF16 pairs and written with 16-byte stores. XL = 0 means the
// raw local position; DL = 0 means no direction input. Columns past the encoding are zero.
template <int XL, int DL>
MLPS_DEV void encode_pairs64(const float (&xl)[3], const float (&d)[3], uint32_t (&pk)[32]) {
  constexpr int NX = XL > 0 ? 6 * XL : 3;
  constexpr int NIN = NX + (DL > 0 ? 6 * DL : 0);
  static_assert(NIN <= 64, "encoded input wider than one 64-column tile");
  static_assert(XL > 0 || DL == 0, "raw position with a direction encoding is not a fast path");
#pragma unroll
  for (int e = 0; e < 32; ++e) pk[e] = 0u;
  if (XL == 0) {
    pk[0] = pack_bf16(xl[0], xl[1]);
    pk[1] = pack_bf16(xl[2], 0.f);
    return;
  }
  // every (sin, cos) pair of one frequency is exactly one BF16x2 word
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    float s, c;
    __sincosf(3.14159265358979f * xl[u], &s, &c);
#pragma unroll
    for (int l = 0; l < (XL > 0 ? XL : 1); ++l) {
      pk[u * XL + l] = pack_bf16(s, c);
      const float s2 = 2.f * s * c;
      c = fmaf(-2.f * s, s, 1.f);
      s = s2;
    }
  }
  if (DL > 0) {
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      float s, c;
      __sincosf(3.14159265358979f * d[u], &s, &c);
#pragma unroll
      for (int l = 0; l < (DL > 0 ? DL : 1); ++l) {
        pk[NX / 2 + u * DL + l] = pack_bf16(s, c);
        const float s2 = 2.f * s * c;
        c = fmaf(-2.f * s, s, 1.f);
        s = s2;
      }
    }
  }
}

// Encoded input row as E4M3 bytes (values times `mul`), compile-time frequency counts, same
// order as encode_pairs64: word e holds columns 4e .. 4e + 3 (low byte first).
template <int XL, int DL>
MLPS_DEV void encode_e4m3_64(const float (&xl)[3], const float (&d)[3], float mul, uint32_t (&pk)[16]) {
  constexpr int NX = XL > 0 ? 6 * XL : 3;
  constexpr int NIN = NX + (DL > 0 ? 6 * DL : 0);
  static_assert(NIN <= 64, "encoded input wider than one 64-column tile");
  static_assert(XL > 0 || DL == 0, "raw position with a direction encoding is not a fast path");
#pragma unroll
  for (int e = 0; e < 16; ++e) pk[e] = 0u;
  if (XL == 0) {
    pk[0] = pack_e4m3(xl[0] * mul, xl[1] * mul) | (pack_e4m3(xl[2] * mul, 0.f) << 16);
    return;
  }
  // pair p (one frequency's sin, cos) is the 16-bit half p & 1 of word p >> 1
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    float s, c;
    __sincosf(3.14159265358979f * xl[u], &s, &c);
#pragma unroll
    for (int l = 0; l < (XL > 0 ? XL : 1); ++l) {
      const int p = u * XL + l;
      pk[p >> 1] |= pack_e4m3(s * mul, c * mul) << (16 * (p & 1));
      const float s2 = 2.f * s * c;
      c = fmaf(-2.f * s, s, 1.f);
      s = s2;
    }
  }
  if (DL > 0) {
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      float s, c;
      __sincosf(3.14159265358979f * d[u], &s, &c);
#pragma unroll
      for (int l = 0; l < (DL > 0 ? DL : 1); ++l) {
        const int p = NX / 2 + u * DL + l;
        pk[p >> 1] |= pack_e4m3(s * mul, c * mul) << (16 * (p & 1));
        const float s2 = 2.f * s * c;
        c = fmaf(-2.f * s, s, 1.f);
        s = s2;
      }
    }
  }
}

}  // namespace tc
}  // namespace mlps
