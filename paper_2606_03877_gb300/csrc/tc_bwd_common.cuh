// tc_bwd_common.cuh -- device helpers shared by the tensor-core MLP backward kernels: MN-major
// shared-memory descriptors, sample-row writers of the swizzled operand tiles, the encoding of
// Eq. 5 in registers and its derivative.
#pragma once

#include <cuda_runtime.h>

#include "mlps_common.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace mlps {
namespace tc {

// MN-major 128-byte-swizzle descriptor: 8-row K groups 1024 bytes apart (SBO), MN atoms of 64
// elements `lbo` bytes apart (LBO).
MLPS_DEV uint64_t sw128_desc_mn(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Store 64 values of one row (BF16-packed pairs) into a swizzled tile.
MLPS_DEV void store_row64(uint32_t tile, int row, const uint32_t (&pk)[32]) {
  const RowSw sw(row);
#pragma unroll
  for (int ch = 0; ch < 8; ++ch)
    st_shared_v4(tile + sw.off(ch), pk[4 * ch], pk[4 * ch + 1], pk[4 * ch + 2], pk[4 * ch + 3]);
}

MLPS_DEV void ld_shared_v4(uint32_t addr, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
               : "r"(addr)
               : "memory");
}

// Encoded input row (Eq. 5) of one sample into tile `A` with compile-time frequency counts
// (zeros for rows past the chunk's intervals).
template <int XL, int DL>
MLPS_DEV void encode_row64(const IntervalRec* T, int nint, int S, int row, uint32_t (&pk)[32]) {
  const int iv = row / S, k = row - iv * S;
  if (iv < nint) {
    const IntervalRec& I = T[iv];
    const float tr = I.r0 + ((float)k + 0.5f) * I.dt;
    float xl[3], d[3];
    for (int u = 0; u < 3; ++u) { xl[u] = fmaf(tr, I.dp[u], I.p[u]); d[u] = I.d[u]; }
    encode_pairs64<XL, DL>(xl, d, pk);
  } else {
#pragma unroll
    for (int e = 0; e < 32; ++e) pk[e] = 0u;
  }
}

template <int XL, int DL>
MLPS_DEV void build_row64(const IntervalRec* T, int nint, int S, int row, uint32_t A) {
  uint32_t pk[32];
  encode_row64<XL, DL>(T, nint, S, row, pk);
  store_row64(A, row, pk);
}

// dL/dx_local of one sample from dL/dX (64 values in registers) through the encoding of Eq. 5:
// d/dx [sin(2^l pi x), cos(2^l pi x)] = 2^l pi [cos, -sin].
template <int XL>
MLPS_DEV void enc_grad64(const float (&xl)[3], const uint32_t (&v0)[32], const uint32_t (&v1)[32],
                         float (&gx)[3]) {
  if (XL == 0) {
    for (int u = 0; u < 3; ++u) gx[u] = __uint_as_float(v0[u]);
    return;
  }
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    float sn, cs;
    __sincosf(3.14159265358979f * xl[u], &sn, &cs);
    float wq = 3.14159265358979f, acc = 0.f;
#pragma unroll
    for (int l = 0; l < (XL > 0 ? XL : 1); ++l) {
      const int c = 2 * (u * XL + l);
      const float g0 = __uint_as_float(c < 32 ? v0[c] : v1[(c - 32) & 31]);
      const float g1 = __uint_as_float(c + 1 < 32 ? v0[c + 1] : v1[(c + 1 - 32) & 31]);
      acc += wq * (g0 * cs - g1 * sn);
      const float s2 = 2.f * sn * cs;
      cs = fmaf(-2.f * sn, sn, 1.f);
      sn = s2;
      wq *= 2.f;
    }
    gx[u] = acc;
  }
}

// The same for coordinate U alone: the terms of enc_grad64 that make gx[U], in the same order.
template <int XL, int U>
MLPS_DEV float enc_grad_coord(float xu, const uint32_t (&v0)[32], const uint32_t (&v1)[32]) {
  if (XL == 0) return __uint_as_float(v0[U]);
  float sn, cs;
  __sincosf(3.14159265358979f * xu, &sn, &cs);
  float wq = 3.14159265358979f, acc = 0.f;
#pragma unroll
  for (int l = 0; l < (XL > 0 ? XL : 1); ++l) {
    const int c = 2 * (U * XL + l);
    const float g0 = __uint_as_float(c < 32 ? v0[c] : v1[(c - 32) & 31]);
    const float g1 = __uint_as_float(c + 1 < 32 ? v0[c + 1] : v1[(c + 1 - 32) & 31]);
    acc += wq * (g0 * cs - g1 * sn);
    const float s2 = 2.f * sn * cs;
    cs = fmaf(-2.f * sn, sn, 1.f);
    sn = s2;
    wq *= 2.f;
  }
  return acc;
}

MLPS_DEV void build_row(const Model& m, const IntervalRec* T, int nint, int row, uint32_t A,
                        int kpad0) {
  const int S = m.S;
  const int iv = row / S, k = row - iv * S;
  RowWriter rw{A, row, 0, 0.f};
  if (iv < nint) {
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
  rw.pad_to(kpad0);
}

}  // namespace tc
}  // namespace mlps
