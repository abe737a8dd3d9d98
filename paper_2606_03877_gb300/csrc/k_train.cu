// k_train.cu -- the training objective and optimizer around the renderer (Sec. 3.5, App. A.4):
// the photometric loss L_rgb = (1 - lam) L1 + lam (1 - SSIM) with its gradient, the L1 feature
// loss, restricted to the selected screen tiles (tile mini-batching), and a fused Adam step.
//
// Loss (means over the selected pixels, N of them, and the channels):
//   L1   = sum_p m_p sum_c |x_pc - y_pc| / (3 N),  SSIM = sum_p m_p sum_c S_pc / (3 N),
//   S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2))
// over an 11 x 11 Gaussian window (sigma 1.5, zero padding), C1 = 0.01^2, C2 = 0.03^2.
// With E[x^2] and E[xy] the windowed second moments, S depends on x through mu_x, E[x^2] and
// E[xy] of every window q containing p, so
//   dS_q/dx_p = w_{q-p} (A_q + 2 B_q x_p + C_q y_p),
//   A = dS/dmu_x = S (2 mu_y / n1 - 2 mu_y / n2 - 2 mu_x / d1 + 2 mu_x / d2),
//   B = dS/dE[x^2] = -S / d2,  C = dS/dE[xy] = 2 S / n2,
// (n1, n2, d1, d2 the four factors of S). The loss gradient is therefore a second windowed sum:
//   dL/dx_p = lam / (3N) (w * a + 2 x_p w * b + y_p w * c)_p + (1 - lam) m_p sign(x_p - y_p) / (3N)
// with a = -m A, b = -m B, c = -m C. Two tiled separable-filter kernels: the first computes the
// window statistics, S and (a, b, c) per pixel and channel and accumulates the loss sums; the
// second filters (a, b, c) and writes dL/dx.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mlps_common.cuh"
#include "mlps_kernels.h"

namespace mlps {
namespace {

constexpr int kTW = 32, kTH = 8;      // output tile (one thread per pixel)
constexpr int kR = 5;                  // window radius (11 taps)
constexpr int kHW = kTW + 2 * kR;      // halo tile width
constexpr int kHH = kTH + 2 * kR;      // halo tile height
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Taps {
  float w[2 * kR + 1];
};

// 1-D normalised Gaussian taps (sigma 1.5), computed on the host in double and rounded once.
Taps make_taps() {
  Taps t;
  double g[2 * kR + 1], s = 0;
  for (int i = 0; i <= 2 * kR; ++i) {
    const double x = i - kR;
    g[i] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
    s += g[i];
  }
  for (int i = 0; i <= 2 * kR; ++i) t.w[i] = (float)(g[i] / s);
  return t;
}

MLPS_DEV float pix_mask(const uint8_t* tm, int v, int y, int x, int tile, int ntx, int nty) {
  if (!tm) return 1.f;
  return tm[((size_t)v * nty + y / tile) * ntx + x / tile] ? 1.f : 0.f;
}

MLPS_DEV double block_sum(double v, double* sred) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sred[warp] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sred[i];
  return t;  // valid in thread 0
}

// Window statistics, SSIM and its partials; loss sums (L1, SSIM, selected pixels) in `sums`.
__global__ void __launch_bounds__(kTW * kTH) k_ssim_fwd(int H, int W, const float* __restrict__ x,
                                                        const float* __restrict__ y, const uint8_t* tm,
                                                        int tile, int ntx, int nty, Taps taps,
                                                        float* __restrict__ abc, double* sums) {
  __shared__ float sx[3][kHH][kHW], sy[3][kHH][kHW];
  __shared__ float sh[5][kHH][kTW];
  __shared__ double sred[kTW * kTH / 32];
  const int v = blockIdx.z;
  const int x0 = blockIdx.x * kTW - kR, y0 = blockIdx.y * kTH - kR;
  const size_t img = (size_t)v * H * W;
  for (int i = threadIdx.x; i < kHH * kHW * 3; i += blockDim.x) {
    const int c = i % 3, q = i / 3, r = q / kHW, col = q - r * kHW;
    const int gy = y0 + r, gx = x0 + col;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    const size_t o = (img + (size_t)(in ? gy : 0) * W + (in ? gx : 0)) * 3 + c;
    sx[c][r][col] = in ? x[o] : 0.f;
    sy[c][r][col] = in ? y[o] : 0.f;
  }
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int px = blockIdx.x * kTW + tx, py = blockIdx.y * kTH + ty;
  const bool inside = px < W && py < H;
  const float m = inside ? pix_mask(tm, v, py, px, tile, ntx, nty) : 0.f;
  double l1 = 0.0, ss = 0.0;
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int i = threadIdx.x; i < kHH * kTW; i += blockDim.x) {
      const int r = i / kTW, col = i - r * kTW;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; ++k) {
        const float xv = sx[c][r][col + k], yv = sy[c][r][col + k], wk = taps.w[k];
        a0 = fmaf(wk, xv, a0);
        a1 = fmaf(wk, yv, a1);
        a2 = fmaf(wk, xv * xv, a2);
        a3 = fmaf(wk, yv * yv, a3);
        a4 = fmaf(wk, xv * yv, a4);
      }
      sh[0][r][col] = a0; sh[1][r][col] = a1; sh[2][r][col] = a2; sh[3][r][col] = a3; sh[4][r][col] = a4;
    }
    __syncthreads();
    if (!inside) continue;
    float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float wk = taps.w[k];
      mx = fmaf(wk, sh[0][ty + k][tx], mx);
      my = fmaf(wk, sh[1][ty + k][tx], my);
      exx = fmaf(wk, sh[2][ty + k][tx], exx);
      eyy = fmaf(wk, sh[3][ty + k][tx], eyy);
      exy = fmaf(wk, sh[4][ty + k][tx], exy);
    }
    const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
    const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
    const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
    const float S = (n1 * n2) / (d1 * d2);
    const float A = S * (2.f * my / n1 - 2.f * my / n2 - 2.f * mx / d1 + 2.f * mx / d2);
    const float B = -S / d2;
    const float Cc = 2.f * S / n2;
    const size_t plane = (size_t)H * W;
    const size_t o = (size_t)v * 9 * plane + (size_t)py * W + px;
    abc[o + (size_t)(3 * c + 0) * plane] = -m * A;
    abc[o + (size_t)(3 * c + 1) * plane] = -m * B;
    abc[o + (size_t)(3 * c + 2) * plane] = -m * Cc;
    l1 += (double)(m * fabsf(sx[c][ty + kR][tx + kR] - sy[c][ty + kR][tx + kR]));
    ss += (double)(m * S);
  }
  const double t0 = block_sum(l1, sred);
  const double t1 = block_sum(ss, sred);
  const double t2 = block_sum((double)m, sred);
  if (threadIdx.x == 0) {
    atomicAdd(&sums[0], t0);
    atomicAdd(&sums[1], t1);
    atomicAdd(&sums[2], t2);
  }
}

// dL/dx = lam / (3N) (w * a + 2 x w * b + y w * c) + (1 - lam) m sign(x - y) / (3N)
__global__ void __launch_bounds__(kTW * kTH) k_ssim_bwd(int H, int W, const float* __restrict__ x,
                                                        const float* __restrict__ y, const uint8_t* tm,
                                                        int tile, int ntx, int nty, Taps taps, float lam,
                                                        const float* __restrict__ abc, const double* sums,
                                                        float* __restrict__ dx) {
  __shared__ float sa[3][kHH][kHW];
  __shared__ float sh[3][kHH][kTW];
  const int v = blockIdx.z;
  const int x0 = blockIdx.x * kTW - kR, y0 = blockIdx.y * kTH - kR;
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int px = blockIdx.x * kTW + tx, py = blockIdx.y * kTH + ty;
  const bool inside = px < W && py < H;
  const double n = sums[2];
  const float inv = n > 0 ? (float)(1.0 / (3.0 * n)) : 0.f;
  const float m = inside ? pix_mask(tm, v, py, px, tile, ntx, nty) : 0.f;
  const size_t plane = (size_t)H * W;
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * kHH * kHW; i += blockDim.x) {
      const int k = i / (kHH * kHW), q = i - k * (kHH * kHW), r = q / kHW, col = q - r * kHW;
      const int gy = y0 + r, gx = x0 + col;
      const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
      sa[k][r][col] = in ? abc[(size_t)v * 9 * plane + (size_t)(3 * c + k) * plane + (size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHH * kTW; i += blockDim.x) {
      const int r = i / kTW, col = i - r * kTW;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; ++k) {
        const float wk = taps.w[k];
        a0 = fmaf(wk, sa[0][r][col + k], a0);
        a1 = fmaf(wk, sa[1][r][col + k], a1);
        a2 = fmaf(wk, sa[2][r][col + k], a2);
      }
      sh[0][r][col] = a0; sh[1][r][col] = a1; sh[2][r][col] = a2;
    }
    __syncthreads();
    if (!inside) continue;
    float fa = 0.f, fb = 0.f, fc = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * kR; ++k) {
      const float wk = taps.w[k];
      fa = fmaf(wk, sh[0][ty + k][tx], fa);
      fb = fmaf(wk, sh[1][ty + k][tx], fb);
      fc = fmaf(wk, sh[2][ty + k][tx], fc);
    }
    const size_t o = ((size_t)v * plane + (size_t)py * W + px) * 3 + c;
    const float xv = x[o], yv = y[o];
    const float d = xv - yv;
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    dx[o] = inv * (lam * (fa + 2.f * xv * fb + yv * fc) + (1.f - lam) * m * sgn);
  }
}

// L1 feature loss: sum and gradient m sign(F - F*) / (C N). One warp per pixel (the mask once per
// pixel), lanes over the channels, float4 when the rows allow it.
MLPS_DEV float sgnf(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__global__ void k_feat_l1(int V, int H, int W, int C, const float* __restrict__ f, const float* __restrict__ ft,
                          const uint8_t* tm, int tile, int ntx, int nty, const double* sums, double* fsum,
                          float* __restrict__ df, int vec) {
  __shared__ double sred[8];
  const double n = sums[2];
  const float inv = n > 0 ? (float)(1.0 / ((double)C * n)) : 0.f;
  const int lane = threadIdx.x & 31;
  const long long npix = (long long)V * H * W;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  double acc = 0.0;
  for (long long p = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < npix; p += nwarps) {
    const int v = (int)(p / ((long long)H * W));
    const int r = (int)(p - (long long)v * H * W);
    const int yy = r / W, xx = r - yy * W;
    const float m = pix_mask(tm, v, yy, xx, tile, ntx, nty);
    const float* a = f + p * C;
    const float* b = ft + p * C;
    float* g = df ? df + p * C : nullptr;
    float part = 0.f;
    if (vec) {
      for (int c = 4 * lane; c < C; c += 128) {
        const float4 x = *reinterpret_cast<const float4*>(a + c);
        const float4 y = *reinterpret_cast<const float4*>(b + c);
        const float4 d = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
        part += fabsf(d.x) + fabsf(d.y) + fabsf(d.z) + fabsf(d.w);
        if (g) *reinterpret_cast<float4*>(g + c) =
            make_float4(m * inv * sgnf(d.x), m * inv * sgnf(d.y), m * inv * sgnf(d.z), m * inv * sgnf(d.w));
      }
    } else {
      for (int c = lane; c < C; c += 32) {
        const float d = a[c] - b[c];
        part += fabsf(d);
        if (g) g[c] = m * inv * sgnf(d);
      }
    }
    acc += (double)(m * part);
  }
  const double t = block_sum(acc, sred);
  if (threadIdx.x == 0) atomicAdd(fsum, t);
}

// loss_out = {L, L1, SSIM, N, L_f}
__global__ void k_loss_finalize(const double* sums, float lam, int has_feat, int C, float* out) {
  const double n = sums[2];
  const double l1 = n > 0 ? sums[0] / (3.0 * n) : 0.0;
  const double ss = n > 0 ? sums[1] / (3.0 * n) : 0.0;
  const double lf = (has_feat && n > 0) ? sums[3] / ((double)C * n) : 0.0;
  out[0] = (float)((1.0 - lam) * l1 + lam * (1.0 - ss) + lf);
  out[1] = (float)l1;
  out[2] = (float)ss;
  out[3] = (float)n;
  out[4] = (float)lf;
}

// ------------------------------------------------------------------------------------------
// Adam

struct AdamGroups {
  AdamGroupDev g[kMaxAdamGroups];
  long long start[kMaxAdamGroups + 1];
  int n;
};

__global__ void k_adam(AdamGroups G, float beta1, float beta2, float eps, float bc1, float bc2) {
  const long long total = G.start[G.n];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (i >= G.start[k + 1]) ++k;
    const AdamGroupDev& a = G.g[k];
    const long long j = i - G.start[k];
    float g = a.grad[j];
    if (a.kind == 1) g *= a.aux[j];  // log-parameter: dL/dlog x = dL/dx * x
    const float m = fmaf(beta1, a.m[j], (1.f - beta1) * g);
    const float v = fmaf(beta2, a.v[j], (1.f - beta2) * g * g);
    a.m[j] = m;
    a.v[j] = v;
    const float p = a.param[j] - a.lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    a.param[j] = p;
    if (a.kind == 1) a.aux[j] = expf(p);
  }
}

}  // namespace

void launch_loss(int V, int H, int W, const float* rgb, const float* rgb_t, const uint8_t* tm, int tile,
                 float lam, int C, const float* feat, const float* feat_t, float* d_rgb, float* d_feat,
                 float* abc, double* sums, float* loss_out, cudaStream_t st) {
  const int ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
  const Taps taps = make_taps();
  cudaMemsetAsync(sums, 0, 4 * sizeof(double), st);
  const dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, V);
  k_ssim_fwd<<<grid, kTW * kTH, 0, st>>>(H, W, rgb, rgb_t, tm, tile, ntx, nty, taps, abc, sums);
  k_ssim_bwd<<<grid, kTW * kTH, 0, st>>>(H, W, rgb, rgb_t, tm, tile, ntx, nty, taps, lam, abc, sums, d_rgb);
  if (C > 0) {
    const bool vec = C % 4 == 0 && ((reinterpret_cast<uintptr_t>(feat) | reinterpret_cast<uintptr_t>(feat_t) |
                                     reinterpret_cast<uintptr_t>(d_feat)) & 15) == 0;
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    k_feat_l1<<<8 * n_sm, 256, 0, st>>>(V, H, W, C, feat, feat_t, tm, tile, ntx, nty, sums, sums + 3, d_feat, vec);
  }
  k_loss_finalize<<<1, 1, 0, st>>>(sums, lam, C > 0, C, loss_out);
}

void launch_adam(const AdamGroupDev* groups, int n, float beta1, float beta2, float eps, int step,
                 int n_sm, cudaStream_t st) {
  AdamGroups G;
  G.n = n;
  G.start[0] = 0;
  for (int k = 0; k < n; ++k) {
    G.g[k] = groups[k];
    G.start[k + 1] = G.start[k] + groups[k].n;
  }
  if (G.start[n] == 0) return;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, step));
  const long long blocks = (G.start[n] + 255) / 256;
  k_adam<<<(int)(blocks < 8LL * n_sm ? blocks : 8LL * n_sm), 256, 0, st>>>(G, beta1, beta2, eps, bc1, bc2);
}

}  // namespace mlps
