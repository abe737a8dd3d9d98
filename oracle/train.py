"""FP64 reference of the training objective and the optimizer step (Sec. 3.5, App. A.4).

TEST INFRASTRUCTURE ONLY: the test suite and the benchmark's CPU-baseline leg are the only
callers. Plain numpy and PyTorch CPU operations in float64; nothing here is imported by, or
imports, the CUDA package.

Objective, per training step over V views of H x W pixels:
  * a mask of screen tiles (tile mini-batching: only the selected T x T tiles enter the loss);
    m_p = 1 for the pixels of selected tiles, N = sum_p m_p;
  * L_rgb = (1 - lam) * L1 + lam * (1 - SSIM), with
    L1   = sum_p m_p sum_c |C_pc - C*_pc| / (3 N)  (Eq. 7, the norm read as a mean),
    SSIM = sum_p m_p sum_c S_pc / (3 N),  S the per-pixel SSIM map of each colour channel:
           11 x 11 Gaussian window with sigma 1.5, zero padding at the image border,
           S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
           C1 = 0.01^2, C2 = 0.03^2 (the common SSIM constants for images in [0, 1]);
  * with features, L_f = sum_p m_p sum_f |F_pf - F*_pf| / (F N) (Eq. 8, also a mean), and
    L = L_rgb + L_f.
The gradient dL/dC (and dL/dF) is taken by reverse-mode autodiff of these float64 formulas;
|x| has derivative sign(x), 0 at x = 0.

Adam (the textbook update): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). A log-parameter group (the
log-scales) holds p = log x, takes g = dL/dx * x, and returns x = exp(p) as well.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window() -> np.ndarray:
    """Normalised 1-D Gaussian taps (the 2-D window is their outer product)."""
    x = np.arange(WINDOW, dtype=np.float64) - (WINDOW - 1) / 2.0
    g = np.exp(-x * x / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def pixel_mask(V: int, H: int, W: int, tile: int, tile_mask: Optional[np.ndarray]) -> np.ndarray:
    """m [V, H, W] from the per-tile selection [V, ceil(H/T), ceil(W/T)] (None = all pixels)."""
    if tile_mask is None:
        return np.ones((V, H, W))
    tm = np.asarray(tile_mask).astype(np.float64)
    return np.repeat(np.repeat(tm, tile, axis=1), tile, axis=2)[:, :H, :W]


def ssim_map_torch(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Per-pixel SSIM of images [V, H, W, 3] (float64), per channel: [V, H, W, 3]."""
    g = torch.from_numpy(gaussian_window())
    w2 = (g[:, None] * g[None, :])[None, None]  # [1, 1, 11, 11]
    xc = x.permute(0, 3, 1, 2).reshape(-1, 1, x.shape[1], x.shape[2])
    yc = y.permute(0, 3, 1, 2).reshape(-1, 1, y.shape[1], y.shape[2])
    f = lambda t: torch.nn.functional.conv2d(t, w2, padding=WINDOW // 2)
    mx, my = f(xc), f(yc)
    sxx = f(xc * xc) - mx * mx
    syy = f(yc * yc) - my * my
    sxy = f(xc * yc) - mx * my
    s = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return s.reshape(x.shape[0], 3, x.shape[1], x.shape[2]).permute(0, 2, 3, 1)


def ssim_map_loops(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The same SSIM map written as explicit window sums (a slow restatement for the pins)."""
    V, H, W, _ = x.shape
    g = gaussian_window()
    r = WINDOW // 2
    out = np.zeros(x.shape)
    for v in range(V):
        for c in range(3):
            for i in range(H):
                for j in range(W):
                    mx = my = exx = eyy = exy = 0.0
                    for a in range(-r, r + 1):
                        for b in range(-r, r + 1):
                            ii, jj = i + a, j + b
                            if 0 <= ii < H and 0 <= jj < W:
                                wgt = g[a + r] * g[b + r]
                                xv, yv = x[v, ii, jj, c], y[v, ii, jj, c]
                                mx += wgt * xv
                                my += wgt * yv
                                exx += wgt * xv * xv
                                eyy += wgt * yv * yv
                                exy += wgt * xv * yv
                    sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
                    out[v, i, j, c] = ((2 * mx * my + C1) * (2 * sxy + C2)) / \
                        ((mx * mx + my * my + C1) * (sx + sy + C2))
    return out


def loss(rgb, rgb_target, lam: float, tile: int = 8, tile_mask=None, feat=None, feat_target=None):
    """(L, parts, dL/drgb [V,H,W,3], dL/dfeat or None); parts = {l1, ssim, l_feat, n}."""
    x = torch.tensor(np.asarray(rgb, dtype=np.float64), requires_grad=True)
    y = torch.tensor(np.asarray(rgb_target, dtype=np.float64))
    V, H, W, _ = x.shape
    m = torch.from_numpy(pixel_mask(V, H, W, tile, tile_mask))
    n = float(m.sum())
    if n == 0:
        raise ValueError("no pixel selected")
    l1 = (m[..., None] * (x - y).abs()).sum() / (3.0 * n)
    ss = (m[..., None] * ssim_map_torch(x, y)).sum() / (3.0 * n)
    L = (1.0 - lam) * l1 + lam * (1.0 - ss)
    f = None
    lf = torch.zeros((), dtype=torch.float64)
    if feat is not None:
        f = torch.tensor(np.asarray(feat, dtype=np.float64), requires_grad=True)
        ft = torch.tensor(np.asarray(feat_target, dtype=np.float64))
        Fd = f.shape[-1]
        lf = (m[..., None] * (f - ft).abs()).sum() / (Fd * n)
        L = L + lf
    L.backward()
    L = L.detach()
    parts = {"l1": float(l1.detach()), "ssim": float(ss.detach()), "l_feat": float(lf.detach()), "n": n}
    return float(L), parts, x.grad.numpy(), (None if f is None else f.grad.numpy())


def adam(param, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-15, log_param: bool = False, aux=None):
    """One Adam step in float64. Returns (param, m, v[, x]); with log_param, `param` holds log x,
    `grad` is dL/dx and `aux` is x (the chain dL/dlog x = dL/dx * x), and x = exp(param) is
    returned too."""
    p = np.asarray(param, dtype=np.float64).copy()
    g = np.asarray(grad, dtype=np.float64)
    if log_param:
        g = g * np.asarray(aux, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p = p - lr * mh / (np.sqrt(vh) + eps)
    if log_param:
        return p, m, v, np.exp(p)
    return p, m, v


def lr_of(group: str) -> float:
    """Learning rates of Sec. 4.1: 1e-2 for log-scales, 1e-4 for positions, 1e-3 otherwise."""
    return {"log_scales": 1e-2, "centers": 1e-4}.get(group, 1e-3)


__all__ = ["gaussian_window", "pixel_mask", "ssim_map_torch", "ssim_map_loops", "loss", "adam", "lr_of",
           "WINDOW", "SIGMA", "C1", "C2"]
