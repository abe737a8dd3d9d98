"""Training step around the renderer (Sec. 3.5, App. A.4).

One step renders a mini-batch of views, evaluates the photometric loss of Eq. 7 (and the feature
loss of Eq. 8 when the model has feature slots) on a seeded random fraction of the screen tiles
(the paper's tile mini-batching: four images per step, a quarter of each image's tiles), runs
the backward pass and takes one Adam step. The parameter groups and learning rates are those of
Sec. 4.1: log-scales 1e-2, positions 1e-4, everything else (MLP weights, slot embeddings,
quaternions) 1e-3. Every step of the loop is a kernel of the library (pack, render, loss,
backward, Adam); torch only holds the buffers.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import _lib
from .render import Renderer, _stream

LR = {"weights": 1e-3, "centers": 1e-4, "log_scales": 1e-2, "quats": 1e-3}


def tile_selection(n_views: int, height: int, width: int, tile: int, fraction: float, seed: int) -> np.ndarray:
    """uint8 [V, ceil(H/T), ceil(W/T)] with round(fraction x tiles) tiles per view set, drawn
    without replacement from a generator seeded with `seed`."""
    ntx, nty = (width + tile - 1) // tile, (height + tile - 1) // tile
    rng = np.random.RandomState(seed)
    mask = np.zeros((n_views, nty * ntx), np.uint8)
    k = max(1, int(round(fraction * nty * ntx)))
    for v in range(n_views):
        mask[v, rng.choice(nty * ntx, k, replace=False)] = 1
    return mask.reshape(n_views, nty, ntx)


class Trainer:
    """Parameters, Adam moments and workspaces of one scene; `step` runs one iteration."""

    def __init__(self, shape, scene: Dict[str, np.ndarray], precision: str = "fp32", lambda_ssim: float = 0.2,
                 tile: int = 8, tile_fraction: float = 0.25, lr: Optional[Dict[str, float]] = None,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15, device: str = "cuda",
                 seed: int = 0):
        self.r = Renderer(shape, precision=precision, device=device)
        self.device = self.r.device
        dev = self.device
        f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        self.params = {"weights": f32(scene["weights"]), "centers": f32(scene["centers"]),
                       "log_scales": f32(np.log(scene["scales"].astype(np.float64))),
                       "quats": f32(scene["quats"])}
        self.scales = torch.exp(self.params["log_scales"])  # kept equal to exp(log_scales) by Adam
        self.m = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.lr = dict(LR, **(lr or {}))
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        self.lambda_ssim, self.tile, self.tile_fraction, self.seed = lambda_ssim, tile, tile_fraction, seed
        self.F = self.r.F
        self.t = 0
        self.K = int(self.params["centers"].shape[0])
        self.packed = torch.empty(max(self.K, 1) * self.r.stride, dtype=torch.uint8, device=dev)
        self.loss_out = torch.zeros(5, device=dev)
        self._bufs = None
        self._mask_ring = None  # pinned staging buffers of the tile masks, with their copy events

    def tile_mask(self, step: int, n_views: int, height: int, width: int) -> np.ndarray:
        return tile_selection(n_views, height, width, self.tile, self.tile_fraction, self.seed * 1000003 + step)

    def _buffers(self, V: int, H: int, W: int):
        if self._bufs is None or self._bufs["key"] != (V, H, W):
            dev = self.device
            desc = _lib.loss_desc(V, H, W, self.tile, None, self.lambda_ssim, self.F)
            ws = _lib.mlps_loss_workspace_size(desc)
            ntx, nty = (W + self.tile - 1) // self.tile, (H + self.tile - 1) // self.tile
            self._bufs = {
                "key": (V, H, W),
                "out": {"rgb": torch.empty(V, H, W, 3, device=dev), "trans": torch.empty(V, H, W, device=dev),
                        "feat": torch.empty(V, H, W, self.F, device=dev) if self.F else None},
                "d_rgb": torch.empty(V, H, W, 3, device=dev),
                "d_feat": torch.empty(V, H, W, self.F, device=dev) if self.F else None,
                "grads": {"d_weights": torch.empty_like(self.params["weights"]),
                          "d_centers": torch.empty_like(self.params["centers"]),
                          "d_scales": torch.empty_like(self.params["log_scales"]),
                          "d_quats": torch.empty_like(self.params["quats"])},
                "mask": torch.empty(V, nty, ntx, dtype=torch.uint8, device=dev),
                "ws": torch.empty(ws, dtype=torch.uint8, device=dev),
            }
        return self._bufs

    def step(self, cams: Sequence[dict], rgb_target: torch.Tensor, feat_target: Optional[torch.Tensor] = None,
             tile_mask: Optional[np.ndarray] = None) -> torch.Tensor:
        """One iteration on views `cams` (same size) against the device targets; returns the
        device tensor {L, L1, SSIM, N, L_f} of this step's loss (before the update)."""
        V, H, W = len(cams), int(cams[0]["height"]), int(cams[0]["width"])
        b = self._buffers(V, H, W)
        self.t += 1
        mask = self.tile_mask(self.t, V, H, W) if tile_mask is None else tile_mask
        self._upload_mask(b["mask"], mask)
        p = self.params
        self.r.pack(p["weights"], out=self.packed)
        out = self.r.forward(p["centers"], self.scales, p["quats"], self.packed, cams, out=b["out"])
        desc = _lib.loss_desc(V, H, W, self.tile, b["mask"], self.lambda_ssim, self.F)
        _lib.mlps_loss(desc, out["rgb"], rgb_target.contiguous(), out.get("feat"),
                       None if feat_target is None else feat_target.contiguous(), b["d_rgb"], b["d_feat"],
                       self.loss_out, b["ws"], b["ws"].numel(), _stream())
        g = self.r.backward(b["d_rgb"], None, b["d_feat"], out=b["grads"])
        groups = [
            _lib.adam_group(p["weights"], g["d_weights"], self.m["weights"], self.v["weights"], self.lr["weights"]),
            _lib.adam_group(p["centers"], g["d_centers"], self.m["centers"], self.v["centers"], self.lr["centers"]),
            _lib.adam_group(p["log_scales"], g["d_scales"], self.m["log_scales"], self.v["log_scales"],
                            self.lr["log_scales"], aux=self.scales, kind=1),
            _lib.adam_group(p["quats"], g["d_quats"], self.m["quats"], self.v["quats"], self.lr["quats"]),
        ]
        _lib.mlps_adam_step(groups, self.beta1, self.beta2, self.eps, self.t, _stream())
        return self.loss_out

    def _upload_mask(self, dst: torch.Tensor, mask: np.ndarray):
        """Stream-ordered upload through a ring of two pinned buffers: the host never waits for
        the GPU except to reuse a buffer whose copy (two steps back) is still in flight."""
        if self._mask_ring is None or self._mask_ring[0][0].shape != dst.shape:
            self._mask_ring = [(torch.empty(dst.shape, dtype=torch.uint8).pin_memory(), torch.cuda.Event())
                               for _ in range(2)]
        buf, ev = self._mask_ring[self.t % 2]
        ev.synchronize()
        buf.numpy()[...] = mask
        dst.copy_(buf, non_blocking=True)
        ev.record()

    def status(self) -> int:
        return self.r.status()
