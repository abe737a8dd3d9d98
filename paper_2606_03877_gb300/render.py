"""Torch-facing wrapper of the CUDA renderer: workspaces, weight packing and autograd.

PyTorch supplies device memory and the stream only; every step of the render runs in
``libmlps.so`` through :mod:`paper_2606_03877_gb300._lib`.
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional, Sequence

import torch

from . import _lib


def make_config(shape, precision: str = "fp32", t_eps: float = 1e-6, max_hits: int = 64,
                hit_capacity: float = 8.0, tile: int = 16, mlp_groups: int = 0,
                early_stop_wave: int = 0) -> _lib.MlpsConfig:
    """mlps_config from any object with xyz_freqs, dir_freqs, hidden_width, hidden_layers,
    feat_dim, samples and optionally contact and slot_dim (e.g. :class:`synth.SceneConfig`)."""
    cfg = _lib.mlps_config_default(int(shape.xyz_freqs), int(shape.dir_freqs), int(shape.hidden_width),
                                   int(shape.hidden_layers), int(shape.feat_dim))
    cfg.samples = int(shape.samples)
    cfg.precision = _lib.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.t_eps = float(t_eps)
    cfg.max_hits_per_ray = int(max_hits)
    cfg.hit_capacity_per_ray = float(hit_capacity)
    cfg.tile = int(tile)
    cfg.mlp_groups = int(mlp_groups)
    cfg.early_stop_wave = int(early_stop_wave)
    cfg.contact = int(getattr(shape, "contact", 0))
    cfg.slot_dim = int(getattr(shape, "slot_dim", 0))
    T = int(getattr(shape, "tile_sort", 0))  # tile-centre order of T x T tiles (T = 8 or 16)
    if T:
        cfg.tile_sort = 1
        cfg.tile = T
    return cfg


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Renderer:
    """One configuration with reusable saved/scratch workspaces (grown on demand)."""

    def __init__(self, shape, precision: str = "fp32", device: str = "cuda", **kw):
        self.shape = shape
        self.precision = precision
        self.cfg = make_config(shape, precision, **kw)
        st = _lib.mlps_check_config(self.cfg)
        if st != _lib.MLPS_OK:
            raise _lib.MlpsError("mlps_check_config", st)
        self.device = torch.device(device)
        self.P = _lib.mlps_param_count(self.cfg)
        self.stride = _lib.mlps_weight_stride(self.cfg)
        # feature row: the MLP's extra outputs, then the slot channels
        self.F = int(shape.feat_dim) + int(getattr(shape, "slot_dim", 0))
        self.saved: Optional[torch.Tensor] = None
        self.scratch: Optional[torch.Tensor] = None
        self._last = None

    # -- weights -------------------------------------------------------------------------
    def pack(self, weights: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        w = weights.detach().to(self.device, torch.float32).contiguous()
        K = w.shape[0]
        assert w.shape[1] == self.P, (w.shape, self.P)
        if out is None:
            out = torch.empty(max(K, 1) * self.stride, dtype=torch.uint8, device=self.device)
        _lib.mlps_pack_weights(self.cfg, K, w, out, _stream())
        return out

    # -- workspaces ------------------------------------------------------------------------
    def workspace_bytes(self, K: int, cams: Sequence[dict]):
        cs = _lib.cameras(cams)
        return _lib.mlps_workspace_size(self.cfg, K, cs, len(cams))

    def _ensure(self, K: int, cs, V: int):
        sb, tb = _lib.mlps_workspace_size(self.cfg, K, cs, V)
        if self.saved is None or self.saved.numel() < sb:
            self.saved = torch.empty(sb, dtype=torch.uint8, device=self.device)
        if self.scratch is None or self.scratch.numel() < tb:
            self.scratch = torch.empty(tb, dtype=torch.uint8, device=self.device)

    # -- passes ----------------------------------------------------------------------------
    def forward(self, centers, scales, quats, packed, cams: Sequence[dict],
                out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
        cs = _lib.cameras(cams)
        V = len(cams)
        H, W = int(cams[0]["height"]), int(cams[0]["width"])
        K = int(centers.shape[0])
        self._ensure(K, cs, V)
        if out is None:
            out = {"rgb": torch.empty(V, H, W, 3, device=self.device),
                   "trans": torch.empty(V, H, W, device=self.device),
                   "feat": torch.empty(V, H, W, self.F, device=self.device) if self.F else None}
        scene = _lib.make_scene(K, centers, scales, quats, packed)
        _lib.mlps_render_forward(self.cfg, scene, cs, V, out["rgb"], out["trans"], out.get("feat"),
                                 self.saved, self.saved.numel(), self.scratch, self.scratch.numel(),
                                 _stream())
        self._last = (scene, cs, V, K, (centers, scales, quats, packed))
        return out

    def backward(self, d_rgb, d_trans=None, d_feat=None,
                 out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
        scene, cs, V, K, _keep = self._last
        if out is None:
            out = {"d_weights": torch.empty(K, self.P, device=self.device),
                   "d_centers": torch.empty(K, 3, device=self.device),
                   "d_scales": torch.empty(K, 3, device=self.device),
                   "d_quats": torch.empty(K, 4, device=self.device)}
        _lib.mlps_render_backward(self.cfg, scene, cs, V, d_rgb.contiguous(),
                                  None if d_trans is None else d_trans.contiguous(),
                                  None if d_feat is None else d_feat.contiguous(),
                                  self.saved, self.saved.numel(), out["d_weights"], out["d_centers"],
                                  out["d_scales"], out["d_quats"], self.scratch, self.scratch.numel(),
                                  _stream())
        return out

    def status(self, region: str = "saved") -> int:
        t = self.saved if region == "saved" else self.scratch
        return _lib.mlps_read_status(t, _stream())

    def hit_count(self) -> int:
        return _lib.mlps_saved_hit_count(self.saved, _stream())

    def wave_counts(self):
        """(hit intervals of the last forward pass, intervals its depth waves evaluated)."""
        return _lib.mlps_forward_wave_counts(self.saved, self.scratch, _stream())

    def chunk_counts(self):
        """(MLP chunks of the last forward pass, chunks its last backward pass walked)."""
        return _lib.mlps_backward_chunk_counts(self.saved, self.scratch, _stream())

    def hits(self, max_out: int = 64):
        _, cs, V, K, _ = self._last
        n_rays = V * cs[0].width * cs[0].height
        dev = self.device
        count = torch.empty(n_rays, dtype=torch.int32, device=dev)
        prim = torch.full((n_rays, max_out), -1, dtype=torch.int32, device=dev)
        t0 = torch.zeros(n_rays, max_out, device=dev)
        t1 = torch.zeros(n_rays, max_out, device=dev)
        tm = torch.zeros(n_rays, max_out, device=dev)
        _lib.mlps_export_hits(self.cfg, cs, V, self.saved, max_out, count, prim, t0, t1, tm, _stream())
        return {"count": count, "prim": prim, "t0": t0, "t1": t1, "tmid": tm}

    def tiles(self):
        _, cs, V, K, _ = self._last
        t = int(self.cfg.tile)
        nt = ((cs[0].width + t - 1) // t) * ((cs[0].height + t - 1) // t)
        count = torch.empty(V * nt, dtype=torch.int32, device=self.device)
        lst = torch.empty(V * nt * K, dtype=torch.int32, device=self.device)
        _lib.mlps_export_tiles(self.cfg, K, cs, V, self.scratch, count, lst, _stream())
        return count, lst.view(V * nt, K)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer: Renderer, cams, centers, scales, quats, weights):
        packed = renderer.pack(weights)
        out = renderer.forward(centers.detach().contiguous(), scales.detach().contiguous(),
                               quats.detach().contiguous(), packed, cams)
        ctx.renderer = renderer
        ctx.keep = packed
        ctx.mark_non_differentiable(*([] if out["feat"] is None else []))
        feat = out["feat"] if out["feat"] is not None else torch.empty(0, device=centers.device)
        return out["rgb"], out["trans"], feat

    @staticmethod
    def backward(ctx, g_rgb, g_trans, g_feat):
        r: Renderer = ctx.renderer
        g = r.backward(g_rgb, g_trans, g_feat if r.F else None)
        return None, None, g["d_centers"], g["d_scales"], g["d_quats"], g["d_weights"]


def render(renderer: Renderer, cams: Sequence[dict], centers: torch.Tensor, scales: torch.Tensor,
           quats: torch.Tensor, weights: torch.Tensor):
    """Differentiable render: returns (rgb [V,H,W,3], trans [V,H,W], feat [V,H,W,F] or empty).

    One forward pass per call; the backward pass of the same renderer must follow before the
    next forward on it (the forward state lives in the renderer's workspace)."""
    return _RenderFn.apply(renderer, cams, centers, scales, quats, weights)


class BatchRenderer:
    """Many scenes of uneven primitive counts and resolutions in one call (mlps_render_batch_*).

    ``items`` are (prim_offset, prim_count, camera) tuples over ONE concatenated set of scene
    arrays with ``K`` primitives in total; item i renders its primitive range through its camera at
    the camera's own resolution. Outputs are concatenated in item order (``split`` gives per-item
    views). Workspaces are allocated here, once, so forward/backward can be captured in a CUDA
    graph and replayed."""

    def __init__(self, shape, items: Sequence[tuple], K: int, precision: str = "bf16",
                 device: str = "cuda", **kw):
        self.shape = shape
        self.precision = precision
        self.cfg = make_config(shape, precision, **kw)
        st = _lib.mlps_check_config(self.cfg)
        if st != _lib.MLPS_OK:
            raise _lib.MlpsError("mlps_check_config", st)
        self.device = torch.device(device)
        self.P = _lib.mlps_param_count(self.cfg)
        self.stride = _lib.mlps_weight_stride(self.cfg)
        # feature row: the MLP's extra outputs, then the slot channels
        self.F = int(shape.feat_dim) + int(getattr(shape, "slot_dim", 0))
        self.K = int(K)
        self.items = _lib.batch_items(items)
        self.n = len(items)
        self.sizes = [(int(c["height"]), int(c["width"])) for _, _, c in items]
        self.offsets = [0]
        for h, w in self.sizes:
            self.offsets.append(self.offsets[-1] + h * w)
        self.n_pixels = self.offsets[-1]
        # workspaces large enough for either tile edge, so the autotuner can try both
        sizes = []
        for t in (16, 8):
            c = make_config(shape, precision, **dict(kw, tile=t))
            sizes.append(_lib.mlps_batch_workspace_size(c, self.K, self.items, self.n))
        sb = max(x[0] for x in sizes)
        tb = max(x[1] for x in sizes)
        self.saved = torch.empty(sb, dtype=torch.uint8, device=self.device)
        self.scratch = torch.empty(tb, dtype=torch.uint8, device=self.device)
        self._scene = None
        self.tuning = None

    def autotune(self, centers, scales, quats, packed, d_rgb=None, reps: int = 3):
        """Pick tile edge and samples per CTA for this batch (mlps_autotune_batch) and use them
        from now on. Times the forward pass, or forward + backward when d_rgb is given.
        Synchronises; call it before capturing a graph."""
        out = self.new_outputs()
        grads = self.new_grads()
        scene = _lib.make_scene(self.K, centers, scales, quats, packed)
        tuned, best, cands = _lib.mlps_autotune_batch(
            self.cfg, scene, self.items, self.n, 1 if d_rgb is not None else 0,
            None if d_rgb is None else d_rgb.contiguous(), out["rgb"], out["trans"], out.get("feat"),
            self.saved, self.saved.numel(), self.scratch, self.scratch.numel(), grads["d_weights"],
            grads["d_centers"], grads["d_scales"], grads["d_quats"], reps, _stream())
        self.cfg = tuned
        self.tuning = {"tile": int(tuned.tile), "mlp_groups": int(tuned.mlp_groups), "best_ms": best,
                       "candidates": cands}
        return self.tuning

    def pack(self, weights: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        w = weights.detach().to(self.device, torch.float32).contiguous()
        assert w.shape == (self.K, self.P), (w.shape, self.K, self.P)
        if out is None:
            out = torch.empty(max(self.K, 1) * self.stride, dtype=torch.uint8, device=self.device)
        _lib.mlps_pack_weights(self.cfg, self.K, w, out, _stream())
        return out

    def new_outputs(self) -> Dict[str, torch.Tensor]:
        P, dev = self.n_pixels, self.device
        return {"rgb": torch.empty(P, 3, device=dev), "trans": torch.empty(P, device=dev),
                "feat": torch.empty(P, self.F, device=dev) if self.F else None}

    def new_grads(self) -> Dict[str, torch.Tensor]:
        K, dev = self.K, self.device
        return {"d_weights": torch.empty(K, self.P, device=dev), "d_centers": torch.empty(K, 3, device=dev),
                "d_scales": torch.empty(K, 3, device=dev), "d_quats": torch.empty(K, 4, device=dev)}

    def forward(self, centers, scales, quats, packed, out: Optional[Dict[str, torch.Tensor]] = None):
        if out is None:
            out = self.new_outputs()
        self._scene = _lib.make_scene(self.K, centers, scales, quats, packed)
        self._keep = (centers, scales, quats, packed)
        _lib.mlps_render_batch_forward(self.cfg, self._scene, self.items, self.n, out["rgb"], out["trans"],
                                       out.get("feat"), self.saved, self.saved.numel(), self.scratch,
                                       self.scratch.numel(), _stream())
        return out

    def backward(self, d_rgb, d_trans=None, d_feat=None, out: Optional[Dict[str, torch.Tensor]] = None):
        if out is None:
            out = self.new_grads()
        _lib.mlps_render_batch_backward(self.cfg, self._scene, self.items, self.n, d_rgb.contiguous(),
                                        None if d_trans is None else d_trans.contiguous(),
                                        None if d_feat is None else d_feat.contiguous(),
                                        self.saved, self.saved.numel(), out["d_weights"], out["d_centers"],
                                        out["d_scales"], out["d_quats"], self.scratch, self.scratch.numel(),
                                        _stream())
        return out

    def split(self, t: torch.Tensor) -> List[torch.Tensor]:
        """Per-item [H_i, W_i, ...] views of a concatenated per-pixel tensor."""
        return [t[self.offsets[i]:self.offsets[i + 1]].view(h, w, *t.shape[1:])
                for i, (h, w) in enumerate(self.sizes)]

    def status(self, region: str = "saved") -> int:
        t = self.saved if region == "saved" else self.scratch
        return _lib.mlps_read_status(t, _stream())


class DeviceBatchRenderer:
    """A batch whose item table lives in device memory (mlps_render_batch_*_dev).

    ``n`` items of at most ``max_width`` x ``max_height`` pixels and ``max_prims`` primitives each,
    over ONE concatenated set of scene arrays with ``K`` primitives. The item table is a device
    tensor written by ``set_items`` (an ordinary stream copy), so a CUDA graph captured around
    ``forward`` / ``backward`` renders whatever items the table holds at replay time. Outputs are
    sized for the caps; items are concatenated at their actual sizes (``split``)."""

    def __init__(self, shape, n: int, max_width: int, max_height: int, max_prims: int, K: int,
                 precision: str = "bf16", device: str = "cuda", **kw):
        self.shape = shape
        self.precision = precision
        self.cfg = make_config(shape, precision, **kw)
        st = _lib.mlps_check_config(self.cfg)
        if st != _lib.MLPS_OK:
            raise _lib.MlpsError("mlps_check_config", st)
        self.device = torch.device(device)
        self.P = _lib.mlps_param_count(self.cfg)
        self.stride = _lib.mlps_weight_stride(self.cfg)
        self.F = int(shape.feat_dim) + int(getattr(shape, "slot_dim", 0))
        self.K = int(K)
        self.n = int(n)
        self.caps = _lib.batch_caps(max_width, max_height, max_prims)
        self.cap_pixels = self.n * int(max_width) * int(max_height)
        sb, tb = _lib.mlps_batch_workspace_size_dev(self.cfg, self.K, self.n, self.caps)
        self.saved = torch.empty(sb, dtype=torch.uint8, device=self.device)
        self.scratch = torch.empty(tb, dtype=torch.uint8, device=self.device)
        self.item_bytes = ctypes.sizeof(_lib.MlpsBatchItem)
        self.items_dev = torch.zeros(self.n * self.item_bytes, dtype=torch.uint8, device=self.device)
        self.sizes = []
        self._scene = None

    def set_items(self, items: Sequence[tuple]):
        """Write (prim_offset, prim_count, camera) tuples into the device table (stream-ordered)."""
        assert len(items) == self.n
        arr = _lib.batch_items(items)
        host = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
        self.items_dev.copy_(host.to(self.device))
        self.sizes = [(int(c["height"]), int(c["width"])) for _, _, c in items]

    def pack(self, weights: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        w = weights.detach().to(self.device, torch.float32).contiguous()
        assert w.shape == (self.K, self.P), (w.shape, self.K, self.P)
        if out is None:
            out = torch.empty(max(self.K, 1) * self.stride, dtype=torch.uint8, device=self.device)
        _lib.mlps_pack_weights(self.cfg, self.K, w, out, _stream())
        return out

    def new_outputs(self) -> Dict[str, torch.Tensor]:
        P, dev = self.cap_pixels, self.device
        return {"rgb": torch.zeros(P, 3, device=dev), "trans": torch.zeros(P, device=dev),
                "feat": torch.zeros(P, self.F, device=dev) if self.F else None}

    def new_grads(self) -> Dict[str, torch.Tensor]:
        K, dev = self.K, self.device
        return {"d_weights": torch.empty(K, self.P, device=dev), "d_centers": torch.empty(K, 3, device=dev),
                "d_scales": torch.empty(K, 3, device=dev), "d_quats": torch.empty(K, 4, device=dev)}

    def forward(self, centers, scales, quats, packed, out: Optional[Dict[str, torch.Tensor]] = None):
        if out is None:
            out = self.new_outputs()
        self._scene = _lib.make_scene(self.K, centers, scales, quats, packed)
        self._keep = (centers, scales, quats, packed)
        _lib.mlps_render_batch_forward_dev(self.cfg, self._scene, self.items_dev, self.n, self.caps, out["rgb"],
                                           out["trans"], out.get("feat"), self.saved, self.saved.numel(),
                                           self.scratch, self.scratch.numel(), _stream())
        return out

    def backward(self, d_rgb, d_trans=None, d_feat=None, out: Optional[Dict[str, torch.Tensor]] = None):
        if out is None:
            out = self.new_grads()
        _lib.mlps_render_batch_backward_dev(self.cfg, self._scene, self.items_dev, self.n, self.caps,
                                            d_rgb.contiguous(), None if d_trans is None else d_trans.contiguous(),
                                            None if d_feat is None else d_feat.contiguous(), self.saved,
                                            self.saved.numel(), out["d_weights"], out["d_centers"],
                                            out["d_scales"], out["d_quats"], self.scratch, self.scratch.numel(),
                                            _stream())
        return out

    def split(self, t: torch.Tensor) -> List[torch.Tensor]:
        """Per-item [H_i, W_i, ...] views (sizes of the last set_items) of a per-pixel tensor."""
        outs, o = [], 0
        for h, w in self.sizes:
            outs.append(t[o:o + h * w].view(h, w, *t.shape[1:]))
            o += h * w
        return outs

    def status(self, region: str = "saved") -> int:
        t = self.saved if region == "saved" else self.scratch
        return _lib.mlps_read_status(t, _stream())
