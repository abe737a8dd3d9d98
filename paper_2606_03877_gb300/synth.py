"""Seeded synthetic inputs: scenes of MLP primitives, pinhole cameras and loss gradients.

This module holds no rendering arithmetic. It only draws the inputs that both the CUDA path
and the FP64 oracle consume, so that every parity test feeds the two sides bit-identical
arrays.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used as a hash of
(seed, stream, counter). Output ``i`` of a stream is ``mix(key + (i + 1) * GAMMA)``; the key
is ``mix(seed * GAMMA2 + stream)``. Uniforms take the top 53 bits; normals use Box-Muller.
Everything is plain uint64 / float64 numpy, so a given (seed, stream, counter) gives the same
value on every platform up to libm's last-bit behaviour in log/cos.

Scene distributions (the paper's Replica/ScanNet scenes are not available; these synthetic
scenes stand in for them):

* centres  ~ U[-1, 1]^3
* scales   ~ log-U[0.05, 0.4] per axis (linear scale, > 0)
* quats    ~ uniform on S^3 (normalised 4-D Gaussian), stored (w, x, y, z)
* MLP      ~ Kaiming-uniform U(+-sqrt(6 / fan_in)) weights, zero biases, except the density
             output's bias, which starts at +1
* cameras  ~ on the sphere of radius 3 around the origin, looking at the origin, vertical FOV
             50 degrees, principal point at the image centre, OpenCV axes (x right, y down,
             z forward), world up +z (fallback +y when looking along z)

Weight layout (the "canonical FP32 layout", one row of ``[K, P]`` per primitive): for each
layer ``l`` in order, ``W_l`` as ``[out_l, in_l]`` row-major, then ``b_l`` as ``[out_l]``.
Layer 0 reads the encoded input; hidden layers have ``hidden_width`` outputs with ReLU; the
last layer has ``4 + feat_dim`` linear outputs ordered (r, g, b, sigma, f_0, ...).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_GAMMA2 = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# One stream id per drawn tensor.
STREAM_CENTERS = 1
STREAM_SCALES = 2
STREAM_QUATS = 3
STREAM_WEIGHTS = 4
STREAM_CAMERA = 5
STREAM_PERTURB = 6
STREAM_GRAD = 7
STREAM_BATCH = 8
STREAM_SLOTS = 9


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GAMMA2 + np.uint64(stream)
    return _mix(np.array([k], dtype=np.uint64))[0]


def bits(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit outputs ``offset .. offset + n - 1`` of stream ``(seed, stream)``."""
    key = _key(seed, stream)
    ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + ctr * _GAMMA)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 in [0, 1) from the top 53 bits."""
    b = bits(seed, stream, n, offset)
    return (b >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller; output ``i`` uses uniforms ``2i`` and ``2i + 1``."""
    u = uniform(seed, stream, 2 * n, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclasses.dataclass(frozen=True)
class SceneConfig:
    """Shape of one workload: image size, primitive count and per-primitive MLP."""

    name: str
    width: int
    height: int
    K: int
    n_views: int
    xyz_freqs: int  # 0: raw local xyz (3 inputs)
    dir_freqs: int  # 0: no view-direction input
    hidden_width: int
    hidden_layers: int
    feat_dim: int
    samples: int  # S midpoint samples per hit interval
    precision: str = "fp32"
    contact: int = 0  # 1: contact-point input gamma([d; mu - p*]), one sample per hit (S = 1)
    slot_dim: int = 0  # C of the four slot embeddings per primitive (feature slots); 0 = none
    tile_sort: int = 0  # T > 0: hits ordered by the tile-centre ray of T x T tiles; 0 = per ray

    @property
    def input_dim(self) -> int:
        nx = 6 * self.xyz_freqs if self.xyz_freqs > 0 else 3
        nd = 6 * self.dir_freqs if self.dir_freqs > 0 else 0
        return nx + nd

    @property
    def output_dim(self) -> int:
        return 4 + self.feat_dim

    def layer_dims(self) -> List[tuple]:
        dims = [self.input_dim] + [self.hidden_width] * self.hidden_layers + [self.output_dim]
        return [(dims[i], dims[i + 1]) for i in range(len(dims) - 1)]

    @property
    def n_mlp_params(self) -> int:
        return sum(i * o + o for i, o in self.layer_dims())

    @property
    def n_params(self) -> int:
        """Parameters per primitive: the MLP's, then the four slot embeddings."""
        return self.n_mlp_params + 4 * self.slot_dim

    @property
    def n_rays(self) -> int:
        return self.width * self.height * self.n_views

    def replace(self, **kw) -> "SceneConfig":
        return dataclasses.replace(self, **kw)


# The five seeded workloads. "prec" is the 1080p headline configuration.
CONFIGS: Dict[str, SceneConfig] = {
    "pr1": SceneConfig("pr1", 64, 64, 8, 1, 0, 0, 32, 2, 0, 16, "fp32"),
    "diff": SceneConfig("diff", 800, 800, 64, 1, 6, 4, 64, 3, 0, 32, "fp32"),
    "prec": SceneConfig("prec", 1920, 1080, 256, 8, 6, 4, 64, 3, 0, 32, "bf16"),
    "stress": SceneConfig("stress", 1920, 1080, 1024, 4, 6, 4, 128, 4, 16, 48, "fp8"),
    # the paper's own per-primitive model: gamma([d; delta]) with L = 6 (72 inputs), 32 x 2, S = 1,
    # on the views and primitives of the precision workload
    "contact": SceneConfig("contact", 1920, 1080, 256, 8, 6, 6, 32, 2, 0, 1, "fp32", 1),
    # the paper's model with its semantic feature slots: four 512-d embeddings per primitive,
    # 1080p x 2 views (a 512-channel FP32 feature map is 2 KB per pixel)
    "slots": SceneConfig("slots", 1920, 1080, 256, 2, 6, 6, 32, 2, 0, 1, "fp32", 1, 512),
    # training: the same model, four views per step at the Replica resolution (1200 x 680)
    "train": SceneConfig("train", 1200, 680, 256, 4, 6, 6, 32, 2, 0, 1, "fp32", 1, 512),
}

# Batched workload: 32 scenes, K ~ U{16..512}, resolution uniform over these four.
BATCH_RESOLUTIONS = [(256, 256), (512, 512), (800, 800), (1920, 1080)]
BATCH_SCENES = 32


def batch_configs(n_scenes: int = BATCH_SCENES, seed: int = 0) -> List[SceneConfig]:
    u = uniform(seed, STREAM_BATCH, 2 * n_scenes)
    out = []
    for i in range(n_scenes):
        K = 16 + int(u[2 * i] * (512 - 16 + 1))
        w, h = BATCH_RESOLUTIONS[int(u[2 * i + 1] * len(BATCH_RESOLUTIONS))]
        out.append(SceneConfig(f"batch{i}", w, h, K, 1, 6, 4, 64, 3, 0, 32, "bf16"))
    return out


def make_batch(cfgs: Sequence[SceneConfig], first_seed: int = 0):
    """A batch of independent scenes: scene i (seed first_seed + i) seen by one camera (view
    seed first_seed + i) at cfgs[i]'s resolution. Returns (scene arrays of all scenes
    concatenated, items as (prim_offset, prim_count, camera), per-scene scenes). All scenes must
    share the MLP shape."""
    scenes, items, off = [], [], 0
    for i, c in enumerate(cfgs):
        sc = make_scene(c, first_seed + i)
        scenes.append(sc)
        items.append((off, c.K, make_camera(c.width, c.height, first_seed + i)))
        off += c.K
    cat = {k: np.concatenate([sc[k] for sc in scenes], axis=0) for k in scenes[0]}
    return cat, items, scenes


def make_scene(cfg: SceneConfig, seed: int = 0) -> Dict[str, np.ndarray]:
    """Primitive poses and canonical-layout FP32 weights for ``cfg`` from ``seed``."""
    K = cfg.K
    centers = (2.0 * uniform(seed, STREAM_CENTERS, 3 * K) - 1.0).reshape(K, 3)
    lo, hi = math.log(0.05), math.log(0.4)
    scales = np.exp(lo + (hi - lo) * uniform(seed, STREAM_SCALES, 3 * K)).reshape(K, 3)
    q = normal(seed, STREAM_QUATS, 4 * K).reshape(K, 4)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    weights = np.zeros((K, cfg.n_params), dtype=np.float64)
    u = uniform(seed, STREAM_WEIGHTS, K * cfg.n_mlp_params).reshape(K, cfg.n_mlp_params)
    off = 0
    dims = cfg.layer_dims()
    for li, (fi, fo) in enumerate(dims):
        bound = math.sqrt(6.0 / fi)
        nw = fi * fo
        weights[:, off:off + nw] = (2.0 * u[:, off:off + nw] - 1.0) * bound
        off += nw
        if li == len(dims) - 1:
            weights[:, off + 3] = 1.0  # density output bias starts at +1
        off += fo
    if cfg.slot_dim:  # slot embeddings U(-1, 1)
        weights[:, off:] = 2.0 * uniform(seed, STREAM_SLOTS, K * 4 * cfg.slot_dim).reshape(K, -1) - 1.0
    return {
        "centers": centers.astype(np.float32),
        "scales": scales.astype(np.float32),
        "quats": q.astype(np.float32),
        "weights": weights.astype(np.float32),
    }


def perturb_scene(scene: Dict[str, np.ndarray], cfg: SceneConfig, seed: int = 1) -> Dict[str, np.ndarray]:
    """Copy of ``scene`` with Gaussian noise from ``seed``: centres 0.02, log-scales 0.05,
    quaternions 0.05 (renormalised), weights 0.05 x the layer's init bound."""
    K = cfg.K
    n = normal(seed, STREAM_PERTURB, 3 * K + 3 * K + 4 * K + K * cfg.n_params)
    o = 0
    c = scene["centers"].astype(np.float64) + 0.02 * n[o:o + 3 * K].reshape(K, 3); o += 3 * K
    s = np.exp(np.log(scene["scales"].astype(np.float64)) + 0.05 * n[o:o + 3 * K].reshape(K, 3)); o += 3 * K
    q = scene["quats"].astype(np.float64) + 0.05 * n[o:o + 4 * K].reshape(K, 4); o += 4 * K
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w = scene["weights"].astype(np.float64).copy()
    noise = n[o:o + K * cfg.n_params].reshape(K, cfg.n_params)
    off = 0
    for fi, fo in cfg.layer_dims():
        bound = math.sqrt(6.0 / fi)
        w[:, off:off + fi * fo + fo] += 0.05 * bound * noise[:, off:off + fi * fo + fo]
        off += fi * fo + fo
    w[:, off:] += 0.05 * noise[:, off:]  # slot embeddings
    return {
        "centers": c.astype(np.float32),
        "scales": s.astype(np.float32),
        "quats": q.astype(np.float32),
        "weights": w.astype(np.float32),
    }


def make_camera(width: int, height: int, view_seed: int, radius: float = 3.0,
                fov_deg: float = 50.0, near: float = 0.0) -> Dict[str, object]:
    """Pinhole camera on the sphere of ``radius`` looking at the origin.

    Returns FP32-representable values: ``w2c`` is the row-major 3x4 [R | t] world-to-camera
    transform with rows (right, down, forward)."""
    g = normal(view_seed, STREAM_CAMERA, 3)
    u = g / np.linalg.norm(g)
    pos = radius * u
    fwd = -u
    up = np.array([0.0, 0.0, 1.0])
    if abs(float(fwd @ up)) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ pos
    w2c = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    f = (height / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return {
        "width": int(width),
        "height": int(height),
        "fx": float(np.float32(f)),
        "fy": float(np.float32(f)),
        "cx": float(np.float32(width / 2.0)),
        "cy": float(np.float32(height / 2.0)),
        "w2c": w2c.reshape(12),
        "near": float(np.float32(near)),
    }


def make_cameras(cfg: SceneConfig, first_view_seed: int = 0) -> List[Dict[str, object]]:
    return [make_camera(cfg.width, cfg.height, first_view_seed + v) for v in range(cfg.n_views)]


def make_grad(shape, seed: int = 0, scale: float = 1.0, offset: int = 0) -> np.ndarray:
    """Seeded N(0, scale^2) loss gradient (e.g. dL/dC of shape [V, H, W, 3]) as FP32."""
    n = int(np.prod(shape))
    return (scale * normal(seed, STREAM_GRAD, n, offset)).reshape(shape).astype(np.float32)


def sample_pixels(cfg: SceneConfig, n: int, seed: int = 0) -> np.ndarray:
    """``n`` distinct pixels as int32 triples (view, x, y), sorted by global ray index."""
    total = cfg.n_rays
    n = min(n, total)
    b = (bits(seed, STREAM_GRAD + 100, 4 * n) % np.uint64(total)).astype(np.int64)
    _, first = np.unique(b, return_index=True)  # distinct values, kept in draw order
    idx = np.sort(b[np.sort(first)][:n])
    hw = cfg.width * cfg.height
    v = idx // hw
    r = idx % hw
    return np.stack([v, r % cfg.width, r // cfg.width], axis=1).astype(np.int32)
