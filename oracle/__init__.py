"""Python binding of the FP64 CPU oracle (``mlps_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the benchmark's
CPU-baseline leg are the only callers. The CUDA library and its Python binding never import
this package, and this package imports nothing from them: configs are taken by duck typing
(any object with ``xyz_freqs, dir_freqs, hidden_width, hidden_layers, feat_dim, samples`` and
optional ``contact``, ``slot_dim`` and ``tile_sort``) and
scenes / cameras as plain numpy arrays and dicts.

All inputs are converted to float64 before the call; outputs are float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlps_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmlps_oracle.so")
_lock = threading.Lock()
_lib = None


class _Cfg(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("xyz_freqs", "dir_freqs", "hidden_width", "hidden_layers", "feat_dim", "samples",
                 "contact", "slot_dim", "tile_sort")]


class _Cam(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("w2c", ctypes.c_double * 12), ("near_t", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, IEEE semantics kept)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            d = P(ctypes.c_double)
            i = P(ctypes.c_int)
            lib.orc_input_dim.argtypes = [P(_Cfg)]
            lib.orc_param_count.argtypes = [P(_Cfg)]
            lib.orc_param_count.restype = ctypes.c_long
            lib.orc_render.argtypes = [P(_Cfg), ctypes.c_int, d, d, d, d, ctypes.c_int, P(_Cam),
                                       ctypes.c_int, i, d, d, d, ctypes.c_int]
            lib.orc_render_backward.argtypes = [P(_Cfg), ctypes.c_int, d, d, d, d, ctypes.c_int,
                                                P(_Cam), ctypes.c_int, i, d, d, d, d, d, d, d, d,
                                                d, d, ctypes.c_int]
            lib.orc_ray_hits.argtypes = [ctypes.c_int, d, d, d, P(_Cam), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, i, d, d, d, d]
            lib.orc_ray_m2.argtypes = [ctypes.c_int, d, d, d, P(_Cam), ctypes.c_int, ctypes.c_int, d, d]
            lib.orc_pixel_ray.argtypes = [P(_Cam), ctypes.c_int, ctypes.c_int, d, d]
            lib.orc_encode.argtypes = [P(_Cfg), d, d, d]
            lib.orc_mlp.argtypes = [P(_Cfg), d, d, d]
            lib.orc_slot_weights.argtypes = [d, d]
            _lib = lib
    return _lib


def _cfg(c) -> _Cfg:
    return _Cfg(int(c.xyz_freqs), int(c.dir_freqs), int(c.hidden_width), int(c.hidden_layers),
                int(c.feat_dim), int(c.samples), int(getattr(c, "contact", 0)),
                int(getattr(c, "slot_dim", 0)), int(getattr(c, "tile_sort", 0)))


def _cam(c: Dict) -> _Cam:
    w2c = (ctypes.c_double * 12)(*[float(v) for v in np.asarray(c["w2c"], dtype=np.float64).reshape(12)])
    return _Cam(int(c["width"]), int(c["height"]), float(c["fx"]), float(c["fy"]), float(c["cx"]),
                float(c["cy"]), w2c, float(c.get("near", 0.0)))


def _cams(cams: Sequence[Dict]):
    arr = (_Cam * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = _cam(c)
    return arr


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _geom(scene):
    return (_f64(scene["centers"]), _f64(scene["scales"]), _f64(scene["quats"]))


def all_pixels(cams: Sequence[Dict]) -> np.ndarray:
    out = []
    for v, c in enumerate(cams):
        ys, xs = np.meshgrid(np.arange(c["height"]), np.arange(c["width"]), indexing="ij")
        out.append(np.stack([np.full(xs.size, v), xs.reshape(-1), ys.reshape(-1)], axis=1))
    return np.ascontiguousarray(np.concatenate(out).astype(np.int32))


def input_dim(cfg) -> int:
    return int(_load().orc_input_dim(ctypes.byref(_cfg(cfg))))


def param_count(cfg) -> int:
    return int(_load().orc_param_count(ctypes.byref(_cfg(cfg))))


def _feat_width(cfg) -> int:
    return int(cfg.feat_dim) + int(getattr(cfg, "slot_dim", 0))


def _weights(cfg, scene, K) -> np.ndarray:
    w = _f64(scene["weights"]).reshape(K, -1) if K > 0 else np.zeros((0, param_count(cfg)))
    if w.shape[1] != param_count(cfg):
        raise ValueError(f"weights have {w.shape[1]} parameters per primitive, the config {param_count(cfg)}")
    return np.ascontiguousarray(w)


def slot_weights(u) -> np.ndarray:
    """softmax_k(a_k . u) over the four tetrahedral directions (Sec. 3.4)."""
    g = np.zeros(4)
    _load().orc_slot_weights(_dp(_f64(u)), _dp(g))
    return g


def render(cfg, scene, cams: Sequence[Dict], pix: Optional[np.ndarray] = None, n_threads: int = 0):
    """Render listed pixels (int32 [n, 3] of (view, x, y); all pixels when None).

    Returns (rgb [n, 3], trans [n], feat [n, F + slot_dim] or None) in float64: the MLP's extra
    outputs, then the slot features."""
    lib = _load()
    if pix is None:
        pix = all_pixels(cams)
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    n = pix.shape[0]
    c, s, q = _geom(scene)
    w = _weights(cfg, scene, c.shape[0])
    K = c.shape[0]
    rgb = np.zeros((n, 3))
    trans = np.zeros(n)
    F = _feat_width(cfg)
    feat = np.zeros((n, F)) if F > 0 else None
    cam_arr = _cams(cams)
    st = lib.orc_render(ctypes.byref(_cfg(cfg)), K, _dp(c), _dp(s), _dp(q), _dp(w), len(cams), cam_arr,
                        n, pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(rgb), _dp(trans),
                        _dp(feat), int(n_threads))
    if st != 0:
        raise RuntimeError(f"orc_render failed with status {st}")
    return rgb, trans, feat


def render_backward(cfg, scene, cams: Sequence[Dict], pix: Optional[np.ndarray], g_rgb,
                    g_trans=None, g_feat=None, n_threads: int = 0):
    """Gradients of L over the listed pixels given dL/dC [n,3], dL/dT [n], dL/dF [n,F].

    Returns a dict with forward outputs and d_weights [K,P], d_centers, d_scales, d_quats."""
    lib = _load()
    if pix is None:
        pix = all_pixels(cams)
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    n = pix.shape[0]
    c, s, q = _geom(scene)
    K = c.shape[0]
    w = _weights(cfg, scene, K)
    P = w.shape[1]
    gr = _f64(g_rgb).reshape(n, 3)
    gt = None if g_trans is None else _f64(g_trans).reshape(n)
    F = _feat_width(cfg)
    gf = None if (g_feat is None or F == 0) else _f64(g_feat).reshape(n, F)
    rgb = np.zeros((n, 3)); trans = np.zeros(n)
    feat = np.zeros((n, F)) if F > 0 else None
    dw = np.zeros((K, P)); dc = np.zeros((K, 3)); ds = np.zeros((K, 3)); dq = np.zeros((K, 4))
    st = lib.orc_render_backward(ctypes.byref(_cfg(cfg)), K, _dp(c), _dp(s), _dp(q), _dp(w), len(cams),
                                 _cams(cams), n, pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 _dp(gr), _dp(gt), _dp(gf), _dp(rgb), _dp(trans), _dp(feat), _dp(dw),
                                 _dp(dc), _dp(ds), _dp(dq), int(n_threads))
    if st != 0:
        raise RuntimeError(f"orc_render_backward failed with status {st}")
    return {"rgb": rgb, "trans": trans, "feat": feat, "d_weights": dw, "d_centers": dc,
            "d_scales": ds, "d_quats": dq}


def ray_hits(scene, cam: Dict, x: int, y: int, tile: int = 0):
    """Sorted hits of one pixel's ray: dict of arrays prim, key, t0, t1, m2 (tile > 0: in the
    tile-centre order of tile x tile tiles, key = the tile key)."""
    lib = _load()
    c, s, q = _geom(scene)
    K = c.shape[0]
    cap = max(K, 1)
    prim = np.zeros(cap, dtype=np.int32)
    key = np.zeros(cap); t0 = np.zeros(cap); t1 = np.zeros(cap); m2 = np.zeros(cap)
    n = lib.orc_ray_hits(K, _dp(c), _dp(s), _dp(q), ctypes.byref(_cam(cam)), int(x), int(y), int(tile), cap,
                         prim.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(key), _dp(t0), _dp(t1),
                         _dp(m2))
    if n < 0:
        raise RuntimeError("orc_ray_hits: invalid input")
    return {"prim": prim[:n], "key": key[:n], "t0": t0[:n], "t1": t1[:n], "m2": m2[:n]}


def ray_m2(scene, cam: Dict, x: int, y: int):
    """Per-primitive squared normalised ray distance m2 and chord midpoint t_mid."""
    lib = _load()
    c, s, q = _geom(scene)
    K = c.shape[0]
    m2 = np.zeros(max(K, 1)); tm = np.zeros(max(K, 1))
    st = lib.orc_ray_m2(K, _dp(c), _dp(s), _dp(q), ctypes.byref(_cam(cam)), int(x), int(y), _dp(m2), _dp(tm))
    if st != 0:
        raise RuntimeError("orc_ray_m2: invalid input")
    return m2[:K], tm[:K]


def pixel_ray(cam: Dict, x: int, y: int):
    lib = _load()
    o = np.zeros(3); d = np.zeros(3)
    lib.orc_pixel_ray(ctypes.byref(_cam(cam)), int(x), int(y), _dp(o), _dp(d))
    return o, d


def encode(cfg, xl, d) -> np.ndarray:
    lib = _load()
    out = np.zeros(512)
    n = lib.orc_encode(ctypes.byref(_cfg(cfg)), _dp(_f64(xl)), _dp(_f64(d)), _dp(out))
    return out[:n]


def mlp(cfg, w, enc) -> np.ndarray:
    lib = _load()
    out = np.zeros(4 + int(cfg.feat_dim))
    st = lib.orc_mlp(ctypes.byref(_cfg(cfg)), _dp(_f64(w)), _dp(_f64(enc)), _dp(out))
    if st != 0:
        raise RuntimeError("orc_mlp failed")
    return out
