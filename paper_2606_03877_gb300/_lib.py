"""ctypes binding of ``libmlps.so`` (include/mlps.h), argument marshalling only.

Every function keeps the C name and takes device pointers as Python ints (``tensor.data_ptr()``)
or torch tensors, host structs as the ctypes classes below, and streams as the integer handle
(``torch.cuda.current_stream().cuda_stream``). All rendering work runs in the CUDA library; there
is no fallback: :func:`load` raises if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmlps.so")

MLPS_OK = 0
MLPS_ERR_INVALID_ARGUMENT = 1
MLPS_ERR_UNSUPPORTED = 2
MLPS_ERR_WORKSPACE_TOO_SMALL = 3
MLPS_ERR_CAPACITY_OVERFLOW = 4
MLPS_ERR_TIMEOUT = 5
MLPS_ERR_NONFINITE = 6
MLPS_ERR_CUDA = 7

MLPS_FP32 = 0
MLPS_BF16 = 1
MLPS_FP8_E4M3 = 2
MLPS_MAX_VIEWS = 64

PRECISIONS = {"fp32": MLPS_FP32, "bf16": MLPS_BF16, "fp8": MLPS_FP8_E4M3}


class MlpsConfig(ctypes.Structure):
    _fields_ = [("xyz_freqs", ctypes.c_int32), ("dir_freqs", ctypes.c_int32),
                ("hidden_width", ctypes.c_int32), ("hidden_layers", ctypes.c_int32),
                ("feat_dim", ctypes.c_int32), ("samples", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_hits_per_ray", ctypes.c_int32),
                ("hit_capacity_per_ray", ctypes.c_float), ("t_eps", ctypes.c_float),
                ("tile", ctypes.c_int32), ("mlp_groups", ctypes.c_int32),
                ("contact", ctypes.c_int32), ("slot_dim", ctypes.c_int32),
                ("tile_sort", ctypes.c_int32), ("early_stop_wave", ctypes.c_int32)]


class MlpsCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("world_to_cam", ctypes.c_float * 12), ("near_t", ctypes.c_float)]


class MlpsBatchItem(ctypes.Structure):
    _fields_ = [("prim_offset", ctypes.c_int32), ("prim_count", ctypes.c_int32), ("cam", MlpsCamera)]


class MlpsBatchCaps(ctypes.Structure):
    _fields_ = [("max_width", ctypes.c_int32), ("max_height", ctypes.c_int32), ("max_prim_count", ctypes.c_int32)]


class MlpsScene(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("centers", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("weights", ctypes.c_void_p)]


class MlpsLossDesc(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int32), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("tile_mask", ctypes.c_void_p), ("lambda_ssim", ctypes.c_float),
                ("feat_dim", ctypes.c_int32)]


class MlpsAdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("aux", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("lr", ctypes.c_float), ("kind", ctypes.c_int32)]


MLPS_MAX_ADAM_GROUPS = 8


class MlpsError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {mlps_status_string(status)} ({status})")


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes)
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_SIGS = [
    ("mlps_abi_version", ctypes.c_int32, []),
    ("mlps_status_string", ctypes.c_char_p, [ctypes.c_int32]),
    ("mlps_config_default", ctypes.c_int32, [_P(MlpsConfig), ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("mlps_input_dim", ctypes.c_int32, [_P(MlpsConfig)]),
    ("mlps_param_count", ctypes.c_int64, [_P(MlpsConfig)]),
    ("mlps_weight_stride", ctypes.c_int64, [_P(MlpsConfig)]),
    ("mlps_check_config", ctypes.c_int32, [_P(MlpsConfig)]),
    ("mlps_pack_weights", ctypes.c_int32, [_P(MlpsConfig), ctypes.c_int32, _vp, _vp, _vp]),
    ("mlps_workspace_size", ctypes.c_int32, [_P(MlpsConfig), ctypes.c_int32, _P(MlpsCamera),
                                             ctypes.c_int32, _P(ctypes.c_size_t), _P(ctypes.c_size_t)]),
    ("mlps_render_forward", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _P(MlpsCamera),
                                             ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                             _vp, ctypes.c_size_t, _vp]),
    ("mlps_render_backward", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _P(MlpsCamera),
                                              ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                              _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    ("mlps_batch_workspace_size", ctypes.c_int32, [_P(MlpsConfig), ctypes.c_int32, _P(MlpsBatchItem),
                                                   ctypes.c_int32, _P(ctypes.c_size_t), _P(ctypes.c_size_t)]),
    ("mlps_render_batch_forward", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _P(MlpsBatchItem),
                                                   ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                                   _vp, ctypes.c_size_t, _vp]),
    ("mlps_render_batch_backward", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _P(MlpsBatchItem),
                                                    ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                                    _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    ("mlps_autotune_batch", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _P(MlpsBatchItem), ctypes.c_int32,
                                             ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp,
                                             ctypes.c_size_t, _vp, _vp, _vp, _vp, ctypes.c_int32,
                                             _P(MlpsConfig), _P(ctypes.c_float), _P(ctypes.c_int32),
                                             _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_float), _vp]),
    ("mlps_autotune_clear", None, []),
    ("mlps_batch_workspace_size_dev", ctypes.c_int32, [_P(MlpsConfig), ctypes.c_int32, ctypes.c_int32,
                                                       _P(MlpsBatchCaps), _P(ctypes.c_size_t),
                                                       _P(ctypes.c_size_t)]),
    ("mlps_render_batch_forward_dev", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _vp, ctypes.c_int32,
                                                       _P(MlpsBatchCaps), _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                                       _vp, ctypes.c_size_t, _vp]),
    ("mlps_render_batch_backward_dev", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _vp, ctypes.c_int32,
                                                        _P(MlpsBatchCaps), _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                                        _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    ("mlps_render_forward_static", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsScene), _P(MlpsCamera),
                                                    ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]),
    ("mlps_read_status", ctypes.c_int32, [_vp, _vp]),
    ("mlps_saved_hit_count", ctypes.c_int32, [_vp, _P(ctypes.c_int64), _vp]),
    ("mlps_backward_chunk_counts", ctypes.c_int32, [_vp, _vp, _P(ctypes.c_int64), _P(ctypes.c_int64), _vp]),
    ("mlps_forward_wave_counts", ctypes.c_int32, [_vp, _vp, _P(ctypes.c_int64), _P(ctypes.c_int64), _vp]),
    ("mlps_selftest_bounded_wait", ctypes.c_int32, [ctypes.c_int32, _vp, ctypes.c_size_t, _vp]),
    ("mlps_export_hits", ctypes.c_int32, [_P(MlpsConfig), _P(MlpsCamera), ctypes.c_int32, _vp,
                                          ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("mlps_export_tiles", ctypes.c_int32, [_P(MlpsConfig), ctypes.c_int32, _P(MlpsCamera),
                                           ctypes.c_int32, _vp, _vp, _vp, _vp]),
    ("mlps_loss_workspace_size", ctypes.c_size_t, [_P(MlpsLossDesc)]),
    ("mlps_loss", ctypes.c_int32, [_P(MlpsLossDesc), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                   _vp]),
    ("mlps_adam_step", ctypes.c_int32, [_P(MlpsAdamGroup), ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_int32, _vp]),
    ("mlps_kernel_launches", ctypes.c_int64, [ctypes.c_int32]),
    ("mlps_profiler_enable", None, [ctypes.c_int32]),
    ("mlps_profiler_read", ctypes.c_int32, [_P(ctypes.c_char_p), _P(ctypes.c_float),
                                            _P(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32]),
]


def exported_symbols() -> list:
    return [s[0] for s in _SIGS]


def load(path: Optional[str] = None):
    """Load the CUDA library. Raises if it is missing: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libmlps.so not found at {p}; build it with "
                               "`python -m paper_2606_03877_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(p)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _check(fn: str, st: int):
    if st != MLPS_OK:
        raise MlpsError(fn, st)


def mlps_backward_chunk_counts(saved, scratch, stream: int = 0):
    """(chunks of the forward pass, chunks the last backward pass walked)."""
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    _check("mlps_backward_chunk_counts", load().mlps_backward_chunk_counts(
        _ptr(saved), _ptr(scratch), ctypes.byref(a), ctypes.byref(b), stream or None))
    return int(a.value), int(b.value)


def mlps_forward_wave_counts(saved, scratch, stream: int = 0):
    """(hit intervals of the last forward pass, intervals its depth waves evaluated)."""
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    _check("mlps_forward_wave_counts", load().mlps_forward_wave_counts(
        _ptr(saved), _ptr(scratch), ctypes.byref(a), ctypes.byref(b), stream or None))
    return int(a.value), int(b.value)


def mlps_selftest_bounded_wait(limit_us: int, scratch, stream: int = 0):
    _check("mlps_selftest_bounded_wait", load().mlps_selftest_bounded_wait(
        int(limit_us), _ptr(scratch), int(scratch.numel() * scratch.element_size()), stream or None))


def mlps_abi_version() -> int:
    return int(load().mlps_abi_version())


def mlps_status_string(st: int) -> str:
    try:
        return load().mlps_status_string(int(st)).decode()
    except Exception:  # library missing: still give a message
        return f"status {st}"


def mlps_config_default(xyz_freqs, dir_freqs, hidden_width, hidden_layers, feat_dim) -> MlpsConfig:
    c = MlpsConfig()
    _check("mlps_config_default", load().mlps_config_default(ctypes.byref(c), xyz_freqs, dir_freqs,
                                                           hidden_width, hidden_layers, feat_dim))
    return c


def mlps_input_dim(cfg: MlpsConfig) -> int:
    return int(load().mlps_input_dim(ctypes.byref(cfg)))


def mlps_param_count(cfg: MlpsConfig) -> int:
    return int(load().mlps_param_count(ctypes.byref(cfg)))


def mlps_weight_stride(cfg: MlpsConfig) -> int:
    return int(load().mlps_weight_stride(ctypes.byref(cfg)))


def mlps_check_config(cfg: MlpsConfig) -> int:
    return int(load().mlps_check_config(ctypes.byref(cfg)))


def mlps_pack_weights(cfg: MlpsConfig, K: int, weights_fp32, packed, stream: int = 0):
    _check("mlps_pack_weights", load().mlps_pack_weights(ctypes.byref(cfg), int(K), _ptr(weights_fp32),
                                                       _ptr(packed), stream or None))


def cameras(cams: Sequence[dict]):
    arr = (MlpsCamera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].width = int(c["width"])
        arr[i].height = int(c["height"])
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = (float(c["fx"]), float(c["fy"]),
                                                      float(c["cx"]), float(c["cy"]))
        w2c = [float(v) for v in list(c["w2c"])]
        for k in range(12):
            arr[i].world_to_cam[k] = w2c[k]
        arr[i].near_t = float(c.get("near", 0.0))
    return arr


def mlps_workspace_size(cfg: MlpsConfig, K: int, cams, n_views: int):
    s = ctypes.c_size_t()
    t = ctypes.c_size_t()
    _check("mlps_workspace_size", load().mlps_workspace_size(ctypes.byref(cfg), int(K), cams, int(n_views),
                                                           ctypes.byref(s), ctypes.byref(t)))
    return int(s.value), int(t.value)


def make_scene(K, centers, scales, quats, packed) -> MlpsScene:
    return MlpsScene(int(K), _ptr(centers), _ptr(scales), _ptr(quats), _ptr(packed))


def mlps_render_forward(cfg, scene: MlpsScene, cams, n_views, rgb, trans, feat, saved, saved_bytes,
                        scratch, scratch_bytes, stream: int = 0):
    _check("mlps_render_forward", load().mlps_render_forward(
        ctypes.byref(cfg), ctypes.byref(scene), cams, int(n_views), _ptr(rgb), _ptr(trans), _ptr(feat),
        _ptr(saved), int(saved_bytes), _ptr(scratch), int(scratch_bytes), stream or None))


def mlps_render_backward(cfg, scene: MlpsScene, cams, n_views, d_rgb, d_trans, d_feat, saved, saved_bytes,
                         d_weights, d_centers, d_scales, d_quats, scratch, scratch_bytes, stream: int = 0):
    _check("mlps_render_backward", load().mlps_render_backward(
        ctypes.byref(cfg), ctypes.byref(scene), cams, int(n_views), _ptr(d_rgb), _ptr(d_trans), _ptr(d_feat),
        _ptr(saved), int(saved_bytes), _ptr(d_weights), _ptr(d_centers), _ptr(d_scales), _ptr(d_quats),
        _ptr(scratch), int(scratch_bytes), stream or None))


def batch_items(items: Sequence[tuple]):
    """Host array of mlps_batch_item from (prim_offset, prim_count, camera dict) tuples."""
    arr = (MlpsBatchItem * len(items))()
    for i, (off, cnt, cam) in enumerate(items):
        arr[i].prim_offset = int(off)
        arr[i].prim_count = int(cnt)
        arr[i].cam = cameras([cam])[0]
    return arr


def mlps_batch_workspace_size(cfg: MlpsConfig, K: int, items, n_items: int):
    s = ctypes.c_size_t()
    t = ctypes.c_size_t()
    _check("mlps_batch_workspace_size", load().mlps_batch_workspace_size(
        ctypes.byref(cfg), int(K), items, int(n_items), ctypes.byref(s), ctypes.byref(t)))
    return int(s.value), int(t.value)


def mlps_render_batch_forward(cfg, scene: MlpsScene, items, n_items, rgb, trans, feat, saved, saved_bytes,
                              scratch, scratch_bytes, stream: int = 0):
    _check("mlps_render_batch_forward", load().mlps_render_batch_forward(
        ctypes.byref(cfg), ctypes.byref(scene), items, int(n_items), _ptr(rgb), _ptr(trans), _ptr(feat),
        _ptr(saved), int(saved_bytes), _ptr(scratch), int(scratch_bytes), stream or None))


def mlps_render_batch_backward(cfg, scene: MlpsScene, items, n_items, d_rgb, d_trans, d_feat, saved,
                               saved_bytes, d_weights, d_centers, d_scales, d_quats, scratch, scratch_bytes,
                               stream: int = 0):
    _check("mlps_render_batch_backward", load().mlps_render_batch_backward(
        ctypes.byref(cfg), ctypes.byref(scene), items, int(n_items), _ptr(d_rgb), _ptr(d_trans), _ptr(d_feat),
        _ptr(saved), int(saved_bytes), _ptr(d_weights), _ptr(d_centers), _ptr(d_scales), _ptr(d_quats),
        _ptr(scratch), int(scratch_bytes), stream or None))


def batch_caps(max_width: int, max_height: int, max_prim_count: int) -> MlpsBatchCaps:
    return MlpsBatchCaps(int(max_width), int(max_height), int(max_prim_count))


def mlps_batch_workspace_size_dev(cfg: MlpsConfig, K: int, n_items: int, caps: MlpsBatchCaps):
    s = ctypes.c_size_t()
    t = ctypes.c_size_t()
    _check("mlps_batch_workspace_size_dev", load().mlps_batch_workspace_size_dev(
        ctypes.byref(cfg), int(K), int(n_items), ctypes.byref(caps), ctypes.byref(s), ctypes.byref(t)))
    return int(s.value), int(t.value)


def mlps_render_batch_forward_dev(cfg, scene: MlpsScene, dev_items, n_items, caps: MlpsBatchCaps, rgb, trans,
                                  feat, saved, saved_bytes, scratch, scratch_bytes, stream: int = 0):
    _check("mlps_render_batch_forward_dev", load().mlps_render_batch_forward_dev(
        ctypes.byref(cfg), ctypes.byref(scene), _ptr(dev_items), int(n_items), ctypes.byref(caps), _ptr(rgb),
        _ptr(trans), _ptr(feat), _ptr(saved), int(saved_bytes), _ptr(scratch), int(scratch_bytes),
        stream or None))


def mlps_render_batch_backward_dev(cfg, scene: MlpsScene, dev_items, n_items, caps: MlpsBatchCaps, d_rgb,
                                   d_trans, d_feat, saved, saved_bytes, d_weights, d_centers, d_scales, d_quats,
                                   scratch, scratch_bytes, stream: int = 0):
    _check("mlps_render_batch_backward_dev", load().mlps_render_batch_backward_dev(
        ctypes.byref(cfg), ctypes.byref(scene), _ptr(dev_items), int(n_items), ctypes.byref(caps), _ptr(d_rgb),
        _ptr(d_trans), _ptr(d_feat), _ptr(saved), int(saved_bytes), _ptr(d_weights), _ptr(d_centers),
        _ptr(d_scales), _ptr(d_quats), _ptr(scratch), int(scratch_bytes), stream or None))


def mlps_autotune_batch(cfg, scene: MlpsScene, items, n_items, do_backward, d_rgb, rgb, trans, feat, saved,
                        saved_bytes, scratch, scratch_bytes, d_weights, d_centers, d_scales, d_quats,
                        reps: int = 3, stream: int = 0):
    """Returns (tuned MlpsConfig, best ms, [(tile, groups, ms), ...] candidates timed)."""
    tuned = MlpsConfig()
    best = ctypes.c_float()
    nc = ctypes.c_int32()
    ct = (ctypes.c_int32 * 16)()
    cg = (ctypes.c_int32 * 16)()
    cm = (ctypes.c_float * 16)()
    _check("mlps_autotune_batch", load().mlps_autotune_batch(
        ctypes.byref(cfg), ctypes.byref(scene), items, int(n_items), int(do_backward), _ptr(d_rgb), _ptr(rgb),
        _ptr(trans), _ptr(feat), _ptr(saved), int(saved_bytes), _ptr(scratch), int(scratch_bytes),
        _ptr(d_weights), _ptr(d_centers), _ptr(d_scales), _ptr(d_quats), int(reps), ctypes.byref(tuned),
        ctypes.byref(best), ctypes.byref(nc), ct, cg, cm, stream or None))
    return tuned, float(best.value), [(int(ct[i]), int(cg[i]), float(cm[i])) for i in range(nc.value)]


def mlps_autotune_clear():
    load().mlps_autotune_clear()


def mlps_render_forward_static(cfg, scene: MlpsScene, cams, n_views, rgb, trans, feat,
                               device_status=None, stream: int = 0):
    _check("mlps_render_forward_static", load().mlps_render_forward_static(
        ctypes.byref(cfg), ctypes.byref(scene), cams, int(n_views), _ptr(rgb), _ptr(trans), _ptr(feat),
        _ptr(device_status), stream or None))


def mlps_read_status(region, stream: int = 0) -> int:
    return int(load().mlps_read_status(_ptr(region), stream or None))


def mlps_saved_hit_count(saved, stream: int = 0) -> int:
    n = ctypes.c_int64()
    _check("mlps_saved_hit_count", load().mlps_saved_hit_count(_ptr(saved), ctypes.byref(n), stream or None))
    return int(n.value)


def mlps_export_hits(cfg, cams, n_views, saved, max_out, count, prim, t0, t1, tmid, stream: int = 0):
    _check("mlps_export_hits", load().mlps_export_hits(ctypes.byref(cfg), cams, int(n_views), _ptr(saved),
                                                     int(max_out), _ptr(count), _ptr(prim), _ptr(t0),
                                                     _ptr(t1), _ptr(tmid), stream or None))


def mlps_export_tiles(cfg, K, cams, n_views, scratch, count, lst, stream: int = 0):
    _check("mlps_export_tiles", load().mlps_export_tiles(ctypes.byref(cfg), int(K), cams, int(n_views),
                                                       _ptr(scratch), _ptr(count), _ptr(lst), stream or None))


def mlps_kernel_launches(reset: bool = False) -> int:
    return int(load().mlps_kernel_launches(1 if reset else 0))


def mlps_profiler_enable(on: bool):
    load().mlps_profiler_enable(1 if on else 0)


def mlps_profiler_read(reset: bool = False) -> dict:
    n = 32
    names = (ctypes.c_char_p * n)()
    ms = (ctypes.c_float * n)()
    cnt = (ctypes.c_int32 * n)()
    k = load().mlps_profiler_read(names, ms, cnt, n, 1 if reset else 0)
    return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(min(k, n))}


def loss_desc(n_views: int, height: int, width: int, tile: int = 8, tile_mask=None, lambda_ssim: float = 0.2,
              feat_dim: int = 0) -> MlpsLossDesc:
    return MlpsLossDesc(int(n_views), int(height), int(width), int(tile), _ptr(tile_mask), float(lambda_ssim),
                        int(feat_dim))


def mlps_loss_workspace_size(desc: MlpsLossDesc) -> int:
    return int(load().mlps_loss_workspace_size(ctypes.byref(desc)))


def mlps_loss(desc: MlpsLossDesc, rgb, rgb_target, feat, feat_target, d_rgb, d_feat, loss_out, workspace,
              workspace_bytes: int, stream: int = 0):
    _check("mlps_loss", load().mlps_loss(ctypes.byref(desc), _ptr(rgb), _ptr(rgb_target), _ptr(feat),
                                         _ptr(feat_target), _ptr(d_rgb), _ptr(d_feat), _ptr(loss_out),
                                         _ptr(workspace), int(workspace_bytes), stream))


def adam_group(param, grad, m, v, lr: float, aux=None, kind: int = 0) -> MlpsAdamGroup:
    return MlpsAdamGroup(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), _ptr(aux), int(param.numel()), float(lr),
                         int(kind))


def mlps_adam_step(groups: Sequence[MlpsAdamGroup], beta1: float, beta2: float, eps: float, step: int,
                   stream: int = 0):
    arr = (MlpsAdamGroup * len(groups))(*groups)
    _check("mlps_adam_step", load().mlps_adam_step(arr, len(groups), float(beta1), float(beta2), float(eps),
                                                   int(step), stream))
