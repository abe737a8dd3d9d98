"""The allocation-free forward entry point (mlps_render_forward_static).

It serves callers that cannot allocate device memory where they render (device memory owned by
another allocator, or frame loops that must not call cudaMalloc / cudaFree). It renders into
the caller's outputs with a fixed 32 MiB workspace kept in a static device array. This file is
named so that pytest collects it last; every test here also passes when run alone in a fresh
process.
"""
import numpy as np
import pytest
import torch

from paper_2606_03877_gb300 import _lib, synth
from paper_2606_03877_gb300.render import Renderer, make_config

from helpers import scaled_scene, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _regular(cfg, scene, cams, precision):
    r = Renderer(cfg, precision=precision)
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    out = r.forward(d["centers"], d["scales"], d["quats"], packed, cams)
    torch.cuda.synchronize()
    assert r.status() == 0
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}, r, packed


def _static(cfg, scene, cams, precision, r, packed):
    d = to_dev(scene)
    V = len(cams)
    rgb = torch.full((V, cfg.height, cfg.width, 3), -1.0, device="cuda")
    trans = torch.full((V, cfg.height, cfg.width), -1.0, device="cuda")
    feat = torch.full((V, cfg.height, cfg.width, cfg.feat_dim), -1.0, device="cuda") if cfg.feat_dim else None
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    packed2 = r.pack(d["weights"])
    scn = _lib.make_scene(cfg.K, d["centers"], d["scales"], d["quats"], packed2)
    _lib.mlps_render_forward_static(r.cfg, scn, _lib.cameras(cams), V, rgb, trans, feat, status,
                                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return {"rgb": rgb.cpu().numpy(), "trans": trans.cpu().numpy(),
            "feat": feat.cpu().numpy() if feat is not None else None}


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_static_forward_matches_regular_entry_point_on_two_calls(precision):
    cfgs = [synth.CONFIGS["prec"].replace(width=96, height=64, K=16, n_views=2),
            synth.CONFIGS["prec"].replace(width=80, height=72, K=24, n_views=1)]
    seeds = [3, 4]
    for cfg, seed in zip(cfgs, seeds):  # two calls in a row, different scenes and sizes
        scene = scaled_scene(cfg, seed, 2.0)
        cams = synth.make_cameras(cfg, first_view_seed=seed)
        ref, r, packed = _regular(cfg, scene, cams, precision)
        got = _static(cfg, scene, cams, precision, r, packed)
        assert np.abs(got["rgb"] - ref["rgb"]).max() <= TOL
        assert np.abs(got["trans"] - ref["trans"]).max() <= TOL
        assert (ref["trans"] < 1).sum() > 100


def test_static_forward_allocates_nothing_after_the_first_call():
    """The first call on a device reserves the static array (module load); from then on a call
    leaves the device's free memory unchanged."""
    cfg = synth.CONFIGS["prec"].replace(width=64, height=48, K=12, n_views=1)
    scene = scaled_scene(cfg, 5, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=5)
    r = Renderer(cfg, precision="fp32")
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    rgb = torch.empty((1, cfg.height, cfg.width, 3), device="cuda")
    trans = torch.empty((1, cfg.height, cfg.width), device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    scn = _lib.make_scene(cfg.K, d["centers"], d["scales"], d["quats"], packed)
    cs = _lib.cameras(cams)
    stream = torch.cuda.current_stream().cuda_stream
    _lib.mlps_render_forward_static(r.cfg, scn, cs, 1, rgb, trans, None, status, stream)  # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _lib.mlps_render_forward_static(r.cfg, scn, cs, 1, rgb, trans, None, status, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(status.item()) == 0


def test_static_forward_reports_device_detected_error():
    """A non-finite primitive centre, made on the host: the call returns MLPS_OK (nothing is
    wrong on the host side) and the device status word it hands back says MLPS_ERR_NONFINITE."""
    cfg = synth.CONFIGS["prec"].replace(width=64, height=48, K=12, n_views=1)
    scene = scaled_scene(cfg, 6, 2.0)
    scene["centers"][3, 1] = np.nan
    cams = synth.make_cameras(cfg, first_view_seed=6)
    r = Renderer(cfg, precision="fp32")
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    rgb = torch.empty((1, cfg.height, cfg.width, 3), device="cuda")
    trans = torch.empty((1, cfg.height, cfg.width), device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    scn = _lib.make_scene(cfg.K, d["centers"], d["scales"], d["quats"], packed)
    _lib.mlps_render_forward_static(r.cfg, scn, _lib.cameras(cams), 1, rgb, trans, None, status,
                                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(status.item()) == _lib.MLPS_ERR_NONFINITE


def test_static_forward_rejects_workspace_beyond_limit():
    cfg = synth.CONFIGS["prec"]  # 1080p x 8 views needs gigabytes
    r = Renderer(cfg.replace(n_views=1), precision="fp32")
    cams = _lib.cameras(synth.make_cameras(cfg))
    scn = _lib.make_scene(cfg.K, 16, 16, 16, 256)  # rejected before any pointer is used
    with pytest.raises(_lib.MlpsError) as e:
        _lib.mlps_render_forward_static(r.cfg, scn, cams, cfg.n_views, 256, 256, None, None, 0)
    assert e.value.status == _lib.MLPS_ERR_WORKSPACE_TOO_SMALL
