"""The configuration's limits on the GPU, against the FP64 oracle: the deepest network (six
hidden layers), the longest intervals (S = 128: one interval per chunk of 128 sample rows), and
the shape combinations the tensor-core backward does not cover, which must be refused with
MLPS_ERR_UNSUPPORTED (and leave the renderer usable) rather than run."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import _lib, synth
from paper_2606_03877_gb300.render import Renderer

from helpers import psnr, rel_l2, scaled_scene, to_dev

pytestmark = pytest.mark.gpu

GROUPS = ["d_weights", "d_centers", "d_scales", "d_quats"]
GRAD_BAR = {"fp32": 1e-3, "bf16": 2e-2, "fp8": 2e-2}


def _l2_grad(cfg, scene, cams):
    cur, _, _ = oracle.render(cfg, scene, cams)
    tgt, _, _ = oracle.render(cfg, synth.perturb_scene(scene, cfg, 1), cams)
    return (cur - tgt).reshape(len(cams), cfg.height, cfg.width, 3).astype(np.float32)


def _forward_backward(cfg, scene, cams, precision, g):
    r = Renderer(cfg, precision=precision)
    d = to_dev(scene)
    out = r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    got = r.backward(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    return out["rgb"].cpu().numpy().reshape(-1, 3), {k: v.cpu().numpy() for k, v in got.items()}


def _check(cfg, scene, cams, precision):
    g = _l2_grad(cfg, scene, cams)
    rgb, got = _forward_backward(cfg, scene, cams, precision, g)
    rgb_o, _, _ = oracle.render(cfg, scene, cams)
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g.reshape(-1, 3), None, None)
    errs = {k: rel_l2(got[k], ref[k]) for k in GROUPS}
    print(cfg.hidden_layers, cfg.samples, precision, "psnr", psnr(rgb, rgb_o), errs)
    if precision == "fp32":
        assert np.abs(rgb - rgb_o).max() < 1e-4
    else:
        assert psnr(rgb, rgb_o) >= (45.0 if precision == "bf16" else 38.0)
    for k, e in errs.items():
        assert e < GRAD_BAR[precision], (k, errs)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_six_hidden_layers(precision):
    """60-64x6-4 on the tensor cores: the backward keeps all seven layers' weight gradients in
    TMEM (6 x 64 + 16 columns) next to one group's accumulator (96 columns). BF16 rounding and
    ReLU-mask flips add up over seven layers, so the image is large enough (2 x 128 x 96 pixels
    over 10 primitives) for them to average out in the pose sums."""
    cfg = synth.CONFIGS["prec"].replace(width=128, height=96, K=10, n_views=2, hidden_layers=6)
    scene = scaled_scene(cfg, 31, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=31)
    _check(cfg, scene, cams, precision)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_128_samples_per_interval(precision):
    """S = 128: every chunk of 128 sample rows is one interval."""
    cfg = synth.CONFIGS["prec"].replace(width=40, height=32, K=8, n_views=1, samples=128)
    scene = scaled_scene(cfg, 33, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=33)
    _check(cfg, scene, cams, precision)


@pytest.mark.parametrize("shape", [{"hidden_layers": 6}, {"samples": 128}])
def test_fp32_backward_limits_are_refused(shape):
    """The FP32 backward stages both weight layouts of a primitive in shared memory and works on
    64-row sub-chunks of whole intervals: deeper than three 64-wide hidden layers, or S > 64,
    it is refused (the forward still matches the oracle, and both status words stay clear)."""
    cfg = synth.CONFIGS["prec"].replace(width=40, height=32, K=8, n_views=1, **shape)
    scene = scaled_scene(cfg, 37, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=37)
    r = Renderer(cfg, precision="fp32")
    d = to_dev(scene)
    out = r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    torch.cuda.synchronize()
    rgb_o, _, _ = oracle.render(cfg, scene, cams)
    assert np.abs(out["rgb"].cpu().numpy().reshape(-1, 3) - rgb_o).max() < 1e-4
    with pytest.raises(_lib.MlpsError) as e:
        r.backward(torch.zeros(1, cfg.height, cfg.width, 3, device="cuda"))
    assert e.value.status == _lib.MLPS_ERR_UNSUPPORTED
    assert r.status() == 0 and r.status("scratch") == 0


def test_unsupported_tensor_core_backward_is_refused():
    """Width 64 with a 16-d feature head: the forward runs on the tensor cores, the BF16 backward
    is refused (the 64-wide kernel's head holds at most 4 + 12 outputs), and the same renderer
    still renders and differentiates the FP32 path's shapes afterwards."""
    cfg = synth.SceneConfig("f16", 32, 24, 6, 1, 6, 4, 64, 2, 16, 16)
    scene = scaled_scene(cfg, 35, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=35)
    r = Renderer(cfg, precision="bf16")
    d = to_dev(scene)
    out = r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    torch.cuda.synchronize()
    rgb_o, _, _ = oracle.render(cfg, scene, cams)
    assert psnr(out["rgb"].cpu().numpy().reshape(-1, 3), rgb_o) >= 45.0
    g = torch.zeros(1, cfg.height, cfg.width, 3, device="cuda")
    with pytest.raises(_lib.MlpsError) as e:
        r.backward(g, None, torch.zeros(1, cfg.height, cfg.width, cfg.feat_dim, device="cuda"))
    assert e.value.status == _lib.MLPS_ERR_UNSUPPORTED
    assert r.status() == 0 and r.status("scratch") == 0
    r32 = Renderer(cfg, precision="fp32")
    r32.forward(d["centers"], d["scales"], d["quats"], r32.pack(d["weights"]), cams)
    got = r32.backward(g, None, torch.ones(1, cfg.height, cfg.width, cfg.feat_dim, device="cuda"))
    torch.cuda.synchronize()
    assert r32.status() == 0 and float(got["d_weights"].abs().sum()) > 0
