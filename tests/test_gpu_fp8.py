"""GPU parity of the FP8 (E4M3) tensor-core MLP path (tcgen05 kind::f8f6f4) against the FP64
oracle.

Bar: PSNR >= 38 dB per view for the colour image, the FP8 contract. Weights are stored as E4M3
with one FP32 scale per (primitive, layer, output); activation rows are stored divided by a
power-of-two scale per row. Geometry, encoding, heads, transmittance and compositing stay FP32,
so hit lists are the same as the FP32 path's. The backward pass of the FP8 precision recomputes
the MLP in BF16 (from the BF16 tiles packed in the same blob); its gradients are reported with
a loose bar because the forward outputs it differentiates come from the FP8 evaluation.
"""
import numpy as np
import pytest

import oracle
from paper_2606_03877_gb300 import synth

from helpers import gpu_render, pixel_index, psnr, rel_l2, scaled_scene, to_dev

pytestmark = pytest.mark.gpu

FP8_PSNR = 38.0


def _psnr_views(cfg, scene, cams, **kw):
    r, out, _, _ = gpu_render(cfg, scene, cams, "fp8", **kw)
    assert r.status() == 0
    rgb_o, T_o, F_o = oracle.render(cfg, scene, cams)
    n = cfg.width * cfg.height
    rgb = out["rgb"].reshape(-1, 3)
    ps = [psnr(rgb[v * n:(v + 1) * n], rgb_o[v * n:(v + 1) * n]) for v in range(len(cams))]
    return ps, r, out, (rgb_o, T_o, F_o)


def test_fp8_small_prec_shape():
    cfg = synth.CONFIGS["prec"].replace(width=64, height=48, K=12, n_views=1)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    ps, r, out, (rgb_o, T_o, _) = _psnr_views(cfg, scene, cams)
    print("fp8 psnr", ps, "max|dT|", np.abs(out["trans"].reshape(-1) - T_o).max())
    assert min(ps) >= FP8_PSNR, ps


@pytest.mark.parametrize("S", [16, 32, 48])
def test_fp8_segment_lengths(S):
    cfg = synth.CONFIGS["prec"].replace(width=100, height=75, K=24, n_views=2, samples=S)
    scene = scaled_scene(cfg, 2, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=2)
    ps, r, out, (rgb_o, T_o, _) = _psnr_views(cfg, scene, cams)
    print("fp8 psnr", S, ps)
    assert min(ps) >= FP8_PSNR, ps


def test_fp8_fp8_is_closer_to_bf16_than_to_zero():
    """The FP8 image differs from the BF16 one by quantisation noise only: far below the signal."""
    cfg = synth.CONFIGS["prec"].replace(width=80, height=60, K=16, n_views=1)
    scene = scaled_scene(cfg, 5, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=5)
    _, o8, _, _ = gpu_render(cfg, scene, cams, "fp8")
    _, o16, _, _ = gpu_render(cfg, scene, cams, "bf16")
    err = np.linalg.norm(o8["rgb"] - o16["rgb"])
    assert err < 0.05 * np.linalg.norm(o16["rgb"]), err


def test_fp8_wide_mlp_with_features():
    """Stress shape: width 128 x 4 hidden layers and a 16-d linear feature head, S = 48."""
    cfg = synth.CONFIGS["stress"].replace(width=80, height=60, K=20, n_views=1)
    scene = scaled_scene(cfg, 3, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=3)
    ps, r, out, (rgb_o, T_o, F_o) = _psnr_views(cfg, scene, cams)
    f = out["feat"].reshape(-1, cfg.feat_dim)
    rel = rel_l2(f, F_o)
    print("fp8 stress-shape psnr", ps, "feature rel-L2", rel)
    assert min(ps) >= FP8_PSNR, ps
    assert rel < 0.1, rel


def test_fp8_generic_encoding_path():
    """Frequency counts without a compile-time fast path go through the byte-wise row writer."""
    cfg = synth.SceneConfig("g", 64, 48, 12, 1, 4, 2, 64, 2, 0, 24)
    scene = scaled_scene(cfg, 6, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=6)
    ps, _, _, _ = _psnr_views(cfg, scene, cams)
    assert min(ps) >= FP8_PSNR, ps


def test_fp8_raw_xyz_input():
    cfg = synth.CONFIGS["pr1"].replace(hidden_width=64)
    scene = scaled_scene(cfg, 0, 2.0)
    cams = synth.make_cameras(cfg)
    ps, _, _, _ = _psnr_views(cfg, scene, cams)
    assert min(ps) >= FP8_PSNR, ps


def test_fp8_hits_identical_to_fp32_path():
    cfg = synth.CONFIGS["prec"].replace(width=96, height=64, K=32, n_views=1)
    scene = scaled_scene(cfg, 4, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=4)
    r8, _, _, _ = gpu_render(cfg, scene, cams, "fp8")
    h8 = {k: v.cpu().numpy() for k, v in r8.hits(64).items()}
    r32, _, _, _ = gpu_render(cfg, scene, cams, "fp32")
    h32 = {k: v.cpu().numpy() for k, v in r32.hits(64).items()}
    assert np.array_equal(h8["count"], h32["count"])
    assert np.array_equal(h8["prim"], h32["prim"])


def test_fp8_full_size_stress_sampled_psnr():
    """The stress workload at full size (1080p x 4 views, K = 1024, width 128 x 4, 16-d
    features, S = 48): PSNR on pixels sampled uniformly over the views."""
    cfg = synth.CONFIGS["stress"]
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    r, out, _, _ = gpu_render(cfg, scene, cams, "fp8", hit_capacity=16.0)
    assert r.status() == 0
    pix = synth.sample_pixels(cfg, 600, seed=13)
    rgb_o, T_o, _ = oracle.render(cfg, scene, cams, pix=pix)
    idx = pixel_index(cfg.width, cfg.height, pix)
    rgb = out["rgb"].reshape(-1, 3)[idx]
    ps = psnr(rgb, rgb_o)
    print("fp8 stress full-size sampled psnr", ps)
    assert ps >= FP8_PSNR, ps


def test_fp8_backward_reported():
    """FP8 forward + BF16 recompute in the backward: gradients against the oracle (L2 loss)."""
    import torch
    from paper_2606_03877_gb300.render import Renderer
    cfg = synth.CONFIGS["prec"].replace(width=160, height=120, K=12, n_views=2)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    tgt = synth.perturb_scene(scene, cfg, 1)
    cur, _, _ = oracle.render(cfg, scene, cams)
    ref_img, _, _ = oracle.render(cfg, tgt, cams)
    g = (cur - ref_img).reshape(2, 120, 160, 3).astype(np.float32)
    r = Renderer(cfg, precision="fp8")
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    r.forward(d["centers"], d["scales"], d["quats"], packed, cams)
    got = r.backward(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    got = {k: v.cpu().numpy() for k, v in got.items()}
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g.reshape(-1, 3))
    errs = {k: rel_l2(got[k], ref[k]) for k in ("d_weights", "d_centers", "d_scales", "d_quats")}
    print("fp8 gradient rel-L2:", errs)
    for k, e in errs.items():
        assert e < 0.1, (k, errs)
