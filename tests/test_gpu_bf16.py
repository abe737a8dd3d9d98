"""GPU parity of the BF16 tensor-core (tcgen05) MLP path against the FP64 oracle.

Bar: PSNR >= 45 dB per view (peak 1, all pixels x 3 channels) for the colour image, the
BF16 contract; hit lists are the same as the FP32 path's (the geometry does not depend on the
MLP precision). Segment lengths S = 16, 32 and 48 exercise interval composites inside one warp,
exactly one warp, and across warps.
"""
import numpy as np
import pytest

import oracle
from paper_2606_03877_gb300 import synth

from helpers import gpu_render, pixel_index, psnr, scaled_scene

pytestmark = pytest.mark.gpu


def _psnr_views(cfg, scene, cams, **kw):
    r, out, _, _ = gpu_render(cfg, scene, cams, "bf16", **kw)
    assert r.status() == 0
    rgb_o, T_o, F_o = oracle.render(cfg, scene, cams)
    n = cfg.width * cfg.height
    rgb = out["rgb"].reshape(-1, 3)
    T = out["trans"].reshape(-1)
    ps = [psnr(rgb[v * n:(v + 1) * n], rgb_o[v * n:(v + 1) * n]) for v in range(len(cams))]
    return ps, r, out, (rgb_o, T_o, F_o)


def test_bf16_small_prec_shape():
    cfg = synth.CONFIGS["prec"].replace(width=64, height=48, K=12, n_views=1)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    ps, r, out, (rgb_o, T_o, _) = _psnr_views(cfg, scene, cams)
    print("psnr", ps, "max|dT|", np.abs(out["trans"].reshape(-1) - T_o).max())
    assert min(ps) >= 45.0, ps


@pytest.mark.parametrize("S", [16, 32, 48])
def test_bf16_segment_lengths(S):
    cfg = synth.CONFIGS["prec"].replace(width=100, height=75, K=24, n_views=2, samples=S)
    scene = scaled_scene(cfg, 2, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=2)
    ps, r, out, (rgb_o, T_o, _) = _psnr_views(cfg, scene, cams)
    assert min(ps) >= 45.0, ps
    assert np.abs(out["trans"].reshape(-1) - T_o).max() < 2e-2


def test_bf16_wide_mlp_with_features():
    cfg = synth.CONFIGS["stress"].replace(width=80, height=60, K=20, n_views=1)
    scene = scaled_scene(cfg, 3, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=3)
    ps, r, out, (rgb_o, T_o, F_o) = _psnr_views(cfg, scene, cams)
    assert min(ps) >= 45.0, ps
    f = out["feat"].reshape(-1, cfg.feat_dim)
    rel = np.linalg.norm(f - F_o) / max(np.linalg.norm(F_o), 1e-12)
    assert rel < 2e-2, rel


def test_bf16_hits_identical_to_fp32_path():
    cfg = synth.CONFIGS["prec"].replace(width=96, height=64, K=32, n_views=1)
    scene = scaled_scene(cfg, 4, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=4)
    r16, _, _, _ = gpu_render(cfg, scene, cams, "bf16")
    h16 = {k: v.cpu().numpy() for k, v in r16.hits(64).items()}
    r32, _, _, _ = gpu_render(cfg, scene, cams, "fp32")
    h32 = {k: v.cpu().numpy() for k, v in r32.hits(64).items()}
    assert np.array_equal(h16["count"], h32["count"])
    assert np.array_equal(h16["prim"], h32["prim"])


def test_bf16_full_size_prec_sampled_psnr():
    cfg = synth.CONFIGS["prec"]
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    r, out, _, _ = gpu_render(cfg, scene, cams, "bf16")
    assert r.status() == 0
    pix = synth.sample_pixels(cfg, 2000, seed=12)
    rgb_o, T_o, _ = oracle.render(cfg, scene, cams, pix=pix)
    idx = pixel_index(cfg.width, cfg.height, pix)
    rgb = out["rgb"].reshape(-1, 3)[idx]
    for v in range(cfg.n_views):
        sel = pix[:, 0] == v
        assert psnr(rgb[sel], rgb_o[sel]) >= 45.0, v


# ------------------------------------------------------------------------------------------
# Backward (tensor-core dgrad / wgrad with TMEM accumulation); bar: relative L2 <= 2e-2 per
# parameter group against the oracle's reverse mode.

def _bf16_grads(cfg, scene, cams, g_rgb, g_T=None, g_F=None):
    import torch
    from paper_2606_03877_gb300.render import Renderer
    from helpers import to_dev
    r = Renderer(cfg, precision="bf16")
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    r.forward(d["centers"], d["scales"], d["quats"], packed, cams)
    g = r.backward(torch.from_numpy(g_rgb).cuda(), None if g_T is None else torch.from_numpy(g_T).cuda(),
                   None if g_F is None else torch.from_numpy(g_F).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    return {k: v.cpu().numpy() for k, v in g.items()}


def _check_bf16_grads(cfg, scene, cams, g_rgb, g_T=None, g_F=None, tol=2e-2):
    from helpers import rel_l2
    got = _bf16_grads(cfg, scene, cams, g_rgb, g_T, g_F)
    pix = oracle.all_pixels(cams)
    ref = oracle.render_backward(cfg, scene, cams, pix, g_rgb.reshape(-1, 3),
                                 None if g_T is None else g_T.reshape(-1),
                                 None if g_F is None else g_F.reshape(-1, cfg.feat_dim))
    errs = {k: rel_l2(got[k], ref[k]) for k in ("d_weights", "d_centers", "d_scales", "d_quats")}
    print("bf16 gradient rel-L2:", errs)
    for k, e in errs.items():
        assert e < tol, (k, errs)
    return errs


def _l2_grad(cfg, scene, cams, pix=None):
    """dL/dC of L = 1/2 sum (C - C*)^2 with C* the oracle render of the scene perturbed with
    seed 1 (the differentiation workload's loss); C from the oracle as well."""
    tgt = synth.perturb_scene(scene, cfg, 1)
    if pix is None:
        cur, _, _ = oracle.render(cfg, scene, cams)
        ref, _, _ = oracle.render(cfg, tgt, cams)
        return (cur - ref).reshape(len(cams), cfg.height, cfg.width, 3).astype(np.float32)
    cur, _, _ = oracle.render(cfg, scene, cams, pix=pix)
    ref, _, _ = oracle.render(cfg, tgt, cams, pix=pix)
    return (cur - ref).astype(np.float32)


def _no_flip(scene, cfg, bias=3.0):
    """Hidden biases +bias: every ReLU stays active, so BF16 rounding cannot flip a mask."""
    w = scene["weights"].astype(np.float64).copy()
    off = 0
    dims = cfg.layer_dims()
    for li, (fi, fo) in enumerate(dims):
        if li < len(dims) - 1:
            w[:, off + fi * fo: off + fi * fo + fo] = bias
        off += fi * fo + fo
    return dict(scene, weights=w.astype(np.float32))


@pytest.mark.parametrize("S", [32, 16, 48])
def test_bf16_backward_l2_loss(S):
    # ReLU mask flips make the BF16 gradient error shrink with the pixels per primitive; this
    # size (~40k rays, K = 12) keeps the oracle's reverse mode at a few seconds.
    cfg = synth.CONFIGS["prec"].replace(width=160, height=120, K=12, n_views=2, samples=S)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    _check_bf16_grads(cfg, scene, cams, _l2_grad(cfg, scene, cams))


@pytest.mark.parametrize("S", [32, 16, 48])
def test_bf16_backward_without_mask_flips_random_gradient(S):
    """With every ReLU active the BF16 backward is a rounding-only approximation, held to the
    BF16 bar of 2e-2 even with random dL/dC and dL/dT, which cancel heavily in the pose sums;
    a wrong term in any formula gives O(1) errors."""
    cfg = synth.CONFIGS["prec"].replace(width=64, height=48, K=12, n_views=2, samples=S)
    scene = _no_flip(scaled_scene(cfg, 1, 2.0), cfg)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    g = synth.make_grad((2, 48, 64, 3), seed=5)
    gT = synth.make_grad((2, 48, 64), seed=6)
    _check_bf16_grads(cfg, scene, cams, g, gT, tol=2e-2)


def test_bf16_backward_random_gradient_reported():
    """Report only, not a parity claim: random dL/dC has no image loss behind it, so nothing
    averages the O(1) per-unit changes of ReLU masks that BF16 rounding flips (~3 % on the
    first layer, ~7 % on quaternions at this size). The bound of 0.1 only catches a broken
    formula; the BF16 bar of 2e-2 is held by the L2-loss tests, including the full-size one."""
    cfg = synth.CONFIGS["prec"].replace(width=64, height=48, K=12, n_views=2)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    g = synth.make_grad((2, 48, 64, 3), seed=5)
    _check_bf16_grads(cfg, scene, cams, g, tol=0.1)


def test_bf16_backward_feature_head():
    cfg = synth.SceneConfig("f", 40, 32, 10, 1, 6, 4, 64, 2, 8, 16)
    scene = _no_flip(scaled_scene(cfg, 7, 2.0), cfg)
    cams = synth.make_cameras(cfg, first_view_seed=7)
    g = synth.make_grad((1, 32, 40, 3), seed=1)
    gF = synth.make_grad((1, 32, 40, 8), seed=2)
    _check_bf16_grads(cfg, scene, cams, g, None, gF, tol=2e-2)


def test_bf16_backward_many_chunks_per_primitive():
    """Enough hits per primitive that each block accumulates many chunks (and several
    primitive segments) in tensor memory before flushing; L2 loss on sampled pixels."""
    cfg = synth.CONFIGS["prec"].replace(width=320, height=240, K=6, n_views=2)
    scene = scaled_scene(cfg, 11, 3.0)
    cams = synth.make_cameras(cfg, first_view_seed=11)
    pix = synth.sample_pixels(cfg, 1500, seed=4)
    g = np.zeros((2, 240, 320, 3), np.float32)
    idx = pixel_index(cfg.width, cfg.height, pix)
    g.reshape(-1, 3)[idx] = _l2_grad(cfg, scene, cams, pix)
    from helpers import rel_l2
    got = _bf16_grads(cfg, scene, cams, g)
    ref = oracle.render_backward(cfg, scene, cams, pix, g.reshape(-1, 3)[idx])
    for k in ("d_weights", "d_centers", "d_scales", "d_quats"):
        assert rel_l2(got[k], ref[k]) < 2e-2, k
