"""GPU parity of the tile-centre approximate ordering (Sec. 3.3, App. A.4) against the oracle.

With `tile_sort` every pixel composites its own hits in the order of max(0, t*) along the
virtual ray through the centre of its T x T tile (ties by primitive index). Hit lists must equal
the oracle's in that order (outside the tangency band); images and gradients are held to the
FP32 bars (max |error| 1e-4, relative L2 1e-3) and the BF16 bar (PSNR >= 45 dB) against the
oracle in the same mode. The image loss of the approximation against the exact order is
reported.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import synth
from paper_2606_03877_gb300.render import Renderer

from helpers import gpu_render, psnr, rel_l2, scaled_scene, to_dev

pytestmark = pytest.mark.gpu

BASE = synth.CONFIGS["prec"]


@pytest.mark.parametrize("T", [8, 16])
def test_tile_order_hit_lists(T):
    cfg = BASE.replace(width=64, height=48, K=40, n_views=1, tile_sort=T)
    scene = scaled_scene(cfg, 6, 3.0)
    cams = synth.make_cameras(cfg, first_view_seed=6)
    r, out, _, _ = gpu_render(cfg, scene, cams)
    h = {k: v.cpu().numpy() for k, v in r.hits(64).items()}
    n_hits = n_diff = 0
    for y in range(cfg.height):
        for x in range(cfg.width):
            ray = y * cfg.width + x
            m2, _ = oracle.ray_m2(scene, cams[0], x, y)
            if np.any(np.abs(m2 - 1.0) < 1e-6):
                continue
            oh = oracle.ray_hits(scene, cams[0], x, y, tile=T)
            n = int(h["count"][ray])
            assert list(h["prim"][ray, :n]) == list(oh["prim"]), (x, y)
            ox = oracle.ray_hits(scene, cams[0], x, y)
            n_diff += list(ox["prim"]) != list(oh["prim"])
            n_hits += n
    assert n_hits > 500
    print(f"T={T}: rays whose tile order differs from the exact one: {n_diff}")
    assert n_diff > 0


@pytest.mark.parametrize("T,precision", [(8, "fp32"), (16, "fp32"), (8, "bf16")])
def test_tile_order_image(T, precision):
    cfg = BASE.replace(width=96, height=72, K=32, n_views=2, tile_sort=T)
    scene = scaled_scene(cfg, 2, 2.5)
    cams = synth.make_cameras(cfg, first_view_seed=2)
    r, out, _, _ = gpu_render(cfg, scene, cams, precision)
    assert r.status() == 0
    rgb_o, T_o, _ = oracle.render(cfg, scene, cams)
    rgb = out["rgb"].reshape(-1, 3)
    if precision == "fp32":
        assert float(np.abs(rgb - rgb_o).max()) < 1e-4
        assert float(np.abs(out["trans"].reshape(-1) - T_o).max()) < 1e-4
    else:
        assert psnr(rgb, rgb_o) >= 45.0
    rgb_x, _, _ = oracle.render(cfg.replace(tile_sort=0), scene, cams)
    print(f"T={T} {precision}: PSNR of the tile order vs the exact order {psnr(rgb, rgb_x):.2f} dB")


def test_tile_order_gradients():
    cfg = BASE.replace(width=80, height=64, K=16, n_views=1, tile_sort=8)
    scene = scaled_scene(cfg, 3, 2.5)
    cams = synth.make_cameras(cfg, first_view_seed=3)
    cur, _, _ = oracle.render(cfg, scene, cams)
    tgt, _, _ = oracle.render(cfg, synth.perturb_scene(scene, cfg, 1), cams)
    g = (cur - tgt).reshape(1, cfg.height, cfg.width, 3).astype(np.float32)
    r = Renderer(cfg, precision="fp32")
    d = to_dev(scene)
    r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    got = r.backward(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g.reshape(-1, 3))
    errs = {k: rel_l2(got[k].cpu().numpy(), ref[k]) for k in ("d_weights", "d_centers", "d_scales", "d_quats")}
    print("tile-order gradient rel-L2", errs)
    for k, e in errs.items():
        assert e < 1e-3, (k, errs)


def test_tile_order_loss_on_the_precision_workload_sampled():
    """1080p x 8 views, K = 256, 8 x 8 tiles: PSNR of the approximate (tile-centre) order against
    the exact oracle, and of the GPU tile-order image against the oracle in the same mode."""
    cfg = BASE.replace(tile_sort=8)
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    r, out, _, _ = gpu_render(cfg, scene, cams, "bf16")
    assert r.status() == 0
    pix = synth.sample_pixels(cfg, 4000, seed=31)
    idx = pix[:, 0].astype(np.int64) * cfg.width * cfg.height + pix[:, 2] * cfg.width + pix[:, 1]
    rgb = out["rgb"].reshape(-1, 3)[idx]
    rgb_t, _, _ = oracle.render(cfg, scene, cams, pix=pix)
    rgb_x, _, _ = oracle.render(cfg.replace(tile_sort=0), scene, cams, pix=pix)
    p_same, p_exact = psnr(rgb, rgb_t), psnr(rgb, rgb_x)
    print(f"prec 1080p x 8, T = 8: PSNR vs oracle (tile order) {p_same:.2f} dB, vs exact order {p_exact:.2f} dB")
    assert p_same >= 45.0
