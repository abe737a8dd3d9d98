"""GPU parity of the feature slots (Sec. 3.4) against the FP64 oracle.

Each primitive carries four slot embeddings e_k in R^C after its MLP parameters; a hit's feature
f = sum_k softmax_k(a_k . u) e_k is composited with the hit's weight into F_slot, returned after
the MLP's own feature outputs. Bars: max |error| <= 1e-4 on F_slot and relative L2 <= 1e-3 per
gradient group (FP32 path); with the BF16 MLP the slot map inherits the BF16 compositing weights
and is held to relative L2 <= 1e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import synth
from paper_2606_03877_gb300.render import Renderer

from helpers import gpu_render, rel_l2, scaled_scene, to_dev

pytestmark = pytest.mark.gpu

BASE = synth.CONFIGS["contact"]


def _fwd(cfg, scene, cams, precision="fp32", tol=1e-4):
    r, out, _, _ = gpu_render(cfg, scene, cams, precision)
    assert r.status() == 0
    rgb_o, T_o, F_o = oracle.render(cfg, scene, cams)
    FT = cfg.feat_dim + cfg.slot_dim
    f = out["feat"].reshape(-1, FT)
    assert f.shape == F_o.shape
    if precision == "fp32":
        e = float(np.abs(f - F_o).max())
        assert e < tol, e
        assert float(np.abs(out["rgb"].reshape(-1, 3) - rgb_o).max()) < tol
    else:
        e = rel_l2(f[:, cfg.feat_dim:], F_o[:, cfg.feat_dim:])
        assert e < 1e-2, e
    assert float(np.abs(F_o[:, cfg.feat_dim:]).max()) > 0.1  # the map is not empty
    return e


@pytest.mark.parametrize("contact,S,C", [(1, 1, 512), (0, 4, 64), (1, 1, 1024)])
def test_slots_forward_fp32(contact, S, C):
    cfg = BASE.replace(width=64, height=48, K=12, n_views=2, contact=contact, samples=S, slot_dim=C)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    print("slots fwd max err", _fwd(cfg, scene, cams))


def test_slots_after_mlp_features_unaligned_rows():
    """feat_dim = 3 MLP outputs before 8 slot channels: rows of 11 floats (scalar path)."""
    cfg = BASE.replace(width=48, height=40, K=10, n_views=1, feat_dim=3, slot_dim=8)
    scene = scaled_scene(cfg, 2, 2.0)
    _fwd(cfg, scene, synth.make_cameras(cfg, first_view_seed=2))


def test_slots_with_bf16_mlp():
    cfg = BASE.replace(width=64, height=48, K=12, n_views=1, contact=0, samples=8, hidden_width=64,
                       dir_freqs=4, slot_dim=128)
    scene = scaled_scene(cfg, 3, 2.0)
    print("slots bf16 rel-L2", _fwd(cfg, scene, synth.make_cameras(cfg, first_view_seed=3), "bf16"))


def test_slots_equal_embeddings_give_one_minus_transmittance():
    """A single primitive whose four slots are equal: F_slot = (1 - T) e at every pixel, with
    the GPU's own T (no early termination at these opacities)."""
    cfg = BASE.replace(width=40, height=32, K=1, n_views=1, slot_dim=16)
    scene = synth.make_scene(cfg, 4)
    scene["centers"] = np.zeros((1, 3), np.float32)
    scene["scales"] = np.full((1, 3), 0.7, np.float32)
    e = np.linspace(-1, 1, 16).astype(np.float32)
    scene["weights"] = scene["weights"].copy()
    scene["weights"][0, cfg.n_mlp_params:] = np.tile(e, 4)
    r, out, _, _ = gpu_render(cfg, scene, synth.make_cameras(cfg, first_view_seed=4), "fp32")
    T = out["trans"].reshape(-1).astype(np.float64)
    f = out["feat"].reshape(-1, 16).astype(np.float64)
    assert T.min() < 0.5
    assert np.abs(f - (1 - T)[:, None] * e[None, :]).max() < 2e-6


def _inside(cfg, cam):
    scene = scaled_scene(cfg, 5, 2.0)
    o, d = oracle.pixel_ray(cam, cam["width"] // 2, cam["height"] // 2)
    scene["centers"][0] = (o + np.array([0.21, -0.13, 0.0]) - 0.17 * d).astype(np.float32)
    scene["scales"][0] = np.array([0.9, 0.8, 1.0], np.float32)
    return scene


def test_slots_camera_inside_a_primitive():
    cfg = BASE.replace(width=48, height=40, K=10, n_views=1, slot_dim=32)
    cam = synth.make_cameras(cfg, first_view_seed=6)[0]
    _fwd(cfg, _inside(cfg, cam), [cam])


def _grad(cfg, scene, cams, tol=1e-3):
    """L = 1/2 |C - C*|^2 + 1/2 |F - F*|^2 with (C*, F*) the oracle render of the perturbed scene."""
    cur, _, Fc = oracle.render(cfg, scene, cams)
    tgt, _, Ft = oracle.render(cfg, synth.perturb_scene(scene, cfg, 1), cams)
    V, H, W = len(cams), cfg.height, cfg.width
    FT = cfg.feat_dim + cfg.slot_dim
    g = (cur - tgt).reshape(V, H, W, 3).astype(np.float32)
    gf = (Fc - Ft).reshape(V, H, W, FT).astype(np.float32)
    r = Renderer(cfg, precision="fp32")
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    r.forward(d["centers"], d["scales"], d["quats"], packed, cams)
    got = r.backward(torch.from_numpy(g).cuda(), None, torch.from_numpy(gf).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    got = {k: v.cpu().numpy() for k, v in got.items()}
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g.reshape(-1, 3), None,
                                 gf.reshape(-1, FT))
    P = cfg.n_mlp_params
    errs = {k: rel_l2(got[k], ref[k]) for k in ("d_centers", "d_scales", "d_quats")}
    errs["d_mlp"] = rel_l2(got["d_weights"][:, :P], ref["d_weights"][:, :P])
    errs["d_slots"] = rel_l2(got["d_weights"][:, P:], ref["d_weights"][:, P:])
    print("slots gradient rel-L2", errs)
    for k, e in errs.items():
        assert e < tol, (k, errs)
    assert np.linalg.norm(ref["d_weights"][:, P:]) > 0
    return errs


@pytest.mark.parametrize("contact,S,C", [(1, 1, 512), (0, 4, 64)])
def test_slots_gradients(contact, S, C):
    cfg = BASE.replace(width=64, height=48, K=10, n_views=2, contact=contact, samples=S, slot_dim=C)
    _grad(cfg, scaled_scene(cfg, 7, 2.0), synth.make_cameras(cfg, first_view_seed=7))


def test_slots_gradients_camera_inside_and_mlp_features():
    cfg = BASE.replace(width=48, height=40, K=10, n_views=1, feat_dim=2, slot_dim=16)
    cam = synth.make_cameras(cfg, first_view_seed=6)[0]
    _grad(cfg, _inside(cfg, cam), [cam])


def test_slots_gradient_of_embeddings_only_from_the_slot_map():
    """dL/dF_slot = 0: the embeddings get no gradient and the others equal the slot-free render."""
    cfg = BASE.replace(width=48, height=40, K=8, n_views=1, slot_dim=32)
    scene = scaled_scene(cfg, 8, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=8)
    g = torch.from_numpy(synth.make_grad((1, 40, 48, 3), seed=8)).cuda()
    res = []
    for c, sc in ((cfg, scene), (cfg.replace(slot_dim=0), dict(scene, weights=scene["weights"][:, :cfg.n_mlp_params]))):
        r = Renderer(c, precision="fp32")
        d = to_dev(sc)
        r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
        gf = torch.zeros(1, 40, 48, c.slot_dim, device="cuda") if c.slot_dim else None
        out = r.backward(g, None, gf)
        torch.cuda.synchronize()
        res.append({k: v.cpu().numpy() for k, v in out.items()})
    P = cfg.n_mlp_params
    assert float(np.abs(res[0]["d_weights"][:, P:]).max()) == 0.0
    assert rel_l2(res[0]["d_weights"][:, :P], res[1]["d_weights"]) < 1e-6
    for k in ("d_centers", "d_scales", "d_quats"):
        assert rel_l2(res[0][k], res[1][k]) < 1e-6, k


def test_slots_equal_embeddings_under_early_termination():
    """With early termination active (T_eps = 0.3) the slot map uses the same hits and weights
    as the colour composite: four equal slots give F = (1 - T) e with the GPU's own T."""
    cfg = BASE.replace(width=40, height=32, K=6, n_views=1, slot_dim=8)
    scene = synth.make_scene(cfg, 9)
    scene["scales"] = (scene["scales"] * 4.0).astype(np.float32)
    e = np.linspace(-1, 1, 8).astype(np.float32)
    scene["weights"] = scene["weights"].copy()
    scene["weights"][:, cfg.n_mlp_params:] = np.tile(e, 4)[None, :]
    r, out, _, _ = gpu_render(cfg, scene, synth.make_cameras(cfg, first_view_seed=9), "fp32", t_eps=0.3)
    T = out["trans"].reshape(-1).astype(np.float64)
    f = out["feat"].reshape(-1, 8).astype(np.float64)
    assert T.min() < 0.3  # termination fired on some rays
    assert np.abs(f - (1 - T)[:, None] * e[None, :]).max() < 2e-6


def test_slots_with_no_primitives():
    cfg = BASE.replace(width=24, height=16, K=0, n_views=1, slot_dim=16)
    scene = {"centers": np.zeros((0, 3), np.float32), "scales": np.zeros((0, 3), np.float32),
             "quats": np.zeros((0, 4), np.float32), "weights": np.zeros((0, cfg.n_params), np.float32)}
    r, out, d, packed = gpu_render(cfg, scene, synth.make_cameras(cfg), "fp32")
    assert r.status() == 0 and float(np.abs(out["feat"]).max()) == 0.0
    g = r.backward(torch.ones(1, 16, 24, 3, device="cuda"), None, torch.ones(1, 16, 24, 16, device="cuda"))
    torch.cuda.synchronize()
    assert r.status("scratch") == 0
