"""GPU parity of the contact-point mode (Sec. 3.2, Eq. 2-4) against the FP64 oracle.

In this mode every hit is evaluated once, at the soft contact point p* = o + max(0, t*) d, and
the primitive's MLP reads gamma([d; delta]) with delta = mu - p*; the hit's alpha uses its chord
length. FP32 path bars: max |error| <= 1e-4 on colour and transmittance, and relative L2 <= 1e-3
per gradient group, the FP32 contract; tensor cores: PSNR >= 45 dB (BF16) / 38 dB (E4M3) and
gradients within relative L2 2e-2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import synth
from paper_2606_03877_gb300.render import Renderer

from helpers import gpu_render, pixel_index, rel_l2, scaled_scene, to_dev

pytestmark = pytest.mark.gpu

CONTACT = synth.CONFIGS["contact"]  # 72-32-32-4, L = 6 on d and on delta, S = 1


def _forward_check(cfg, scene, cams, pix=None, tol=1e-4):
    r, out, _, _ = gpu_render(cfg, scene, cams, "fp32")
    assert r.status() == 0
    rgb_o, T_o, F_o = oracle.render(cfg, scene, cams, pix=pix)
    rgb = out["rgb"].reshape(-1, 3)
    T = out["trans"].reshape(-1)
    if pix is not None:
        idx = pixel_index(cfg.width, cfg.height, pix)
        rgb, T = rgb[idx], T[idx]
    e_rgb = float(np.abs(rgb - rgb_o).max())
    e_T = float(np.abs(T - T_o).max())
    assert e_rgb < tol and e_T < tol, (e_rgb, e_T)
    assert float(T_o.min()) < 0.9  # the scene is hit
    if cfg.feat_dim:
        f = out["feat"].reshape(-1, cfg.feat_dim)
        if pix is not None:
            f = f[idx]
        assert float(np.abs(f - F_o).max()) < tol
    return e_rgb, e_T


def test_contact_paper_model_small():
    cfg = CONTACT.replace(width=96, height=72, K=24, n_views=2)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    print("contact fwd max err", _forward_check(cfg, scene, cams))


@pytest.mark.parametrize("xyzL,dirL,feat", [(0, 0, 0), (3, 2, 5), (6, 0, 0)])
def test_contact_encodings_and_features(xyzL, dirL, feat):
    cfg = CONTACT.replace(width=80, height=60, K=16, n_views=1, xyz_freqs=xyzL, dir_freqs=dirL,
                          feat_dim=feat, hidden_width=64 if feat else 32)
    scene = scaled_scene(cfg, 2, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=2)
    _forward_check(cfg, scene, cams)


def _inside_scene(cfg, cam):
    """Primitive 0 encloses the camera centre: most rays meet it with t* < 0 (delta = mu - o)."""
    scene = scaled_scene(cfg, 3, 2.0)
    o, d = oracle.pixel_ray(cam, cam["width"] // 2, cam["height"] // 2)
    scene["centers"][0] = (o + np.array([0.21, -0.13, 0.0]) - 0.17 * d).astype(np.float32)
    scene["scales"][0] = np.array([0.9, 0.8, 1.0], np.float32)
    return scene


def test_contact_camera_inside_a_primitive():
    cfg = CONTACT.replace(width=64, height=48, K=12, n_views=1)
    cam = synth.make_cameras(cfg, first_view_seed=4)[0]
    scene = _inside_scene(cfg, cam)
    neg = sum(oracle.ray_m2(scene, cam, x, y)[1][0] < 0 for x in range(0, 64, 8) for y in range(0, 48, 8))
    assert neg > 10
    _forward_check(cfg, scene, [cam])


def _grad_check(cfg, scene, cams, tol=1e-3):
    """L = 1/2 sum (C - C*)^2 with C* the oracle render of the scene perturbed with seed 1."""
    cur, _, _ = oracle.render(cfg, scene, cams)
    tgt, _, _ = oracle.render(cfg, synth.perturb_scene(scene, cfg, 1), cams)
    g = (cur - tgt).reshape(len(cams), cfg.height, cfg.width, 3).astype(np.float32)
    r = Renderer(cfg, precision="fp32")
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    r.forward(d["centers"], d["scales"], d["quats"], packed, cams)
    got = r.backward(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    got = {k: v.cpu().numpy() for k, v in got.items()}
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g.reshape(-1, 3))
    errs = {k: rel_l2(got[k], ref[k]) for k in ("d_weights", "d_centers", "d_scales", "d_quats")}
    print("contact gradient rel-L2", errs)
    for k, e in errs.items():
        assert e < tol, (k, errs)
    return errs


def test_contact_gradients_paper_model():
    cfg = CONTACT.replace(width=96, height=72, K=16, n_views=2)
    _grad_check(cfg, scaled_scene(cfg, 5, 2.0), synth.make_cameras(cfg, first_view_seed=5))


def test_contact_gradients_raw_delta_with_features():
    cfg = CONTACT.replace(width=64, height=48, K=10, n_views=1, xyz_freqs=0, dir_freqs=2,
                          feat_dim=3, hidden_width=64)
    _grad_check(cfg, scaled_scene(cfg, 6, 2.0), synth.make_cameras(cfg, first_view_seed=6))


def test_contact_gradients_camera_inside():
    cfg = CONTACT.replace(width=64, height=48, K=12, n_views=1)
    cam = synth.make_cameras(cfg, first_view_seed=4)[0]
    _grad_check(cfg, _inside_scene(cfg, cam), [cam])


def test_midpoint_mode_single_sample_gradients():
    """S = 1 without the contact input (one midpoint sample per hit at t*): the thread-per-
    interval reverse of the FP32 backward against the oracle."""
    cfg = CONTACT.replace(width=80, height=60, K=14, n_views=1, contact=0, xyz_freqs=4, dir_freqs=2)
    _grad_check(cfg, scaled_scene(cfg, 9, 2.0), synth.make_cameras(cfg, first_view_seed=9))


def test_contact_full_size_sampled():
    """1920 x 1080 x 8 views, K = 256 (the contact workload): colour and T on sampled pixels."""
    cfg = CONTACT
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    pix = synth.sample_pixels(cfg, 3000, seed=17)
    print("contact full-size sampled max err", _forward_check(cfg, scene, cams, pix=pix))


def test_contact_equals_midpoint_mode_when_the_mlp_ignores_its_input():
    """S = 1, W_0 = 0: both modes evaluate the same input-independent MLP once per hit, so the
    images are bit-identical and the pose gradients agree."""
    cfg = CONTACT.replace(width=64, height=48, K=12, n_views=1)
    scene = scaled_scene(cfg, 8, 2.0)
    n0 = cfg.layer_dims()[0][0] * cfg.layer_dims()[0][1]
    scene["weights"] = scene["weights"].copy()
    scene["weights"][:, :n0] = 0.0
    cams = synth.make_cameras(cfg, first_view_seed=8)
    g = torch.from_numpy(synth.make_grad((1, cfg.height, cfg.width, 3), seed=8)).cuda()
    res = []
    for c in (cfg, cfg.replace(contact=0)):
        r, o, _, _ = gpu_render(c, scene, cams, "fp32")
        gr = r.backward(g)
        torch.cuda.synchronize()
        assert r.status("scratch") == 0
        res.append((o, {k: v.cpu().numpy() for k, v in gr.items()}))
    (o1, g1), (o0, g0) = res
    assert np.array_equal(o1["rgb"], o0["rgb"]) and np.array_equal(o1["trans"], o0["trans"])
    for k in ("d_centers", "d_scales", "d_quats"):
        assert rel_l2(g1[k], g0[k]) < 1e-5, k
    assert rel_l2(g1["d_weights"][:, n0:], g0["d_weights"][:, n0:]) < 1e-5


def test_contact_differs_from_midpoint_sampling():
    """Same weights, S = 1: the contact input gamma([d; delta]) and the midpoint input
    gamma(x') then gamma(d) give different images (the mode switch reaches the kernels)."""
    cfg = CONTACT.replace(width=64, height=48, K=12, n_views=1)
    scene = scaled_scene(cfg, 7, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=7)
    _, o1, _, _ = gpu_render(cfg, scene, cams, "fp32")
    _, o0, _, _ = gpu_render(cfg.replace(contact=0), scene, cams, "fp32")
    assert float(np.abs(o1["rgb"] - o0["rgb"]).max()) > 1e-3
    assert np.array_equal(o1["trans"] < 1, o0["trans"] < 1)  # same hits


@pytest.mark.parametrize("precision,bar", [("bf16", 45.0), ("fp8", 38.0)])
def test_contact_tensor_core_forward(precision, bar):
    """The paper's 32-wide model on the tensor cores: hidden layers zero-padded to the 64-wide
    tiles, contact-point rows built in the tensor-core kernel. PSNR against the FP64 oracle."""
    from helpers import psnr
    cfg = CONTACT.replace(width=96, height=72, K=24, n_views=2)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    r, out, _, _ = gpu_render(cfg, scene, cams, precision)
    assert r.status() == 0
    rgb_o, T_o, _ = oracle.render(cfg, scene, cams)
    p = psnr(out["rgb"].reshape(-1, 3), rgb_o)
    print(f"contact {precision} forward PSNR {p:.1f} dB")
    assert p >= bar


def test_contact_tensor_core_full_size_sampled():
    from helpers import psnr
    cfg = CONTACT
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    r, out, _, _ = gpu_render(cfg, scene, cams, "bf16")
    assert r.status() == 0
    pix = synth.sample_pixels(cfg, 3000, seed=19)
    rgb_o, _, _ = oracle.render(cfg, scene, cams, pix=pix)
    idx = pixel_index(cfg.width, cfg.height, pix)
    p = psnr(out["rgb"].reshape(-1, 3)[idx], rgb_o)
    print(f"contact bf16 1080p x 8 sampled PSNR {p:.1f} dB")
    assert p >= 45.0


def _l2_loss_grad(cfg, scene, cams):
    """dL/dC of L = 1/2 |C - C*|^2 against the oracle render of the scene perturbed with seed 1."""
    cur, _, _ = oracle.render(cfg, scene, cams)
    tgt, _, _ = oracle.render(cfg, synth.perturb_scene(scene, cfg, 1), cams)
    return (cur - tgt).reshape(len(cams), cfg.height, cfg.width, 3).astype(np.float32)


def _tc_gradients(cfg, scene, cams, precision, g_rgb):
    r = Renderer(cfg, precision=precision)
    d = to_dev(scene)
    r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    got = r.backward(torch.from_numpy(g_rgb).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g_rgb.reshape(-1, 3))
    return {k: rel_l2(got[k].cpu().numpy(), ref[k]) for k in ("d_weights", "d_centers", "d_scales", "d_quats")}


def test_width32_midpoint_model_on_tensor_cores():
    """A 32-wide model without the contact input (3 -> 32 -> 32 -> 4, S = 16) through the padded
    tensor-core forward and backward: PSNR >= 45 dB, gradients within the BF16 bar of 2e-2."""
    from helpers import psnr
    cfg = synth.CONFIGS["pr1"].replace(width=160, height=120, K=12, n_views=2)
    scene = scaled_scene(cfg, 0, 2.0)
    cams = synth.make_cameras(cfg)
    r, out, d, packed = gpu_render(cfg, scene, cams, "bf16")
    rgb_o, _, _ = oracle.render(cfg, scene, cams)
    assert psnr(out["rgb"].reshape(-1, 3), rgb_o) >= 45.0
    errs = _tc_gradients(cfg, scene, cams, "bf16", _l2_loss_grad(cfg, scene, cams))
    print("width-32 midpoint model bf16 gradient rel-L2:", errs)
    for k, e in errs.items():
        assert e < 2e-2, (k, errs)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_contact_tensor_core_backward(precision):
    """The paper's model (72-32-32-4, contact-point input) backward on the tensor cores: the
    two-slab input, the contact chain of the pose gradient, the first layer's bias gradient
    through the constant-1 input column. E4M3 forward, then the BF16 recompute. L2 loss against
    the perturbed scene; every gradient group within the BF16 bar of 2e-2."""
    cfg = CONTACT.replace(width=160, height=120, K=12, n_views=2)
    scene = scaled_scene(cfg, 3, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=3)
    errs = _tc_gradients(cfg, scene, cams, precision, _l2_loss_grad(cfg, scene, cams))
    print(f"contact {precision} gradient rel-L2:", errs)
    for k, e in errs.items():
        assert e < 2e-2, (k, errs)


def test_contact_tensor_core_backward_camera_inside():
    """t* < 0 for the primitive around the camera: the clamp of Eq. 3 and its one-sided chain."""
    cfg = CONTACT.replace(width=160, height=120, K=12, n_views=1)
    cam = synth.make_cameras(cfg, first_view_seed=4)[0]
    scene = _inside_scene(cfg, cam)
    errs = _tc_gradients(cfg, scene, [cam], "bf16", _l2_loss_grad(cfg, scene, [cam]))
    print("contact bf16, camera inside, gradient rel-L2:", errs)
    for k, e in errs.items():
        assert e < 2e-2, (k, errs)


def test_contact_bf16_with_slots():
    cfg = CONTACT.replace(width=64, height=48, K=12, n_views=1, slot_dim=64)
    scene = scaled_scene(cfg, 2, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=2)
    r, out, _, _ = gpu_render(cfg, scene, cams, "bf16")
    assert r.status() == 0
    _, _, F_o = oracle.render(cfg, scene, cams)
    e = rel_l2(out["feat"].reshape(-1, 64), F_o)
    print("contact bf16 slot map rel-L2", e)
    assert e < 1e-2


def test_contact_bf16_with_slots_gradients():
    """The paper's model with feature slots on the tensor-core path: L2 loss on the image and the
    slot map against the perturbed scene; every group, slot embeddings included, within the
    BF16 bar of the oracle's reverse mode."""
    cfg = CONTACT.replace(width=64, height=48, K=12, n_views=1, slot_dim=64)
    scene = scaled_scene(cfg, 5, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=5)
    cur, _, Fc = oracle.render(cfg, scene, cams)
    tgt, _, Ft = oracle.render(cfg, synth.perturb_scene(scene, cfg, 1), cams)
    g = (cur - tgt).astype(np.float32)
    gF = (Fc - Ft).astype(np.float32)
    r = Renderer(cfg, precision="bf16")
    d = to_dev(scene)
    r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    got = r.backward(torch.from_numpy(g.reshape(1, 48, 64, 3)).cuda(), None,
                     torch.from_numpy(gF.reshape(1, 48, 64, 64)).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g, None, gF)
    errs = {k: rel_l2(got[k].cpu().numpy(), ref[k]) for k in ("d_weights", "d_centers", "d_scales", "d_quats")}
    print("contact + slots BF16 gradient rel-L2:", errs)
    for k, e in errs.items():
        assert e < 2e-2, (k, errs)
