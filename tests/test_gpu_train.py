"""GPU parity of the training objective, the optimizer and the training step (Sec. 3.5,
App. A.4) against the FP64 oracle (oracle/train.py and the renderer oracle).

Bars: the loss value to 1e-5 relative, its gradient to 1e-4 relative L2 (FP32 window sums
against FP64), Adam to 1e-6 relative, and the training step's first moments (0.1 x the
gradient after one step) to the FP32 gradient bar of 1e-3 relative L2.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import train as otr
from paper_2606_03877_gb300 import _lib, synth
from paper_2606_03877_gb300.train import Trainer, tile_selection

from helpers import rel_l2, scaled_scene

pytestmark = pytest.mark.gpu


def _gpu_loss(rgb, tgt, lam, tile, mask, feat=None, ftgt=None):
    V, H, W, _ = rgb.shape
    F = 0 if feat is None else feat.shape[-1]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    m = None if mask is None else torch.from_numpy(mask.astype(np.uint8)).cuda()
    desc = _lib.loss_desc(V, H, W, tile, m, lam, F)
    ws = torch.empty(_lib.mlps_loss_workspace_size(desc), dtype=torch.uint8, device="cuda")
    d_rgb = torch.empty(V, H, W, 3, device="cuda")
    d_feat = torch.empty(V, H, W, F, device="cuda") if F else None
    out = torch.empty(5, device="cuda")
    _lib.mlps_loss(desc, dev(rgb), dev(tgt), None if feat is None else dev(feat), None if ftgt is None else dev(ftgt),
                   d_rgb, d_feat, out, ws, ws.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy(), d_rgb.cpu().numpy(), None if d_feat is None else d_feat.cpu().numpy()


@pytest.mark.parametrize("V,H,W,tile,frac,F", [(2, 45, 70, 8, 0.25, 0), (1, 33, 40, 16, 0.5, 6), (1, 20, 20, 8, 1.0, 0)])
def test_loss_matches_oracle(V, H, W, tile, frac, F):
    rng = np.random.RandomState(V * 100 + H)
    rgb = rng.uniform(0, 1, (V, H, W, 3))
    tgt = np.clip(rgb + rng.normal(0, 0.1, rgb.shape), 0, 1)
    mask = tile_selection(V, H, W, tile, frac, seed=H)
    feat = rng.normal(0, 1, (V, H, W, F)) if F else None
    ftgt = rng.normal(0, 1, (V, H, W, F)) if F else None
    out, g, gf = _gpu_loss(rgb, tgt, 0.2, tile, mask, feat, ftgt)
    L, parts, g_o, gf_o = otr.loss(rgb.astype(np.float32), tgt.astype(np.float32), 0.2, tile, mask,
                                   None if feat is None else feat.astype(np.float32),
                                   None if ftgt is None else ftgt.astype(np.float32))
    print("loss", out, L, parts)
    assert abs(out[0] - L) < 1e-5 * max(1.0, abs(L))
    assert abs(out[1] - parts["l1"]) < 1e-5 and abs(out[2] - parts["ssim"]) < 1e-5
    assert out[3] == parts["n"]
    assert rel_l2(g, g_o) < 1e-4, rel_l2(g, g_o)
    if F:
        assert abs(out[4] - parts["l_feat"]) < 1e-5 and rel_l2(gf, gf_o) < 1e-6


def test_loss_of_identical_images_is_zero():
    rgb = np.random.RandomState(1).uniform(0, 1, (1, 24, 40, 3))
    out, g, _ = _gpu_loss(rgb, rgb, 0.2, 8, None)
    assert abs(out[0]) < 1e-6 and abs(out[2] - 1.0) < 1e-6 and np.abs(g).max() < 1e-6


def test_adam_matches_oracle():
    rng = np.random.RandomState(2)
    sizes = [1000, 37, 300]
    host = []
    groups = []
    for k, n in enumerate(sizes):
        p = rng.normal(0, 1, n).astype(np.float32)
        g = rng.normal(0, 1, n).astype(np.float32)
        m = rng.normal(0, 0.1, n).astype(np.float32)
        v = np.abs(rng.normal(0, 0.1, n)).astype(np.float32)
        aux = np.exp(p).astype(np.float32) if k == 2 else None
        d = [torch.from_numpy(a).cuda() for a in (p, g, m, v)]
        da = torch.from_numpy(aux).cuda() if aux is not None else None
        groups.append(_lib.adam_group(d[0], d[1], d[2], d[3], [1e-3, 1e-4, 1e-2][k], aux=da, kind=1 if k == 2 else 0))
        host.append((p, g, m, v, aux, d, da))
    _lib.mlps_adam_step(groups, 0.9, 0.999, 1e-15, 3, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k, (p, g, m, v, aux, d, da) in enumerate(host):
        # the kernel takes the hyper-parameters as FP32 values; give the oracle the same numbers
        f = lambda x: float(np.float32(x))
        res = otr.adam(p, g, m, v, 3, f([1e-3, 1e-4, 1e-2][k]), f(0.9), f(0.999), f(1e-15),
                       log_param=(k == 2), aux=aux)
        assert np.allclose(d[0].cpu().numpy(), res[0], rtol=2e-6, atol=1e-7), k
        assert np.allclose(d[2].cpu().numpy(), res[1], rtol=2e-6, atol=1e-8), k
        assert np.allclose(d[3].cpu().numpy(), res[2], rtol=1e-5, atol=1e-9), k
        if k == 2:
            assert np.allclose(da.cpu().numpy(), res[3], rtol=1e-6), k


def _train_setup(slot_dim=0):
    cfg = synth.CONFIGS["contact"].replace(width=64, height=48, K=16, n_views=2, slot_dim=slot_dim)
    scene = scaled_scene(cfg, 1, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=1)
    target = synth.perturb_scene(scene, cfg, 3)
    rgb_t, _, f_t = oracle.render(cfg, target, cams)
    rgb_t = rgb_t.reshape(2, 48, 64, 3)
    f_t = None if f_t is None else f_t.reshape(2, 48, 64, slot_dim)
    return cfg, scene, cams, rgb_t, f_t


@pytest.mark.parametrize("slot_dim", [0, 16])
def test_training_step_matches_oracle_chain(slot_dim):
    """One step: GPU loss equals the oracle loss of the oracle render, and the first Adam moments
    (0.1 x the gradient of each group, log-scales through dL/ds * s) match the oracle's chain."""
    cfg, scene, cams, rgb_t, f_t = _train_setup(slot_dim)
    tr = Trainer(cfg, scene, precision="fp32")
    mask = tr.tile_mask(1, 2, 48, 64)
    out = tr.step(cams, torch.from_numpy(rgb_t.astype(np.float32)).cuda(),
                  None if f_t is None else torch.from_numpy(f_t.astype(np.float32)).cuda(), tile_mask=mask)
    torch.cuda.synchronize()
    assert tr.status() == 0
    loss = out.cpu().numpy()
    rgb_o, _, f_o = oracle.render(cfg, scene, cams)
    L, parts, g_rgb, g_f = otr.loss(rgb_o.reshape(2, 48, 64, 3), rgb_t, 0.2, 8, mask,
                                    None if f_o is None else f_o.reshape(2, 48, 64, slot_dim), f_t)
    assert abs(loss[0] - L) < 1e-4 * abs(L), (loss, L)
    ref = oracle.render_backward(cfg, scene, cams, oracle.all_pixels(cams), g_rgb.reshape(-1, 3), None,
                                 None if g_f is None else g_f.reshape(-1, slot_dim))
    want = {"weights": ref["d_weights"], "centers": ref["d_centers"], "quats": ref["d_quats"],
            "log_scales": ref["d_scales"] * scene["scales"].astype(np.float64)}
    for k, g in want.items():
        e = rel_l2(tr.m[k].cpu().numpy(), 0.1 * g)
        assert e < 1e-3, (k, e)


def test_training_reduces_the_loss():
    cfg, scene, cams, rgb_t, f_t = _train_setup(16)
    tr = Trainer(cfg, scene, precision="fp32")
    tgt = torch.from_numpy(rgb_t.astype(np.float32)).cuda()
    ft = torch.from_numpy(f_t.astype(np.float32)).cuda()
    full = np.ones((2, 6, 8), np.uint8)
    losses = [float(tr.step(cams, tgt, ft, tile_mask=full)[0])]
    for _ in range(40):
        tr.step(cams, tgt, ft)
    losses.append(float(tr.step(cams, tgt, ft, tile_mask=full)[0]))
    torch.cuda.synchronize()
    print("loss before / after 41 steps:", losses)
    assert tr.status() == 0 and losses[1] < 0.8 * losses[0]


def test_bf16_training_of_the_midpoint_model_reduces_the_loss():
    """The tensor-core path trains too: the 60-64x64x64-4 midpoint model (S = 16) in BF16."""
    cfg = synth.CONFIGS["prec"].replace(width=64, height=48, K=12, n_views=2, samples=16)
    scene = scaled_scene(cfg, 2, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=2)
    rgb_t, _, _ = oracle.render(cfg, synth.perturb_scene(scene, cfg, 4), cams)
    tgt = torch.from_numpy(rgb_t.reshape(2, 48, 64, 3).astype(np.float32)).cuda()
    tr = Trainer(cfg, scene, precision="bf16")
    full = np.ones((2, 6, 8), np.uint8)
    first = float(tr.step(cams, tgt, tile_mask=full)[0])
    for _ in range(40):
        tr.step(cams, tgt)
    last = float(tr.step(cams, tgt, tile_mask=full)[0])
    torch.cuda.synchronize()
    print("bf16 loss before / after 41 steps:", first, last)
    assert tr.status() == 0 and last < 0.8 * first
