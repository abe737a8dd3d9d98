"""Early termination that saves forward work (App. B.2): with early_stop_wave = k the MLP
forward runs in two depth waves (each ray's first k hits; then the later hits of the rays whose
composite has not stopped), so the intervals behind a ray's termination point are never
evaluated. The composite never reaches them either, so the image, the transmittance and the
gradients are those of the single-wave forward, bit for bit for the image."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import synth
from paper_2606_03877_gb300.render import Renderer

from helpers import rel_l2, scaled_scene, to_dev

pytestmark = pytest.mark.gpu

GROUPS = ["d_weights", "d_centers", "d_scales", "d_quats"]


def _cfg():
    return synth.CONFIGS["prec"].replace(width=64, height=48, K=16, n_views=2)


def _opaque(cfg, seed, shift=60.0):
    """Density pre-activations raised by `shift`: a ray's transmittance falls below 1e-6 inside
    its first interval."""
    sc = scaled_scene(cfg, seed, 2.5)
    w = sc["weights"].copy()
    w[:, cfg.n_params - cfg.output_dim + 3] += shift
    return dict(sc, weights=w)


def _run(cfg, scene, cams, precision, wave, g=None):
    r = Renderer(cfg, precision=precision, early_stop_wave=wave)
    d = to_dev(scene)
    out = r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    counts = r.wave_counts()
    grads = None
    if g is not None:
        grads = r.backward(torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert r.status() == 0 and r.status("scratch") == 0
    out = {k: v.clone() for k, v in out.items() if v is not None}
    return out, counts, (None if grads is None else {k: v.cpu().numpy() for k, v in grads.items()})


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("wave", [1, 2])
def test_waves_skip_terminated_intervals_and_change_no_output(precision, wave):
    cfg = _cfg()
    scene = _opaque(cfg, 41)
    cams = synth.make_cameras(cfg, first_view_seed=41)
    g = synth.make_grad((cfg.n_views, cfg.height, cfg.width, 3), seed=42)
    ref, (n_ref, e_ref), g_ref = _run(cfg, scene, cams, precision, 0, g)
    got, (n, evaluated), g_got = _run(cfg, scene, cams, precision, wave, g)
    print(precision, "wave", wave, "intervals", n, "evaluated", evaluated)
    assert e_ref == 0 and n == n_ref
    assert 0 < evaluated < (0.8 * n if wave == 1 else n)  # most rays here have 2-3 hits
    assert torch.equal(got["rgb"], ref["rgb"]) and torch.equal(got["trans"], ref["trans"])
    for k in GROUPS:
        assert rel_l2(g_got[k], g_ref[k]) < 1e-5, k


def test_waves_fp32_image_matches_the_oracle():
    cfg = _cfg()
    scene = _opaque(cfg, 43)
    cams = synth.make_cameras(cfg, first_view_seed=43)
    got, (n, evaluated), _ = _run(cfg, scene, cams, "fp32", 1)
    rgb_o, T_o, _ = oracle.render(cfg, scene, cams)
    assert evaluated < n
    assert np.abs(got["rgb"].cpu().numpy().reshape(-1, 3) - rgb_o).max() < 1e-4
    assert np.abs(got["trans"].cpu().numpy().reshape(-1) - T_o).max() < 1e-4


def test_waves_on_a_transparent_scene_evaluate_everything():
    """Nothing terminates on the semi-transparent benchmark scenes: the two waves together
    evaluate every interval once."""
    cfg = _cfg()
    scene = scaled_scene(cfg, 45, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=45)
    ref, _, _ = _run(cfg, scene, cams, "bf16", 0)
    got, (n, evaluated), _ = _run(cfg, scene, cams, "bf16", 1)
    assert evaluated == n > 0
    assert torch.equal(got["rgb"], ref["rgb"])
