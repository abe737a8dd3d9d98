"""GPU parity of the forward path (FP32 SIMT MLP) against the FP64 oracle, through the C ABI.

Bars (from the method's FP32 contract): pixel channels and final transmittance within max-abs
1e-4 of the oracle; hit lists (primitive order) identical to the oracle's on every ray that is
not within 1e-6 of tangency (|1 - m^2| < 1e-6, m^2 in FP64), such rays counted; every oracle
hit's primitive present in the GPU tile list of its pixel (conservative binning).
"""
import numpy as np
import pytest

import oracle
from paper_2606_03877_gb300 import synth

from helpers import gpu_render, pixel_index, scaled_scene

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _compare_full(cfg, scene, cams, precision="fp32", tol=TOL, **kw):
    r, out, _, _ = gpu_render(cfg, scene, cams, precision, **kw)
    assert r.status() == 0
    rgb_o, T_o, F_o = oracle.render(cfg, scene, cams)
    rgb = out["rgb"].reshape(-1, 3)
    T = out["trans"].reshape(-1)
    err = np.abs(rgb - rgb_o).max()
    errT = np.abs(T - T_o).max()
    assert err < tol and errT < tol, (err, errT)
    if cfg.feat_dim:
        errF = np.abs(out["feat"].reshape(-1, cfg.feat_dim) - F_o).max()
        assert errF < tol * 10, errF
    return r, out, (rgb_o, T_o)


def test_pr1_forward_matches_oracle():
    cfg = synth.CONFIGS["pr1"]
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    r, out, (rgb_o, T_o) = _compare_full(cfg, scene, cams)
    assert (T_o < 1).sum() > 50


@pytest.mark.parametrize("W,H,K,V,seed", [(100, 75, 24, 2, 1), (37, 53, 40, 1, 2), (16, 16, 5, 1, 3)])
def test_prec_shape_forward_ragged(W, H, K, V, seed):
    """Prec-shaped MLP (60 -> 64x3 -> 4, S = 32) on ragged images spanning several tiles."""
    cfg = synth.CONFIGS["prec"].replace(width=W, height=H, K=K, n_views=V)
    scene = scaled_scene(cfg, seed, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=seed)
    _compare_full(cfg, scene, cams)


def test_feature_head_and_wide_mlp():
    """Stress-shaped MLP (width 128, 4 hidden layers, 16-d linear feature head, S = 48)."""
    cfg = synth.CONFIGS["stress"].replace(width=48, height=40, K=12, n_views=1)
    scene = scaled_scene(cfg, 4, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=5)
    _compare_full(cfg, scene, cams)


def test_hit_lists_exact_outside_tangency_band():
    cfg = synth.CONFIGS["prec"].replace(width=96, height=80, K=48, n_views=1)
    scene = scaled_scene(cfg, 6, 2.5)
    cams = synth.make_cameras(cfg, first_view_seed=6)
    r, out, _, _ = gpu_render(cfg, scene, cams)
    h = {k: v.cpu().numpy() for k, v in r.hits(64).items()}
    n_band = 0
    n_hits = 0
    for y in range(cfg.height):
        for x in range(cfg.width):
            ray = y * cfg.width + x
            oh = oracle.ray_hits(scene, cams[0], x, y)
            m2, _ = oracle.ray_m2(scene, cams[0], x, y)
            if np.any(np.abs(m2 - 1.0) < 1e-6):
                n_band += 1
                continue
            n = int(h["count"][ray])
            assert n == len(oh["prim"]), (x, y, n, oh["prim"])
            assert list(h["prim"][ray, :n]) == list(oh["prim"]), (x, y)
            assert np.allclose(h["t0"][ray, :n], oh["t0"], atol=1e-5)
            assert np.allclose(h["t1"][ray, :n], oh["t1"], atol=1e-5)
            n_hits += n
    assert n_hits > 500
    print(f"rays within 1e-6 of tangency (excluded): {n_band}")


def test_hit_lists_full_size_sampled_rays():
    """The benchmark's launch (1080p x 8 views, K = 256): on 3000 rays sampled over the views
    the hit lists equal the oracle's (same primitives, same order, chord ends within 1e-5)
    except on rays with a primitive within 1e-6 of tangency, which are counted and excluded."""
    cfg = synth.CONFIGS["prec"]
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    r, out, _, _ = gpu_render(cfg, scene, cams)
    h = r.hits(32)
    pix = synth.sample_pixels(cfg, 3000, seed=77)
    import torch
    idx = torch.from_numpy(pixel_index(cfg.width, cfg.height, pix)).cuda()
    count = h["count"][idx].cpu().numpy()
    prim, t0, t1 = (h[k][idx].cpu().numpy() for k in ("prim", "t0", "t1"))
    del h
    n_band = n_hits = 0
    for j, (v, x, y) in enumerate(pix):
        m2, _ = oracle.ray_m2(scene, cams[v], int(x), int(y))
        if np.any(np.abs(m2 - 1.0) < 1e-6):
            n_band += 1
            continue
        oh = oracle.ray_hits(scene, cams[v], int(x), int(y))
        n = int(count[j])
        assert n == len(oh["prim"]) and n <= 32, (v, x, y, n, oh["prim"])
        assert list(prim[j, :n]) == list(oh["prim"]), (v, x, y)
        assert np.allclose(t0[j, :n], oh["t0"], atol=1e-5) and np.allclose(t1[j, :n], oh["t1"], atol=1e-5)
        n_hits += n
    assert n_hits > 3000
    print(f"full size: {len(pix)} rays, {n_hits} hits identical; {n_band} rays within 1e-6 of tangency excluded")


def test_tile_binning_is_conservative():
    cfg = synth.CONFIGS["prec"].replace(width=120, height=90, K=64, n_views=1)
    scene = scaled_scene(cfg, 8, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=8)
    r, out, _, _ = gpu_render(cfg, scene, cams)
    count, lst = (t.cpu().numpy() for t in r.tiles())
    ntx = (cfg.width + 15) // 16
    checked = 0
    for y in range(0, cfg.height, 2):
        for x in range(0, cfg.width, 2):
            oh = oracle.ray_hits(scene, cams[0], x, y)
            t = (y // 16) * ntx + x // 16
            cands = set(lst[t, :count[t]].tolist())
            for p in oh["prim"]:
                assert int(p) in cands, (x, y, p)
                checked += 1
    assert checked > 100


def test_empty_scene_and_degenerate_cases():
    cfg = synth.CONFIGS["prec"].replace(width=33, height=17, K=0, n_views=1)
    scene = {"centers": np.zeros((0, 3), np.float32), "scales": np.ones((0, 3), np.float32),
             "quats": np.zeros((0, 4), np.float32), "weights": np.zeros((0, cfg.n_params), np.float32)}
    cams = synth.make_cameras(cfg)
    r, out, _, _ = gpu_render(cfg, scene, cams)
    assert np.all(out["rgb"] == 0) and np.all(out["trans"] == 1)
    assert r.hit_count() == 0
    # a primitive behind the camera and one containing the camera (near clipping)
    cfg1 = synth.CONFIGS["prec"].replace(width=24, height=20, K=2, n_views=1)
    sc = synth.make_scene(cfg1, 3)
    cam = synth.make_camera(24, 20, 2, near=0.05)
    P = np.asarray(cam["w2c"], np.float64).reshape(3, 4)
    o = -P[:, :3].T @ P[:, 3]
    sc["centers"] = np.stack([o * 1.5, o * 0.98]).astype(np.float32)  # behind; around the camera
    sc["scales"] = np.array([[0.3, 0.3, 0.3], [0.5, 0.4, 0.45]], np.float32)
    _compare_full(cfg1, sc, [cam])


def test_capacity_overflow_is_reported():
    cfg = synth.CONFIGS["prec"].replace(width=48, height=48, K=30, n_views=1)
    scene = scaled_scene(cfg, 9, 3.0)
    cams = synth.make_cameras(cfg, first_view_seed=9)
    r, out, _, _ = gpu_render(cfg, scene, cams, max_hits=1)
    assert r.status() == 4  # MLPS_ERR_CAPACITY_OVERFLOW
    r2, out2, _, _ = gpu_render(cfg, scene, cams, hit_capacity=0.01)
    assert r2.status() == 4
    # the context stays usable: a clean render afterwards
    _compare_full(cfg, scene, cams)


def test_invalid_arguments_rejected():
    from paper_2606_03877_gb300 import _lib
    from paper_2606_03877_gb300.render import make_config
    cfg = make_config(synth.CONFIGS["prec"])
    cfg.samples = 0
    assert _lib.mlps_check_config(cfg) == _lib.MLPS_ERR_INVALID_ARGUMENT
    cfg = make_config(synth.CONFIGS["prec"])
    cams = _lib.cameras(synth.make_cameras(synth.CONFIGS["prec"].replace(n_views=1)))
    with pytest.raises(_lib.MlpsError) as e:
        _lib.mlps_render_forward(cfg, _lib.make_scene(4, 0, 0, 0, 0), cams, 1, 0, 0, 0, 0, 0, 0, 0, 0)
    assert e.value.status == _lib.MLPS_ERR_INVALID_ARGUMENT


def test_full_size_prec_sampled_pixels():
    """Full 1080p x 8 views, K = 256 (the benchmark's launch configuration), sampled pixels."""
    cfg = synth.CONFIGS["prec"]
    scene = synth.make_scene(cfg, 0)
    cams = synth.make_cameras(cfg)
    r, out, _, _ = gpu_render(cfg, scene, cams)
    assert r.status() == 0
    pix = synth.sample_pixels(cfg, 400, seed=11)
    rgb_o, T_o, _ = oracle.render(cfg, scene, cams, pix=pix)
    idx = pixel_index(cfg.width, cfg.height, pix)
    rgb = out["rgb"].reshape(-1, 3)[idx]
    T = out["trans"].reshape(-1)[idx]
    assert np.abs(rgb - rgb_o).max() < TOL and np.abs(T - T_o).max() < TOL
    assert (T_o < 1).sum() > 100


def test_non_finite_and_degenerate_primitives_are_skipped_and_reported():
    """A NaN centre, a zero scale and a zero quaternion make their primitives invalid: the
    device status reports MLPS_ERR_NONFINITE and the image is the render of the valid ones."""
    cfg = synth.CONFIGS["prec"].replace(width=40, height=32, K=9, n_views=1)
    scene = scaled_scene(cfg, 12, 2.5)
    bad = {k: v.copy() for k, v in scene.items()}
    bad["centers"][1, 0] = np.nan
    bad["scales"][4, 2] = 0.0
    bad["quats"][7] = 0.0
    cams = synth.make_cameras(cfg, first_view_seed=12)
    r, out, _, _ = gpu_render(cfg, bad, cams)
    assert r.status() == 6  # MLPS_ERR_NONFINITE
    keep = [i for i in range(cfg.K) if i not in (1, 4, 7)]
    valid = {k: v[keep] for k, v in scene.items()}
    rgb_o, T_o, _ = oracle.render(cfg.replace(K=len(keep)), valid, cams)
    assert np.abs(out["rgb"].reshape(-1, 3) - rgb_o).max() < 1e-4
    assert np.abs(out["trans"].reshape(-1) - T_o).max() < 1e-4
