"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: closed forms, an
independent restatement with different formulas (quadratic roots instead of the closest-point
form, library rotations, product-form transmittance), numerical quadrature of the continuous
operator, invariances, printed numbers of the paper, and central finite differences.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.spatial.transform import Rotation

import oracle
from paper_2606_03877_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cam(width=24, height=18, seed=0, **kw):
    return synth.make_camera(width, height, seed, **kw)


def _layout(cfg):
    """(W slice, b slice) per layer of the canonical layout."""
    out, off = [], 0
    for fi, fo in cfg.layer_dims():
        out.append((slice(off, off + fi * fo), slice(off + fi * fo, off + fi * fo + fo), fi, fo))
        off += fi * fo + fo
    return out


def _constant_weights(cfg, K, rgb_bias, sigma_bias, feat_bias=None):
    """All weights zero; last-layer bias gives constant raw outputs."""
    w = np.zeros((K, cfg.n_params))
    _, bs, _, _ = _layout(cfg)[-1]
    for p in range(K):
        w[p, bs][0:3] = rgb_bias[p]
        w[p, bs][3] = sigma_bias[p]
        if feat_bias is not None:
            w[p, bs][4:] = feat_bias[p]
    return w


def _ray_np(cam, x, y):
    """Pixel ray from the pinhole model (independent restatement)."""
    P = np.asarray(cam["w2c"], dtype=np.float64).reshape(3, 4)
    R, t = P[:, :3], P[:, 3]
    o = -R.T @ t
    dc = np.array([(x + 0.5 - cam["cx"]) / cam["fx"], (y + 0.5 - cam["cy"]) / cam["fy"], 1.0])
    d = R.T @ dc
    return o, d / np.linalg.norm(d)


def _rot(q):
    w, x, y, z = [float(v) for v in q]
    return Rotation.from_quat([x, y, z, w]).as_matrix()  # scipy is scalar-last; normalises


def _ray_np_uv(cam, u, v):
    """Ray through the image point (u, v) (pixel centres at x + 1/2)."""
    P = np.asarray(cam["w2c"], dtype=np.float64).reshape(3, 4)
    R, t = P[:, :3], P[:, 3]
    dc = np.array([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], 1.0])
    d = R.T @ dc
    return -R.T @ t, d / np.linalg.norm(d)


def _np_hits(scene, cam, x, y, tile=0):
    """Hits by the quadratic-formula roots of (o+td-mu)^T Lambda (o+td-mu) = 1 (Eq. 1-2). With
    tile > 0 they are ordered by max(0, t*) of the ray through the tile centre (Sec. 3.3)."""
    o, d = _ray_np(cam, x, y)
    if tile:
        _, dcen = _ray_np_uv(cam, (x // tile) * tile + tile / 2.0, (y // tile) * tile + tile / 2.0)
    hits = []
    for i in range(scene["centers"].shape[0]):
        mu = scene["centers"][i].astype(np.float64)
        s = scene["scales"][i].astype(np.float64)
        R = _rot(scene["quats"][i])
        Lam = R @ np.diag(1.0 / s ** 2) @ R.T
        A = d @ Lam @ d
        B = 2.0 * d @ Lam @ (o - mu)
        C = (o - mu) @ Lam @ (o - mu) - 1.0
        disc = B * B - 4 * A * C
        if disc <= 0:
            continue
        r0 = (-B - math.sqrt(disc)) / (2 * A)
        r1 = (-B + math.sqrt(disc)) / (2 * A)
        tstar = (d @ Lam @ (mu - o)) / (d @ Lam @ d)  # Eq. 2 before the max(0, .)
        t0 = max(r0, cam.get("near", 0.0))
        if not r1 > t0:
            continue
        key = max(0.0, tstar)
        if tile:
            key = max(0.0, (dcen @ Lam @ (mu - o)) / (dcen @ Lam @ dcen))
            hits.append((key, i, t0, r1, tstar, r0))
        else:
            hits.append((key, t0, i, r1, tstar, r0))
    hits.sort()
    if tile:  # back to the (key, t0, i, ...) layout
        hits = [(k, t0, i, r1, ts, r0) for k, i, t0, r1, ts, r0 in hits]
    return o, d, hits


def _np_encode(cfg, xl, d):
    parts = []
    if cfg.xyz_freqs == 0:
        parts += list(xl)
    else:
        for c in range(3):
            for l in range(cfg.xyz_freqs):
                parts += [math.sin((2 ** l) * math.pi * xl[c]), math.cos((2 ** l) * math.pi * xl[c])]
    if cfg.dir_freqs > 0:
        for c in range(3):
            for l in range(cfg.dir_freqs):
                parts += [math.sin((2 ** l) * math.pi * d[c]), math.cos((2 ** l) * math.pi * d[c])]
    return np.array(parts)


def _np_mlp(cfg, w, e):
    h = e
    lay = _layout(cfg)
    for li, (ws, bs, fi, fo) in enumerate(lay):
        h = w[ws].reshape(fo, fi) @ h + w[bs]
        if li < len(lay) - 1:
            h = np.maximum(h, 0.0)
    return h


def _np_encode_contact(cfg, d, delta):
    """gamma([d; delta]) of Eq. 4-5: the direction block first, then the residual."""
    parts = []
    if cfg.dir_freqs > 0:
        for c in range(3):
            for l in range(cfg.dir_freqs):
                parts += [math.sin((2 ** l) * math.pi * d[c]), math.cos((2 ** l) * math.pi * d[c])]
    if cfg.xyz_freqs == 0:
        parts += list(delta)
    else:
        for c in range(3):
            for l in range(cfg.xyz_freqs):
                parts += [math.sin((2 ** l) * math.pi * delta[c]), math.cos((2 ** l) * math.pi * delta[c])]
    return np.array(parts)


def _probe_slot_frame():
    """The four slot directions a_k, recovered from the oracle's slot weights alone:
    log(g_k / g_0) at u = e_c gives (a_k - a_0)_c, and a regular tetrahedron of unit vectors is
    centred at the origin, which fixes a_0."""
    D = np.zeros((4, 3))
    for c in range(3):
        u = np.zeros(3)
        u[c] = 1.0
        g = oracle.slot_weights(u)
        D[:, c] = np.log(g / g[0])
    a0 = -D.sum(axis=0) / 4.0
    return a0[None, :] + D


def _np_slot_feature(cfg, scene, i, o, d, tstar):
    """f = sum_k softmax_k(a_k . u) e_k with u = clip(R^T (mu - p*) / s), p* = o + max(0, t*) d."""
    mu = scene["centers"][i].astype(np.float64)
    s = scene["scales"][i].astype(np.float64)
    R = _rot(scene["quats"][i])
    u = np.clip(R.T @ (mu - (o + max(0.0, tstar) * d)) / s, -1.0, 1.0)
    z = _probe_slot_frame() @ u
    g = np.exp(z - z.max())
    g /= g.sum()
    C = cfg.slot_dim
    e = scene["weights"][i].astype(np.float64)[cfg.n_mlp_params:].reshape(4, C)
    return g @ e


def _np_render_pixel(cfg, scene, cam, x, y):
    return _np_render_pixel_hits(cfg, scene, cam, x, y, getattr(cfg, "tile_sort", 0))


def _np_render_pixel_hits(cfg, scene, cam, x, y, tile):
    """Independent restatement: quadratic roots, library rotations, matmul MLP, and the
    product form T_j = prod_{l<j} (1 - alpha_l) of the discrete operator (App. D.1). In
    contact-point mode the input is gamma([d; mu - p*]) with p* = o + max(0, t*) d and t* in
    Eq. 2's world-frame form d^T Lambda (mu - o) / d^T Lambda d."""
    o, d, hits = _np_hits(scene, cam, x, y, tile)
    C = np.zeros(3)
    F = np.zeros(cfg.feat_dim)
    Fs = np.zeros(cfg.slot_dim)
    T = 1.0
    S = cfg.samples
    for key, t0, i, t1, tstar, _ in hits:
        T_hit = T
        mu = scene["centers"][i].astype(np.float64)
        s = scene["scales"][i].astype(np.float64)
        R = _rot(scene["quats"][i])
        w = scene["weights"][i].astype(np.float64)
        dt = (t1 - t0) / S
        for k in range(S):
            t = t0 + (k + 0.5) * dt
            xl = (R.T @ (o + t * d - mu)) / s
            if getattr(cfg, "contact", 0):
                z = _np_mlp(cfg, w, _np_encode_contact(cfg, d, mu - (o + max(0.0, tstar) * d)))
            else:
                z = _np_mlp(cfg, w, _np_encode(cfg, xl, d))
            c = 1.0 / (1.0 + np.exp(-z[:3]))
            sigma = np.logaddexp(0.0, z[3])
            alpha = 1.0 - math.exp(-sigma * dt)
            C += T * alpha * c
            F += T * alpha * z[4:]
            T *= 1.0 - alpha
        if cfg.slot_dim:
            Fs += (T_hit - T) * _np_slot_feature(cfg, scene, i, o, d, tstar)
    return C, T, np.concatenate([F, Fs])


# ------------------------------------------------------------------------------------------
# Printed numbers of the paper


def test_paper_printed_shapes():
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    # 6-D input [d; delta] with L = 6 -> 72 (Sec. 4.1): the oracle's input dimension for two
    # encoded 3-vectors at L = 6 must equal the printed number (no identity term, Eq. 5).
    cfg6 = synth.SceneConfig("x", 1, 1, 1, 1, 6, 6, 32, 2, 0, 1)
    assert oracle.input_dim(cfg6) == facts["encoding_dim_6d_L6"]["value"]
    shape = facts["mlp_shape"]["value"]
    assert oracle.input_dim(cfg6) == shape[0]
    n_mlp = oracle.param_count(cfg6)
    assert n_mlp == 72 * 32 + 32 + 32 * 32 + 32 + 32 * 4 + 4
    # Model memory vs primitive count (App. A.3): MLP + 4 x 512 slots + pose, fp32.
    pm = facts["primitive_ablation_memory_mb"]
    for n, mb in zip(pm["primitives"], pm["memory_mb"]):
        est = n * (n_mlp + 4 * facts["feature_dim"]["value"] + 10) * 4 / 1e6
        assert abs(est - mb) / mb < 0.10, (n, est, mb)


# ------------------------------------------------------------------------------------------
# Camera model


def test_pixel_ray_projects_to_pixel_centre():
    cam = _cam(37, 23, seed=3)
    P = np.asarray(cam["w2c"], dtype=np.float64).reshape(3, 4)
    for (x, y) in [(0, 0), (36, 22), (18, 11), (5, 17)]:
        o, d = oracle.pixel_ray(cam, x, y)
        assert abs(np.linalg.norm(d) - 1) < 1e-14
        # The 3x3 block is treated as a rotation (origin -R^T t, direction R^T K^-1 (u, v, 1));
        # its FP32 rounding leaves it orthonormal to ~1e-7, hence the tolerances below.
        assert np.allclose(P[:, :3] @ o + P[:, 3], 0, atol=1e-6)
        X = P[:, :3] @ (o + 2.5 * d) + P[:, 3]
        u = cam["fx"] * X[0] / X[2] + cam["cx"]
        v = cam["fy"] * X[1] / X[2] + cam["cy"]
        assert abs(u - (x + 0.5)) < 1e-4 and abs(v - (y + 0.5)) < 1e-4 and X[2] > 0


# ------------------------------------------------------------------------------------------
# Closed forms


@pytest.mark.parametrize("S", [1, 3, 16])
def test_constant_sphere_closed_form(S):
    """Zero weights: c = sigmoid(b_rgb), sigma = softplus(b_sigma) everywhere. For a sphere of
    radius r the chord at ray distance b is 2 sqrt(r^2 - b^2); then C = c (1 - e^{-sigma
    chord}) and T = e^{-sigma chord} for every S (the midpoint sum is exact for constants)."""
    cfg = synth.SceneConfig("c", 40, 30, 1, 1, 6, 4, 16, 2, 0, S)
    cam = synth.make_camera(40, 30, 5, radius=2.2)
    r = 0.6
    mu = np.array([0.05, -0.1, 0.07])
    scene = {"centers": mu[None], "scales": np.full((1, 3), r), "quats": np.array([[0.3, -0.2, 0.9, 0.1]]),
             "weights": _constant_weights(cfg, 1, [[0.4, -1.2, 2.0]], [0.7])}
    rgb, T, _ = oracle.render(cfg, scene, [cam])
    c = 1.0 / (1.0 + np.exp(-np.array([0.4, -1.2, 2.0])))
    sig = math.log1p(math.exp(0.7))
    pix = oracle.all_pixels([cam])
    n_hit = 0
    for n, (v, x, y) in enumerate(pix):
        o, d = _ray_np(cam, x, y)
        b = np.linalg.norm(np.cross(mu - o, d))
        chord = 2 * math.sqrt(r * r - b * b) if b < r else 0.0
        n_hit += chord > 0
        assert abs(T[n] - math.exp(-sig * chord)) < 1e-12
        assert np.allclose(rgb[n], c * (1 - math.exp(-sig * chord)), atol=1e-12)
    assert n_hit > 50


def test_constant_ellipsoid_chord_from_quadratic_roots():
    """Anisotropic constant primitive: T = exp(-sigma (r1 - r0)) with r0, r1 the roots of the
    ellipsoid quadratic built from a library rotation matrix."""
    cfg = synth.SceneConfig("c", 32, 24, 1, 1, 0, 0, 8, 1, 0, 5)
    cam = synth.make_camera(32, 24, 11, radius=2.0)
    scene = {"centers": np.array([[0.1, 0.2, -0.1]]), "scales": np.array([[0.9, 0.25, 0.5]]),
             "quats": np.array([[0.7, 0.1, -0.5, 0.3]]),
             "weights": _constant_weights(cfg, 1, [[0, 0, 0]], [1.3])}
    _, T, _ = oracle.render(cfg, scene, [cam])
    sig = math.log1p(math.exp(1.3))
    n_hit = 0
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam])):
        _, _, hits = _np_hits(scene, cam, x, y)
        chord = sum(h[3] - h[1] for h in hits)
        n_hit += bool(hits)
        assert abs(T[n] - math.exp(-sig * chord)) < 1e-10
    assert n_hit > 40


def test_two_disjoint_primitives_order_and_storage_independence():
    """Two constant primitives one behind the other: C = c1 a1 + (1 - a1) c2 a2 with 1 the
    nearer (Eq. 6 in the order of Eq. 2's t*), whatever the storage order."""
    cfg = synth.SceneConfig("c", 20, 16, 2, 1, 0, 0, 8, 1, 0, 4)
    cam = synth.make_camera(20, 16, 2, radius=3.0)
    o, _ = _ray_np(cam, 10, 8)
    u = -o / np.linalg.norm(o)  # viewing direction to the origin
    near_c = o + 2.2 * u
    far_c = o + 3.8 * u
    base = {"centers": np.stack([far_c, near_c]), "scales": np.array([[0.5] * 3, [0.3] * 3]),
            "quats": np.array([[1.0, 0, 0, 0], [0.2, 0.4, 0.1, 0.8]]),
            "weights": _constant_weights(cfg, 2, [[3.0, -3.0, 0.0], [-2.0, 1.0, 0.5]], [0.4, 1.1])}
    rgb, T, _ = oracle.render(cfg, base, [cam])
    perm = {k: v[::-1].copy() for k, v in base.items()}
    rgb2, T2, _ = oracle.render(cfg, perm, [cam])
    assert np.array_equal(rgb, rgb2) and np.array_equal(T, T2)
    sig = [math.log1p(math.exp(0.4)), math.log1p(math.exp(1.1))]
    cols = [1 / (1 + np.exp(-np.array([3.0, -3.0, 0.0]))), 1 / (1 + np.exp(-np.array([-2.0, 1.0, 0.5])))]
    checked = 0
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam])):
        oo, d = _ray_np(cam, x, y)
        ch = []
        for i, (mu, r) in enumerate([(far_c, 0.5), (near_c, 0.3)]):
            b = np.linalg.norm(np.cross(mu - oo, d))
            ch.append(2 * math.sqrt(r * r - b * b) if b < r else 0.0)
        a_far = 1 - math.exp(-sig[0] * ch[0])
        a_near = 1 - math.exp(-sig[1] * ch[1])
        expect = cols[1] * a_near + (1 - a_near) * cols[0] * a_far
        assert np.allclose(rgb[n], expect, atol=1e-12)
        checked += ch[0] > 0 and ch[1] > 0
    assert checked >= 4


def test_contact_point_is_chord_midpoint_and_hits_match_roots():
    """Eq. 2's t* = d^T Lambda (mu - o) / d^T Lambda d is the midpoint of the quadratic's roots,
    and the oracle's hit list (order, keys, endpoints) matches the root form."""
    cfg = synth.CONFIGS["pr1"].replace(K=24)
    scene = synth.make_scene(cfg, 7)
    scene = dict(scene, scales=scene["scales"] * 2.5)
    cam = synth.make_camera(48, 40, 1, radius=3.0)
    total = 0
    for x in range(0, 48, 3):
        for y in range(0, 40, 3):
            _, _, hits = _np_hits(scene, cam, x, y)
            oh = oracle.ray_hits(scene, cam, x, y)
            assert list(oh["prim"]) == [h[2] for h in hits]
            for k, h in enumerate(hits):
                assert abs(h[4] - 0.5 * (h[5] + h[3])) < 1e-9 * max(1, abs(h[4]))
                assert abs(oh["key"][k] - h[0]) < 1e-9
                assert abs(oh["t0"][k] - h[1]) < 1e-9 and abs(oh["t1"][k] - h[3]) < 1e-9
            total += len(hits)
    assert total > 30


# ------------------------------------------------------------------------------------------
# Independent restatement on random small scenes


@pytest.mark.parametrize("name,xyzL,dirL,width,layers,feat,S", [
    ("raw", 0, 0, 32, 2, 0, 16),   # PR1 shape
    ("enc", 6, 4, 16, 3, 0, 5),
    ("feat", 6, 4, 12, 2, 5, 3),
])
def test_oracle_matches_independent_restatement(name, xyzL, dirL, width, layers, feat, S):
    cfg = synth.SceneConfig(name, 20, 14, 10, 1, xyzL, dirL, width, layers, feat, S)
    scene = synth.make_scene(cfg, 3)
    scene = dict(scene, scales=scene["scales"] * 2.0)
    cam = synth.make_camera(20, 14, 4, radius=3.0)
    rgb, T, F = oracle.render(cfg, scene, [cam])
    hit = 0
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam])):
        C2, T2, F2 = _np_render_pixel(cfg, scene, cam, x, y)
        assert np.allclose(rgb[n], C2, atol=1e-10), (x, y)
        assert abs(T[n] - T2) < 1e-10
        if feat:
            assert np.allclose(F[n], F2, atol=1e-10)
        hit += T2 < 1
    assert hit > 20


@pytest.mark.parametrize("xyzL,dirL,width,layers,feat", [
    (6, 6, 32, 2, 0),   # the paper's 72-32-32-4 model
    (0, 0, 16, 1, 0),   # raw residual, no direction
    (3, 2, 12, 2, 4),   # with a feature head
])
def test_contact_mode_matches_independent_restatement(xyzL, dirL, width, layers, feat):
    """Contact-point mode (Sec. 3.2, Eq. 2-5) against the numpy restatement, on random scenes
    with one camera outside every primitive and one inside a large primitive (t* < 0, so
    p* = o and delta = mu - o)."""
    cfg = synth.SceneConfig("k", 20, 14, 10, 1, xyzL, dirL, width, layers, feat, 1, contact=1)
    scene = synth.make_scene(cfg, 5)
    scene = dict(scene, scales=scene["scales"] * 2.0)
    cam_out = synth.make_camera(20, 14, 4, radius=3.0)
    rgb, T, F = oracle.render(cfg, scene, [cam_out])
    hit = 0
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam_out])):
        C2, T2, F2 = _np_render_pixel(cfg, scene, cam_out, x, y)
        assert np.allclose(rgb[n], C2, atol=1e-10), (x, y)
        assert abs(T[n] - T2) < 1e-10
        if feat:
            assert np.allclose(F[n], F2, atol=1e-10)
        hit += T2 < 1
    assert hit > 20
    # camera inside primitive 0: it is hit from the near plane on, with t* < 0 on most rays
    cam_in = synth.make_camera(20, 14, 6, radius=2.0)
    o_in, _ = _ray_np(cam_in, 10, 7)
    big = {k: v.copy() for k, v in scene.items()}
    big["centers"][0] = o_in + np.array([0.05, -0.04, 0.03])
    big["scales"][0] = [0.8, 0.6, 0.7]
    rgb, T, _ = oracle.render(cfg, big, [cam_in])
    neg = 0
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam_in])):
        C2, T2, _ = _np_render_pixel(cfg, big, cam_in, x, y)
        assert np.allclose(rgb[n], C2, atol=1e-10), (x, y)
        assert abs(T[n] - T2) < 1e-10
        neg += any(h[4] < 0 for h in _np_hits(big, cam_in, x, y)[2])
    assert neg > 20


def test_contact_mode_reduces_to_midpoint_mode_when_the_mlp_ignores_its_input():
    """With S = 1 and a zero first-layer weight matrix the MLP output no longer depends on its
    input, so the contact-point mode and the midpoint mode (whose one sample is also at t*) must
    give the same image bit for bit, and the same gradients for every parameter but W_0."""
    cfg = synth.SceneConfig("k", 20, 14, 10, 1, 6, 6, 16, 2, 0, 1, contact=1)
    scene = synth.make_scene(cfg, 9)
    scene = dict(scene, scales=scene["scales"] * 2.0)
    ws, bs, _, _ = _layout(cfg)[0]
    scene["weights"] = scene["weights"].copy()
    scene["weights"][:, ws] = 0.0
    scene["weights"][:, bs] = np.linspace(-0.5, 0.5, bs.stop - bs.start)
    cam = synth.make_camera(20, 14, 4, radius=3.0)
    rgb1, T1, _ = oracle.render(cfg, scene, [cam])
    rgb0, T0, _ = oracle.render(cfg.replace(contact=0), scene, [cam])
    assert np.array_equal(rgb1, rgb0) and np.array_equal(T1, T0) and T1.min() < 0.9
    pix = oracle.all_pixels([cam])
    g = synth.make_grad((pix.shape[0], 3), seed=3).astype(np.float64)
    r1 = oracle.render_backward(cfg, scene, [cam], pix, g)
    r0 = oracle.render_backward(cfg.replace(contact=0), scene, [cam], pix, g)
    for k in ("d_centers", "d_scales", "d_quats"):
        assert np.allclose(r1[k], r0[k], rtol=1e-12, atol=1e-14), k
    assert np.allclose(r1["d_weights"][:, bs.start:], r0["d_weights"][:, bs.start:], rtol=1e-12, atol=1e-14)
    assert not np.allclose(r1["d_weights"][:, ws], r0["d_weights"][:, ws])  # the inputs differ


def test_contact_mode_single_sample_and_input_dim():
    """Contact-point mode needs S = 1 and keeps the 72-wide input of Sec. 4.1 at L = 6."""
    cfg = synth.CONFIGS["contact"]
    assert cfg.samples == 1 and cfg.input_dim == 72
    scene = synth.make_scene(cfg.replace(K=2), 0)
    cam = synth.make_camera(4, 4, 0)
    with pytest.raises(RuntimeError):
        oracle.render(cfg.replace(samples=2, K=2), scene, [cam])
    enc = oracle.encode(cfg, [0.1, -0.2, 0.3], [0.6, 0.0, 0.8])
    assert enc.shape == (72,)
    assert np.allclose(enc, _np_encode_contact(cfg, [0.6, 0.0, 0.8], [0.1, -0.2, 0.3]), atol=1e-15)


def test_slot_frame_is_a_regular_tetrahedron():
    """Sec. 3.4: four unit directions forming a regular tetrahedron (the minimal affinely
    independent basis); g = softmax(a_k . u) is uniform at u = 0 and sums to one."""
    A = _probe_slot_frame()
    assert np.allclose(np.linalg.norm(A, axis=1), 1.0, atol=1e-12)
    for k in range(4):
        for m in range(k + 1, 4):
            assert abs(A[k] @ A[m] + 1.0 / 3.0) < 1e-12
    assert np.allclose(oracle.slot_weights(np.zeros(3)), 0.25, atol=1e-15)
    rng = np.random.RandomState(0)
    for _ in range(20):
        u = rng.uniform(-1, 1, 3)
        g = oracle.slot_weights(u)
        assert abs(g.sum() - 1) < 1e-14 and np.argmax(g) == np.argmax(A @ u)


def test_slots_with_equal_embeddings_are_one_minus_transmittance():
    """All four slots of a primitive equal e: f = e whatever u, so for a single primitive
    F_slot = sum_i w_i e = (1 - T_final) e at every pixel (weights and T of Eq. 6)."""
    cfg = synth.SceneConfig("s", 24, 18, 1, 1, 6, 4, 16, 2, 0, 7, slot_dim=5)
    cam = synth.make_camera(24, 18, 3, radius=2.0)
    scene = synth.make_scene(cfg, 2)
    scene = dict(scene, centers=np.zeros((1, 3), np.float32), scales=np.full((1, 3), 0.7, np.float32))
    e = np.array([0.3, -1.2, 0.5, 2.0, -0.25])
    w = scene["weights"].astype(np.float64).copy()
    w[0, cfg.n_mlp_params:] = np.tile(e, 4)
    scene["weights"] = w
    rgb, T, Fo = oracle.render(cfg, scene, [cam])
    assert Fo.shape == (24 * 18, 5) and T.min() < 0.5
    assert np.allclose(Fo, (1.0 - T)[:, None] * e[None, :], atol=1e-13)
    rgb0, T0, _ = oracle.render(cfg.replace(slot_dim=0), dict(scene, weights=w[:, :cfg.n_mlp_params]), [cam])
    assert np.array_equal(rgb, rgb0) and np.array_equal(T, T0)  # slots change no colour


@pytest.mark.parametrize("contact,S,feat", [(0, 4, 0), (1, 1, 3)])
def test_slots_match_independent_restatement(contact, S, feat):
    cfg = synth.SceneConfig("s", 20, 14, 10, 1, 4, 2, 16, 2, feat, S, contact=contact, slot_dim=6)
    scene = synth.make_scene(cfg, 4)
    scene = dict(scene, scales=scene["scales"] * 2.0)
    cam = synth.make_camera(20, 14, 4, radius=3.0)
    rgb, T, Fo = oracle.render(cfg, scene, [cam])
    hit = 0
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam])):
        C2, T2, F2 = _np_render_pixel(cfg, scene, cam, x, y)
        assert np.allclose(rgb[n], C2, atol=1e-10) and abs(T[n] - T2) < 1e-10
        assert np.allclose(Fo[n], F2, atol=1e-10), (x, y)
        hit += T2 < 1
    assert hit > 20


def test_stability_bound_of_the_rendering_operator():
    """The stability lemma of the appendix: for densities in [0, sigma_max] and colours bounded by
    C_c, |R[sigma, c] - R[sigma~, c~]|_2 <= C_c (1 + sigma_max L) int |sigma - sigma~| dt
    + sigma_max L |c - c~|_inf along every ray. With constant primitives (bias-only MLPs) both
    renders are exact, the ray's compositing sequence is its hit intervals laid end to end, and
    the bound holds with L the summed chord length; checked per ray on random perturbations."""
    cfg = synth.SceneConfig("s", 28, 20, 10, 1, 0, 0, 8, 1, 0, 3)
    rng = np.random.RandomState(7)
    base = synth.make_scene(cfg, 5)
    base = dict(base, scales=(base["scales"] * 3.0).astype(np.float32))
    cam = synth.make_camera(28, 20, 3, radius=2.8)
    worst = 0.0
    for trial in range(4):
        rgb_b = rng.normal(0, 1.5, (cfg.K, 3))
        sig_b = rng.normal(0.5, 1.0, cfg.K)
        rgb_b2 = rgb_b + rng.normal(0, 0.3, rgb_b.shape) * (trial % 2)
        sig_b2 = sig_b + rng.normal(0, 0.5, sig_b.shape) * (trial >= 1)
        s1 = dict(base, weights=_constant_weights(cfg, cfg.K, rgb_b, sig_b))
        s2 = dict(base, weights=_constant_weights(cfg, cfg.K, rgb_b2, sig_b2))
        r1, _, _ = oracle.render(cfg, s1, [cam])
        r2, _, _ = oracle.render(cfg, s2, [cam])
        sig1, sig2 = np.logaddexp(0.0, sig_b), np.logaddexp(0.0, sig_b2)
        c1, c2 = 1 / (1 + np.exp(-rgb_b)), 1 / (1 + np.exp(-rgb_b2))
        smax = max(sig1.max(), sig2.max())
        Cc = max(np.linalg.norm(c1, axis=1).max(), np.linalg.norm(c2, axis=1).max())
        for n, (v, x, y) in enumerate(oracle.all_pixels([cam])):
            _, _, hits = _np_hits(base, cam, x, y)
            if not hits:
                assert np.array_equal(r1[n], r2[n])
                continue
            ch = np.array([h[3] - h[1] for h in hits])
            ps = [h[2] for h in hits]
            L = ch.sum()
            dsig = float(np.sum(np.abs(sig1[ps] - sig2[ps]) * ch))
            dc = float(np.max(np.linalg.norm(c1[ps] - c2[ps], axis=1)))
            lhs = float(np.linalg.norm(r1[n] - r2[n]))
            rhs = Cc * (1 + smax * L) * dsig + smax * L * dc
            assert lhs <= rhs + 1e-12, (trial, x, y, lhs, rhs)
            if rhs > 0:
                worst = max(worst, lhs / rhs)
    assert 0 < worst <= 1.0


@pytest.mark.parametrize("T", [8, 16])
def test_tile_centre_order_matches_restatement(T):
    """Sec. 3.3 / App. A.4: with T x T tiles every pixel composites its own hits in the order of
    max(0, t*) along the virtual ray through its tile's centre. The oracle against the numpy
    restatement (quadratic roots, Lambda-form t* of the centre ray); on this dense scene the order
    differs from the exact one on some pixels, so the mode is not a no-op."""
    cfg = synth.SceneConfig("t", 40, 30, 24, 1, 4, 2, 16, 2, 0, 3, tile_sort=T)
    scene = synth.make_scene(cfg, 11)
    scene = dict(scene, scales=scene["scales"] * 3.0)
    cam = synth.make_camera(40, 30, 2, radius=2.6)
    rgb, Tr, _ = oracle.render(cfg, scene, [cam])
    rgb_x, Tr_x, _ = oracle.render(cfg.replace(tile_sort=0), scene, [cam])
    assert np.allclose(Tr, Tr_x, atol=1e-12)  # the order changes no transmittance
    differ = 0
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam])):
        C2, T2, _ = _np_render_pixel(cfg, scene, cam, x, y)
        assert np.allclose(rgb[n], C2, atol=1e-10), (x, y)
        oh = oracle.ray_hits(scene, cam, x, y, tile=T)
        assert list(oh["prim"]) == [h[2] for h in _np_hits(scene, cam, x, y, T)[2]]
        differ += not np.allclose(rgb[n], rgb_x[n], atol=1e-9)
    assert differ > 5


def test_tile_centre_key_is_clamped_at_zero():
    """Camera inside two large primitives whose centres lie behind it: along the tile-centre ray
    both have t* < 0, so both keys are max(0, t*) = 0 and the tie goes to the lower primitive
    index, whatever their unclamped t* (restatement with the clamp)."""
    cfg = synth.SceneConfig("t", 16, 16, 2, 1, 4, 2, 16, 2, 0, 2, tile_sort=8)
    cam = synth.make_camera(16, 16, 5, radius=2.5)
    o, d = _ray_np(cam, 8, 8)
    scene = synth.make_scene(cfg, 13)
    scene["centers"] = np.stack([o - 0.05 * d, o - 0.35 * d]).astype(np.float32)  # unclamped: 1 first
    scene["scales"] = np.array([[1.2, 1.0, 1.1], [0.9, 1.3, 1.0]], np.float32)
    rgb, _, _ = oracle.render(cfg, scene, [cam])
    for n, (v, x, y) in enumerate(oracle.all_pixels([cam])):
        oh = oracle.ray_hits(scene, cam, x, y, tile=8)
        assert list(oh["prim"]) == [0, 1] and np.all(oh["key"] == 0.0), (x, y, oh)
        C2, _, _ = _np_render_pixel(cfg, scene, cam, x, y)
        assert np.allclose(rgb[n], C2, atol=1e-10)


def test_tile_of_one_pixel_is_the_exact_order():
    """T = 1: the tile centre is the pixel centre, so the order is the exact one of Eq. 2."""
    cfg = synth.SceneConfig("t", 24, 18, 16, 1, 4, 2, 16, 2, 0, 3, tile_sort=1)
    scene = synth.make_scene(cfg, 12)
    scene = dict(scene, scales=scene["scales"] * 3.0)
    cam = synth.make_camera(24, 18, 3, radius=2.6)
    rgb, Tr, _ = oracle.render(cfg, scene, [cam])
    rgb_x, Tr_x, _ = oracle.render(cfg.replace(tile_sort=0), scene, [cam])
    assert np.array_equal(rgb, rgb_x) and np.array_equal(Tr, Tr_x)


def test_encoding_order_probe():
    """An MLP that routes exactly one encoded input j to the density recovers gamma_j from T;
    gamma_j must equal sin/cos(2^l pi p) of the expected component (Eq. 5: per scalar,
    interleaved by frequency, local xyz first, then the view direction)."""
    cfg = synth.SceneConfig("p", 8, 8, 1, 1, 3, 2, 4, 1, 0, 1)
    nin = cfg.input_dim
    assert nin == 18 + 12
    cam = synth.make_camera(8, 8, 9, radius=2.0)
    mu = np.array([0.02, -0.03, 0.01])
    r = 0.5
    lay = _layout(cfg)
    (w0, b0, _, _), (w1, b1, _, _) = lay
    x, y = 3, 4
    o, d = _ray_np(cam, x, y)
    t_c = (mu - o) @ d
    p = o + t_c * d
    chord = 2 * math.sqrt(r * r - np.sum((p - mu) ** 2))
    xl = (p - mu) / r  # identity rotation: local = (world - mu)/r; S = 1 samples the midpoint
    expect = []
    for c in range(3):
        for l in range(3):
            expect += [math.sin(2 ** l * math.pi * xl[c]), math.cos(2 ** l * math.pi * xl[c])]
    for c in range(3):
        for l in range(2):
            expect += [math.sin(2 ** l * math.pi * d[c]), math.cos(2 ** l * math.pi * d[c])]
    for j in range(nin):
        w = np.zeros(cfg.n_params)
        W0 = np.zeros((4, nin)); W0[0, j] = 1.0
        w[w0] = W0.reshape(-1); w[b0] = [2.0, 0, 0, 0]
        W1 = np.zeros((4, 4)); W1[3, 0] = 1.0
        w[w1] = W1.reshape(-1)
        scene = {"centers": mu[None], "scales": np.full((1, 3), r), "quats": np.array([[1.0, 0, 0, 0]]),
                 "weights": w[None]}
        _, T, _ = oracle.render(cfg, scene, [cam], pix=np.array([[0, x, y]], dtype=np.int32))
        sigma = -math.log(T[0]) / chord
        z = math.log(math.expm1(sigma))  # inverse softplus
        assert abs((z - 2.0) - expect[j]) < 1e-9, j


# ------------------------------------------------------------------------------------------
# The discrete operator converges to the continuous one (App. D.1)


def _smooth_single(S):
    # no hidden layer: the field is a linear map of the (smooth) encoding, so the midpoint
    # rule's error constant does not jump with ReLU kinks
    cfg = synth.SceneConfig("s", 6, 6, 1, 1, 2, 0, 8, 0, 0, S)
    scene = synth.make_scene(cfg, 21)
    scene = dict(scene, centers=np.zeros((1, 3)), scales=np.array([[0.8, 0.6, 0.7]]),
                 weights=scene["weights"] * 0.7)
    return cfg, scene


@pytest.mark.parametrize("px", [(2, 3), (1, 2)])
def test_midpoint_rule_second_order_to_continuous_operator(px):
    """The discrete operator converges to the continuous one as the step goes to zero
    (App. D.1); with midpoint samples (k + 1/2) the error falls 4x per doubling of S. The
    continuous value comes from an independent ODE integration of d tau/dt = sigma,
    dC/dt = e^{-tau} sigma c along the chord."""
    cam = synth.make_camera(6, 6, 2, radius=2.5)
    pix = np.array([[0, px[0], px[1]]], dtype=np.int32)
    cfg_ref, scene = _smooth_single(1)
    o, d, hits = _np_hits(scene, cam, px[0], px[1])
    assert len(hits) == 1
    _, t0, _, t1, _, _ = hits[0]
    R = _rot(scene["quats"][0])
    s = scene["scales"][0].astype(np.float64)
    w = scene["weights"][0].astype(np.float64)

    def rhs(t, y):
        xl = (R.T @ (o + t * d)) / s
        z = _np_mlp(cfg_ref, w, _np_encode(cfg_ref, xl, d))
        c = 1 / (1 + np.exp(-z[:3]))
        return np.concatenate([[np.logaddexp(0, z[3])], math.exp(-y[0]) * np.logaddexp(0, z[3]) * c])

    sol = solve_ivp(rhs, (t0, t1), np.zeros(4), method="DOP853", rtol=1e-13, atol=1e-15)
    cont = sol.y[1:, -1]
    errs = []
    for S in [4, 8, 16, 32, 64]:
        cfg, _ = _smooth_single(S)
        rgb, _, _ = oracle.render(cfg, scene, [cam], pix=pix)
        errs.append(np.abs(rgb[0] - cont).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[-1] < 5e-5
    for rt in ratios[1:]:
        assert 3.6 < rt < 4.4, (errs, ratios)


# ------------------------------------------------------------------------------------------
# Invariants


def _rand_scene(K=12, seed=5, S=4, feat=0):
    cfg = synth.SceneConfig("r", 24, 18, K, 1, 6, 4, 16, 2, feat, S)
    scene = synth.make_scene(cfg, seed)
    scene = dict(scene, scales=scene["scales"] * 2.0)
    return cfg, scene


def test_transmittance_and_colour_ranges():
    cfg, scene = _rand_scene()
    cams = [synth.make_camera(24, 18, v) for v in range(2)]
    rgb, T, _ = oracle.render(cfg, scene, cams)
    assert np.all(T >= 0) and np.all(T <= 1) and np.all(rgb >= 0) and np.all(rgb <= 1)
    assert np.any(T < 0.9)


def test_weights_plus_final_transmittance_is_one():
    """White colour everywhere: C = sum_j w_j = 1 - T_final (telescoping of Eq. 6)."""
    cfg, scene = _rand_scene()
    w = scene["weights"].astype(np.float64).copy()
    ws, bs, fi, fo = _layout(cfg)[-1]
    for p in range(w.shape[0]):
        Wl = w[p, ws].reshape(fo, fi)
        Wl[:3] = 0
        w[p, ws] = Wl.reshape(-1)
        b = w[p, bs]
        b[:3] = 60.0
        w[p, bs] = b
    cam = synth.make_camera(24, 18, 1)
    rgb, T, _ = oracle.render(cfg, dict(scene, weights=w), [cam])
    assert np.allclose(rgb, (1 - T)[:, None], atol=1e-14)


def test_invariances_permutation_quat_sign_scale_rigid_motion():
    cfg, scene = _rand_scene(K=10, seed=8)
    cam = synth.make_camera(24, 18, 3)
    rgb, T, _ = oracle.render(cfg, scene, [cam])
    perm = np.random.RandomState(0).permutation(10)
    sp = {k: v[perm] for k, v in scene.items()}
    rgb_p, T_p, _ = oracle.render(cfg, sp, [cam])
    assert np.allclose(rgb, rgb_p, atol=1e-13) and np.allclose(T, T_p, atol=1e-13)
    sq = dict(scene, quats=-2.5 * scene["quats"].astype(np.float64))
    rgb_q, T_q, _ = oracle.render(cfg, sq, [cam])
    assert np.allclose(rgb, rgb_q, atol=1e-12) and np.allclose(T, T_q, atol=1e-12)
    # joint rigid motion (x -> Q x + c) of primitives and camera (Sec. 4.3 editing by poses)
    Q = Rotation.from_rotvec([0.3, -0.8, 0.4]).as_matrix()
    cvec = np.array([0.2, -0.1, 0.3])
    qrot = Rotation.from_matrix(Q)
    new_q = []
    for q in scene["quats"].astype(np.float64):
        r = qrot * Rotation.from_quat([q[1], q[2], q[3], q[0]])
        x, y, z, w = r.as_quat()
        new_q.append([w, x, y, z])
    sm = dict(scene, centers=(scene["centers"].astype(np.float64) @ Q.T) + cvec, quats=np.array(new_q))
    P = np.asarray(cam["w2c"], dtype=np.float64).reshape(3, 4)
    U, _, Vt = np.linalg.svd(P[:, :3])  # exact rotation, so that -R^T t moves rigidly too
    P[:, :3] = U @ Vt
    cam = dict(cam, w2c=P.reshape(12))
    Rn = P[:, :3] @ Q.T
    tn = P[:, 3] - Rn @ cvec
    cam_m = dict(cam, w2c=np.concatenate([Rn, tn[:, None]], axis=1).reshape(12))
    # the view direction input changes with the motion; switch it off for this check
    cfg_nd = cfg.replace(dir_freqs=0)
    sc_nd = synth.make_scene(cfg_nd, 8)
    sc_nd = dict(sc_nd, scales=scene["scales"], centers=scene["centers"], quats=scene["quats"])
    rgb0, T0, _ = oracle.render(cfg_nd, sc_nd, [cam])
    rgb1, T1, _ = oracle.render(cfg_nd, dict(sc_nd, centers=sm["centers"], quats=sm["quats"]), [cam_m])
    assert np.allclose(rgb0, rgb1, atol=1e-9) and np.allclose(T0, T1, atol=1e-9)
    assert np.any(T0 < 0.95)


# ------------------------------------------------------------------------------------------
# Gradients by central finite differences


def _loss(cfg, scene, cams, pix, g_rgb, g_T, g_F):
    rgb, T, F = oracle.render(cfg, scene, cams, pix=pix, n_threads=4)
    L = float(np.sum(rgb * g_rgb) + np.sum(T * g_T))
    if F is not None:
        L += float(np.sum(F * g_F))
    return L


def _check_central_differences(cfg, scene, cams, contact_kink=False):
    """Analytic reverse mode against central differences of the forward loss L = <g, outputs>
    on the pose (all of centres, scales, quaternions) and 40 random weights."""
    pix = oracle.all_pixels(cams)
    n = pix.shape[0]
    # stay away from tangency (and, in contact mode, from t* = 0, where max(0, t*) has a kink)
    # so that no step changes a hit set, an order or a branch
    for (v, x, y) in pix:
        m2, tm = oracle.ray_m2(scene, cams[v], x, y)
        assert np.all(np.abs(m2 - 1) > 1e-4)
        if contact_kink:
            assert np.all(np.abs(tm[m2 < 1]) > 1e-3)
    g_rgb = synth.make_grad((n, 3), seed=1).astype(np.float64)
    g_T = synth.make_grad((n,), seed=2).astype(np.float64)
    FT = cfg.feat_dim + cfg.slot_dim
    g_F = synth.make_grad((n, max(FT, 1)), seed=3).astype(np.float64)[:, :FT]
    res = oracle.render_backward(cfg, scene, cams, pix, g_rgb, g_T, g_F if FT else None)
    assert np.any(res["trans"] < 0.9)
    h = 1e-6
    K = scene["centers"].shape[0]
    rng = np.random.RandomState(1)
    checks = [("centers", i) for i in range(3 * K)] + [("scales", i) for i in range(3 * K)] + \
             [("quats", i) for i in range(4 * K)] + \
             [("weights", int(i)) for i in rng.choice(K * cfg.n_params, 40, replace=False)]
    if cfg.slot_dim:  # and 12 slot-embedding entries
        slots = [p * cfg.n_params + cfg.n_mlp_params + j for p in range(K) for j in range(4 * cfg.slot_dim)]
        checks += [("weights", int(i)) for i in rng.choice(slots, 12, replace=False)]
    key = {"centers": "d_centers", "scales": "d_scales", "quats": "d_quats", "weights": "d_weights"}
    for name, flat in checks:
        sp = {k: v.copy() for k, v in scene.items()}
        sm = {k: v.copy() for k, v in scene.items()}
        sp[name].reshape(-1)[flat] += h
        sm[name].reshape(-1)[flat] -= h
        fd = (_loss(cfg, sp, cams, pix, g_rgb, g_T, g_F) - _loss(cfg, sm, cams, pix, g_rgb, g_T, g_F)) / (2 * h)
        an = res[key[name]].reshape(-1)[flat]
        err = abs(fd - an) / max(1e-3, abs(fd), abs(an))
        assert err < 2e-5, (name, flat, fd, an)


def _grad_scene(cfg):
    scene = synth.make_scene(cfg, 13)
    scene = {k: v.astype(np.float64) for k, v in scene.items()}
    scene["centers"] = scene["centers"] * 0.4
    scene["scales"] = scene["scales"] * 0.0 + np.array([[0.55, 0.4, 0.5], [0.35, 0.6, 0.45], [0.5, 0.5, 0.3]])
    return scene


@pytest.mark.parametrize("feat,xyzL", [(0, 6), (3, 0)])
def test_gradients_central_differences(feat, xyzL):
    cfg = synth.SceneConfig("g", 14, 10, 3, 1, xyzL, 2, 8, 2, feat, 4)
    _check_central_differences(cfg, _grad_scene(cfg), [synth.make_camera(14, 10, 6, radius=2.2)])


@pytest.mark.parametrize("feat,xyzL,dirL", [(0, 6, 6), (2, 0, 2)])
def test_gradients_central_differences_contact_mode(feat, xyzL, dirL):
    """Contact-point mode: delta = mu - o - max(0, t*) d adds dL/dmu directly and, through t*,
    the chain of Eq. 2 into the pose."""
    cfg = synth.SceneConfig("g", 14, 10, 3, 1, xyzL, dirL, 8, 2, feat, 1, contact=1)
    _check_central_differences(cfg, _grad_scene(cfg), [synth.make_camera(14, 10, 6, radius=2.2)],
                               contact_kink=True)


def test_gradients_central_differences_contact_mode_camera_inside():
    """Contact-point mode with the camera inside a primitive: rays on which t* < 0 feed
    delta = mu - o, whose only pose gradient is the direct dL/dmu."""
    cfg = synth.SceneConfig("g", 10, 8, 2, 1, 3, 2, 8, 2, 0, 1, contact=1)
    cam = synth.make_camera(10, 8, 6, radius=2.2)
    o, d = _ray_np(cam, 5, 4)
    scene = _grad_scene(cfg.replace(K=3))
    scene = {k: v[:2].copy() for k, v in scene.items()}
    scene["centers"][0] = o + np.array([0.21, -0.13, 0.0]) - 0.17 * d  # centre behind the camera
    scene["scales"][0] = [0.9, 0.8, 1.0]
    scene["centers"][1] = o + 1.6 * d
    m2s = []
    for (v, x, y) in oracle.all_pixels([cam]):
        m2, tm = oracle.ray_m2(scene, cam, x, y)
        m2s.append(tm[0])
    assert min(m2s) < 0  # some rays meet primitive 0 with t* < 0
    _check_central_differences(cfg, scene, [cam], contact_kink=True)


@pytest.mark.parametrize("contact,S,feat", [(0, 3, 0), (1, 1, 2)])
def test_gradients_central_differences_slots(contact, S, feat):
    """Slot features (Sec. 3.4): their gradient reaches the embeddings, the compositing weights
    (and through them the MLP) and the pose through u = clip(R^T delta / s)."""
    cfg = synth.SceneConfig("g", 14, 10, 3, 1, 3, 2, 8, 2, feat, S, contact=contact, slot_dim=4)
    _check_central_differences(cfg, _grad_scene(cfg), [synth.make_camera(14, 10, 6, radius=2.2)],
                               contact_kink=True)
