"""Pins of the training-objective and optimizer oracle (oracle/train.py) (CPU only): SSIM
identities and closed forms, an explicit-loop restatement of the SSIM map, central differences
of the loss, the tile mask's reach, and Adam's bias correction."""
import numpy as np
import pytest

from oracle import train as otr


def _imgs(V=1, H=20, W=24, seed=0):
    rng = np.random.RandomState(seed)
    return rng.uniform(0, 1, (V, H, W, 3)), rng.uniform(0, 1, (V, H, W, 3))


def test_window_is_normalised_gaussian():
    g = otr.gaussian_window()
    assert g.shape == (11,) and abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert abs(g[5 + 1] / g[5] - np.exp(-1 / (2 * 1.5 ** 2))) < 1e-14


def test_ssim_of_an_image_with_itself_is_one_and_the_loss_zero():
    x, _ = _imgs()
    assert np.allclose(otr.ssim_map_loops(x, x), 1.0, atol=1e-12)
    L, parts, gx, _ = otr.loss(x, x, 0.2)
    assert abs(L) < 1e-12 and abs(parts["ssim"] - 1) < 1e-12 and np.abs(gx).max() < 1e-9


def test_ssim_torch_equals_explicit_window_sums():
    x, y = _imgs(V=2, H=13, W=15, seed=1)
    import torch
    a = otr.ssim_map_torch(torch.from_numpy(x), torch.from_numpy(y)).numpy()
    b = otr.ssim_map_loops(x, y)
    assert np.allclose(a, b, atol=1e-12)


def test_ssim_of_constant_images_in_the_interior():
    """Window fully inside the image: mu = the constants, no variance, S = (2ab + C1)/(a^2 + b^2 + C1)."""
    H, W = 16, 18
    x = np.full((1, H, W, 3), 0.3)
    y = np.full((1, H, W, 3), 0.75)
    s = otr.ssim_map_loops(x, y)
    a, b = 0.3, 0.75
    want = (2 * a * b + otr.C1) / (a * a + b * b + otr.C1)
    assert np.allclose(s[0, 5:H - 5, 5:W - 5], want, atol=1e-12)
    assert not np.allclose(s[0, 0, 0], want)  # zero padding at the border


def test_loss_gradient_central_differences():
    x, y = _imgs(V=1, H=12, W=14, seed=2)
    tm = np.array([[[1, 0], [0, 1]]], np.uint8)  # 8 x 8 tiles, two of four selected
    f = np.random.RandomState(3).uniform(-1, 1, (1, 12, 14, 5))
    ft = np.random.RandomState(4).uniform(-1, 1, (1, 12, 14, 5))
    L, parts, gx, gf = otr.loss(x, y, 0.2, 8, tm, f, ft)
    h = 1e-6
    rng = np.random.RandomState(5)
    for _ in range(25):
        i = tuple(rng.randint(s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (otr.loss(xp, y, 0.2, 8, tm, f, ft)[0] - otr.loss(xm, y, 0.2, 8, tm, f, ft)[0]) / (2 * h)
        assert abs(fd - gx[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, gx[i])
    for _ in range(10):
        i = tuple(rng.randint(s) for s in f.shape)
        fp, fm = f.copy(), f.copy()
        fp[i] += h
        fm[i] -= h
        fd = (otr.loss(x, y, 0.2, 8, tm, fp, ft)[0] - otr.loss(x, y, 0.2, 8, tm, fm, ft)[0]) / (2 * h)
        assert abs(fd - gf[i]) < 1e-6, (i, fd, gf[i])


def test_tile_mask_reach():
    """Only selected tiles enter the loss; the SSIM window carries their gradient at most 5
    pixels out, so pixels farther from every selected tile get exactly zero."""
    x, y = _imgs(V=1, H=32, W=32, seed=6)
    tm = np.zeros((1, 4, 4), np.uint8)
    tm[0, 0, 0] = 1  # the 8 x 8 tile at the origin
    _, parts, gx, _ = otr.loss(x, y, 0.2, 8, tm)
    assert parts["n"] == 64
    assert np.abs(gx[0, 13:, :]).max() == 0 and np.abs(gx[0, :, 13:]).max() == 0
    assert np.abs(gx[0, 8:13, :8]).max() > 0  # reached by the SSIM window only
    L_all, _, _, _ = otr.loss(x, y, 0.2, 8, None)
    L_ones, _, _, _ = otr.loss(x, y, 0.2, 8, np.ones((1, 4, 4), np.uint8))
    assert abs(L_all - L_ones) < 1e-15


def test_adam_constant_gradient_moves_by_lr_per_step():
    """With a constant gradient the bias corrections make m_hat = g and v_hat = g^2 at every
    step, so each step moves p by lr * g / (|g| + eps) (Kingma & Ba's update)."""
    g = np.array([0.5, -2.0, 1e-3, -7.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    m = np.zeros(4)
    v = np.zeros(4)
    q = p.copy()
    for t in range(1, 6):
        q, m, v = otr.adam(q, g, m, v, t, 1e-2)
    assert np.allclose(q, p - 5 * 1e-2 * g / (np.abs(g) + 1e-15), atol=1e-12)


def test_adam_log_parameter_group():
    """log-scales: the gradient reaching log x is dL/dx * x, and x = exp(log x) is returned."""
    x = np.array([0.1, 0.5, 2.0])
    gx = np.array([3.0, -1.0, 0.25])
    lp, m, v, xn = otr.adam(np.log(x), gx, np.zeros(3), np.zeros(3), 1, 1e-2, log_param=True, aux=x)
    assert np.allclose(xn, x * np.exp(-1e-2 * np.sign(gx)), atol=1e-12)
    assert np.allclose(m, 0.1 * gx * x)


def test_learning_rates_of_the_paper():
    assert otr.lr_of("log_scales") == 1e-2 and otr.lr_of("centers") == 1e-4
    assert otr.lr_of("weights") == 1e-3 and otr.lr_of("quats") == 1e-3
