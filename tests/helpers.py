"""Shared helpers of the test suite: run the CUDA path and the oracle on the same inputs."""
import numpy as np

from paper_2606_03877_gb300 import synth


def scaled_scene(cfg, seed=0, scale_mul=1.0):
    sc = synth.make_scene(cfg, seed)
    if scale_mul != 1.0:
        sc = dict(sc, scales=(sc["scales"] * scale_mul).astype(np.float32))
    return sc


def to_dev(scene, device="cuda"):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in scene.items()}


def gpu_render(cfg, scene, cams, precision="fp32", **kw):
    """Returns (renderer, outputs as numpy)."""
    import torch
    from paper_2606_03877_gb300.render import Renderer
    r = Renderer(cfg, precision=precision, **kw)
    d = to_dev(scene)
    packed = r.pack(d["weights"])
    out = r.forward(d["centers"], d["scales"], d["quats"], packed, cams)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    return r, res, d, packed


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / max(nb, 1e-30))


def pixel_index(cfg_w, cfg_h, pix):
    """Global ray index of (view, x, y) triples."""
    return pix[:, 0].astype(np.int64) * cfg_w * cfg_h + pix[:, 2].astype(np.int64) * cfg_w + pix[:, 1]
