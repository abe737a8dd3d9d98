"""Batches with a device-resident item table (mlps_render_batch_*_dev): the same output bits as
the host-table call, a CUDA graph captured once and replayed with new items written into the
device table (other cameras, resolutions and primitive ranges within the caps), and an invalid
item reported through the device status word."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import _lib, synth
from paper_2606_03877_gb300.render import BatchRenderer, DeviceBatchRenderer

from helpers import rel_l2, to_dev

pytestmark = pytest.mark.gpu

SHAPE = synth.CONFIGS["prec"]  # 60-64x64x64-4, S = 32
CAP_W, CAP_H, CAP_P = 80, 64, 30


def _batch(sizes, first_seed):
    cfgs = [SHAPE.replace(width=w, height=h, K=k, n_views=1) for w, h, k in sizes]
    cat, items, scenes = synth.make_batch(cfgs, first_seed)
    cat = dict(cat, scales=(cat["scales"] * 2.0).astype(np.float32))
    scenes = [dict(sc, scales=(sc["scales"] * 2.0).astype(np.float32)) for sc in scenes]
    return cfgs, cat, items, scenes


SIZES_A = [(64, 48, 12), (40, 40, 30), (80, 60, 7), (48, 64, 21), (32, 24, 16)]


def _other_items(items, seed):
    """New items over the same scene arrays: other cameras and resolutions, ranges moved (item i
    renders scene (i + 2) mod n's primitives, the last one a sub-range)."""
    n = len(items)
    res = [(72, 40), (24, 64), (80, 64), (16, 16), (56, 36)]
    out = []
    for i in range(n):
        off, cnt, _ = items[(i + 2) % n]
        if i == n - 1:
            off, cnt = off + cnt // 3, cnt - cnt // 3
        w, h = res[i]
        out.append((off, cnt, synth.make_camera(w, h, seed + i)))
    return out


def _host_eager(precision, cat, items, g_rgb=None):
    K = cat["centers"].shape[0]
    br = BatchRenderer(SHAPE, items, K, precision=precision)
    d = to_dev(cat)
    packed = br.pack(d["weights"])
    out = br.forward(d["centers"], d["scales"], d["quats"], packed)
    grads = br.backward(g_rgb[: br.n_pixels]) if g_rgb is not None else None
    torch.cuda.synchronize()
    assert br.status() == 0
    return out, grads


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_device_table_matches_host_table(precision):
    cfgs, cat, items, scenes = _batch(SIZES_A, 40)
    K = cat["centers"].shape[0]
    g = torch.from_numpy(synth.make_grad((len(items) * CAP_W * CAP_H, 3), seed=5)).cuda()
    ref, ref_g = _host_eager(precision, cat, items, g)
    db = DeviceBatchRenderer(SHAPE, len(items), CAP_W, CAP_H, CAP_P, K, precision=precision)
    db.set_items(items)
    d = to_dev(cat)
    packed = db.pack(d["weights"])
    out = db.forward(d["centers"], d["scales"], d["quats"], packed)
    grads = db.backward(g)
    torch.cuda.synchronize()
    assert db.status() == 0 and db.status("scratch") == 0
    n = sum(w * h for w, h, _ in SIZES_A)
    assert torch.equal(out["rgb"][:n], ref["rgb"]) and torch.equal(out["trans"][:n], ref["trans"])
    assert torch.count_nonzero(out["rgb"][n:]) == 0  # past the live total: not written
    for k in ref_g:
        assert rel_l2(grads[k].cpu().numpy(), ref_g[k].cpu().numpy()) < 1e-5, k


def test_device_table_graph_replays_new_items():
    """One capture, two item tables: each replay equals the host-table eager call on the items the
    device table held at replay time (forward bits equal; gradients to FP32 summation order), and
    item 0 of the second table matches the FP64 oracle."""
    cfgs, cat, items_a, scenes = _batch(SIZES_A, 50)
    items_b = _other_items(items_a, 300)
    K = cat["centers"].shape[0]
    db = DeviceBatchRenderer(SHAPE, len(items_a), CAP_W, CAP_H, CAP_P, K, precision="fp32")
    d = to_dev(cat)
    packed = db.pack(d["weights"])
    out = db.new_outputs()
    grads = db.new_grads()
    g = torch.from_numpy(synth.make_grad((db.cap_pixels, 3), seed=6)).cuda()
    db.set_items(items_a)

    def step():
        db.forward(d["centers"], d["scales"], d["quats"], packed, out=out)
        db.backward(g, out=grads)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm-up outside the capture (kernel attributes, lazy loading)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for items in (items_a, items_b):
        db.set_items(items)
        out["rgb"].zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert db.status() == 0 and db.status("scratch") == 0
        ref, ref_g = _host_eager("fp32", cat, items, g)
        n = sum(int(c["width"]) * int(c["height"]) for _, _, c in items)
        assert torch.equal(out["rgb"][:n], ref["rgb"]) and torch.equal(out["trans"][:n], ref["trans"])
        for k in ref_g:
            assert rel_l2(grads[k].cpu().numpy(), ref_g[k].cpu().numpy()) < 1e-5, k
    off, cnt, cam = items_b[0]
    sc = {k: v[off:off + cnt] for k, v in cat.items()}
    c0 = SHAPE.replace(width=int(cam["width"]), height=int(cam["height"]), K=cnt, n_views=1)
    rgb_o, T_o, _ = oracle.render(c0, sc, [cam])
    rgb = db.split(out["rgb"])[0].cpu().numpy().reshape(-1, 3)
    assert np.abs(rgb - rgb_o).max() < 1e-4


def test_device_table_invalid_item_sets_status_and_renders_empty():
    """An item over the caps becomes an empty view: the status word says
    MLPS_ERR_INVALID_ARGUMENT and the items before it render as in the host-table call."""
    cfgs, cat, items, scenes = _batch(SIZES_A, 60)
    K = cat["centers"].shape[0]
    bad = list(items)
    off, cnt, cam = bad[2]
    big = dict(cam, width=CAP_W + 16)
    bad[2] = (off, cnt, big)
    db = DeviceBatchRenderer(SHAPE, len(items), CAP_W, CAP_H, CAP_P, K, precision="fp32")
    db.set_items(bad)
    d = to_dev(cat)
    packed = db.pack(d["weights"])
    out = db.forward(d["centers"], d["scales"], d["quats"], packed)
    torch.cuda.synchronize()
    assert db.status() == _lib.MLPS_ERR_INVALID_ARGUMENT
    assert db.status() == 0  # read and cleared
    ref, _ = _host_eager("fp32", cat, items[:2])
    n2 = sum(w * h for w, h, _ in SIZES_A[:2])
    assert torch.equal(out["rgb"][:n2], ref["rgb"])
    # the items after it follow directly (the invalid item has no pixels)
    ref_all, _ = _host_eager("fp32", cat, items[:2] + items[3:])
    n_all = n2 + sum(w * h for w, h, _ in SIZES_A[3:])
    assert torch.equal(out["rgb"][:n_all], ref_all["rgb"])
