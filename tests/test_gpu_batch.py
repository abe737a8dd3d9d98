"""Batched rendering (many scenes of uneven primitive counts and resolutions in one call) on the
GPU: every item against the oracle, against the single-scene call, gradients, shared primitive
ranges and CUDA-graph capture and replay."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import synth
from paper_2606_03877_gb300.render import BatchRenderer

from helpers import gpu_render, psnr, rel_l2, to_dev

pytestmark = pytest.mark.gpu

SHAPE = synth.CONFIGS["prec"]  # MLP shape shared by the batch (60-64x64x64-4, S = 32)


def _small_batch(first_seed=20):
    sizes = [(64, 48, 12), (40, 40, 30), (80, 60, 7), (48, 64, 21), (32, 24, 16)]
    cfgs = [SHAPE.replace(width=w, height=h, K=k, n_views=1) for w, h, k in sizes]
    cat, items, scenes = synth.make_batch(cfgs, first_seed)
    cat = dict(cat, scales=(cat["scales"] * 2.0).astype(np.float32))  # more hits per ray
    scenes = [dict(sc, scales=(sc["scales"] * 2.0).astype(np.float32)) for sc in scenes]
    return cfgs, cat, items, scenes


def _batch_forward(precision, cat, items, **kw):
    K = cat["centers"].shape[0]
    br = BatchRenderer(SHAPE, items, K, precision=precision, **kw)
    d = to_dev(cat)
    packed = br.pack(d["weights"])
    out = br.forward(d["centers"], d["scales"], d["quats"], packed)
    torch.cuda.synchronize()
    assert br.status() == 0
    return br, out, d, packed


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_items_match_oracle(precision):
    cfgs, cat, items, scenes = _small_batch()
    br, out, _, _ = _batch_forward(precision, cat, items)
    for i, (c, sc, it) in enumerate(zip(cfgs, scenes, items)):
        rgb_o, T_o, _ = oracle.render(c, sc, [it[2]])
        rgb = br.split(out["rgb"])[i].cpu().numpy().reshape(-1, 3)
        T = br.split(out["trans"])[i].cpu().numpy().reshape(-1)
        if precision == "fp32":
            assert np.abs(rgb - rgb_o).max() < 1e-4, i
            assert np.abs(T - T_o).max() < 1e-4, i
        else:
            assert psnr(rgb, rgb_o) >= 45.0, i


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_forward_is_bit_identical_to_single_scene_calls(precision):
    """Each sample row's MLP result and each interval's composite depend only on that interval,
    so batching changes no output bit."""
    cfgs, cat, items, scenes = _small_batch(30)
    br, out, _, _ = _batch_forward(precision, cat, items)
    for i, (c, sc, it) in enumerate(zip(cfgs, scenes, items)):
        _, o1, _, _ = gpu_render(c, sc, [it[2]], precision)
        assert np.array_equal(br.split(out["rgb"])[i].cpu().numpy(), o1["rgb"][0]), i
        assert np.array_equal(br.split(out["trans"])[i].cpu().numpy(), o1["trans"][0]), i


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_backward_matches_single_scene_calls(precision):
    from paper_2606_03877_gb300.render import Renderer
    cfgs, cat, items, scenes = _small_batch(40)
    br, out, d, packed = _batch_forward(precision, cat, items)
    g = torch.from_numpy(synth.make_grad((br.n_pixels, 3), seed=9)).cuda()
    gb = br.backward(g)
    torch.cuda.synchronize()
    assert br.status("scratch") == 0
    gs = br.split(g)
    for i, (c, sc, it) in enumerate(zip(cfgs, scenes, items)):
        r = Renderer(c, precision=precision)
        ds = to_dev(sc)
        pk = r.pack(ds["weights"])
        r.forward(ds["centers"], ds["scales"], ds["quats"], pk, [it[2]])
        g1 = r.backward(gs[i].reshape(1, c.height, c.width, 3))
        torch.cuda.synchronize()
        o, n = it[0], it[1]
        for k in ("d_weights", "d_centers", "d_scales", "d_quats"):
            e = rel_l2(gb[k][o:o + n].cpu().numpy(), g1[k].cpu().numpy())
            assert e < (1e-5 if precision == "fp32" else 1e-4), (i, k, e)


def test_batch_fp32_gradients_match_oracle():
    """L = 1/2 sum (C - C*)^2 per item with C* the oracle render of the item's scene perturbed
    with seed 1 (the differentiation workload's loss)."""
    cfgs, cat, items, scenes = _small_batch(50)
    br, out, d, packed = _batch_forward("fp32", cat, items)
    gs = []
    for c, sc, it in zip(cfgs, scenes, items):
        cur, _, _ = oracle.render(c, sc, [it[2]])
        tgt, _, _ = oracle.render(c, synth.perturb_scene(sc, c, 1), [it[2]])
        gs.append((cur - tgt).astype(np.float32))
    g = torch.from_numpy(np.concatenate(gs, axis=0)).cuda()
    gb = br.backward(g)
    torch.cuda.synchronize()
    for i in (0, 2):
        c, sc, it = cfgs[i], scenes[i], items[i]
        ref = oracle.render_backward(c, sc, [it[2]], oracle.all_pixels([it[2]]), gs[i].reshape(-1, 3))
        o, n = it[0], it[1]
        for k in ("d_weights", "d_centers", "d_scales", "d_quats"):
            e = rel_l2(gb[k][o:o + n].cpu().numpy(), ref[k])
            assert e < 1e-3, (i, k, e)


def test_batch_items_sharing_primitives_equal_multiview_call():
    c = SHAPE.replace(width=56, height=40, K=20, n_views=3)
    sc = synth.make_scene(c, 7)
    sc = dict(sc, scales=(sc["scales"] * 2.0).astype(np.float32))
    cams = synth.make_cameras(c, first_view_seed=7)
    _, o1, _, _ = gpu_render(c, sc, cams, "bf16")
    br, out, _, _ = _batch_forward("bf16", sc, [(0, c.K, cam) for cam in cams])
    assert np.array_equal(out["rgb"].cpu().numpy().reshape(o1["rgb"].shape), o1["rgb"])


def test_batch_cuda_graph_capture_and_replay():
    """Forward + backward of a batch captured once in a CUDA graph; replays match eager calls,
    also after the scene parameters are changed in place."""
    cfgs, cat, items, scenes = _small_batch(60)
    K = cat["centers"].shape[0]
    br = BatchRenderer(SHAPE, items, K, precision="bf16")
    d = to_dev(cat)
    w = d["weights"]
    packed = torch.empty(K * br.stride, dtype=torch.uint8, device="cuda")
    out = br.new_outputs()
    grads = br.new_grads()
    g = torch.from_numpy(synth.make_grad((br.n_pixels, 3), seed=2)).cuda()

    def step():
        br.pack(w, out=packed)
        br.forward(d["centers"], d["scales"], d["quats"], packed, out=out)
        br.backward(g, out=grads)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm-up outside capture (kernel attributes, driver entry points)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for trial in range(2):
        if trial == 1:
            with torch.no_grad():
                d["centers"].mul_(1.01)  # new inputs, same buffers
        graph.replay()
        torch.cuda.synchronize()
        assert br.status() == 0 and br.status("scratch") == 0
        rgb_g = out["rgb"].clone()
        gw = grads["d_weights"].clone()
        step()  # eager
        torch.cuda.synchronize()
        assert torch.equal(rgb_g, out["rgb"])
        assert rel_l2(gw.cpu().numpy(), grads["d_weights"].cpu().numpy()) < 1e-5


def test_autotuner_picks_a_candidate_and_changes_no_output_bit():
    """The tuner times tile 16/8 x samples-per-CTA 6/5/4/3/2 on this batch, returns the fastest, caches
    it, and the tuned configuration renders the same image bit for bit (tile edge and groups
    change scheduling only)."""
    from paper_2606_03877_gb300 import _lib
    _lib.mlps_autotune_clear()
    cfgs, cat, items, scenes = _small_batch(70)
    br, out0, d, packed = _batch_forward("bf16", cat, items)
    ref = out0["rgb"].clone()
    g = torch.from_numpy(synth.make_grad((br.n_pixels, 3), seed=4)).cuda()
    tun = br.autotune(d["centers"], d["scales"], d["quats"], packed, d_rgb=g, reps=2)
    print("autotune", tun)
    assert len(tun["candidates"]) == 8 and all(ms > 0 for _, _, ms in tun["candidates"])  # 2 tiles x 2..5 groups
    assert (tun["tile"], tun["mlp_groups"]) in [(t, gg) for t, gg, _ in tun["candidates"]]
    assert tun["best_ms"] == min(ms for _, _, ms in tun["candidates"])
    out = br.forward(d["centers"], d["scales"], d["quats"], packed)
    torch.cuda.synchronize()
    assert br.status() == 0
    assert torch.equal(out["rgb"], ref)
    again = br.autotune(d["centers"], d["scales"], d["quats"], packed, d_rgb=g, reps=2)
    assert again["best_ms"] == 0.0 and (again["tile"], again["mlp_groups"]) == (tun["tile"], tun["mlp_groups"])


def test_batch_edge_cases_empty_items_and_tiny_images():
    """Items with no primitives render black with T = 1; a 1 x 1 item and a batch whose scene
    arrays are empty (K = 0) run; gradients of unreferenced primitives are zero."""
    cfgs, cat, items, scenes = _small_batch(80)
    K = cat["centers"].shape[0]
    tiny = dict(items[0][2], width=1, height=1, cx=0.5, cy=0.5)
    its = [items[0], (0, 0, items[1][2]), (items[2][0], items[2][1], tiny), (items[3][0], 0, items[3][2])]
    br, out, d, packed = _batch_forward("bf16", cat, its)
    rgb, T = br.split(out["rgb"]), br.split(out["trans"])
    for i in (1, 3):
        assert float(rgb[i].abs().max()) == 0.0 and bool((T[i] == 1.0).all()), i
    c0 = cfgs[0]
    _, o1, _, _ = gpu_render(c0, scenes[0], [items[0][2]], "bf16")
    assert np.array_equal(rgb[0].cpu().numpy(), o1["rgb"][0])
    g = br.backward(torch.ones(br.n_pixels, 3, device="cuda"))
    torch.cuda.synchronize()
    assert br.status("scratch") == 0
    used = np.zeros(K, bool)
    for off, cnt, _ in its:
        used[off:off + cnt] = True
    assert float(np.abs(g["d_weights"].cpu().numpy()[~used]).max()) == 0.0
    # no primitives at all
    empty = {k: v[:0] for k, v in cat.items()}
    br0 = BatchRenderer(SHAPE, [(0, 0, items[0][2]), (0, 0, tiny)], 0, precision="bf16")
    d0 = to_dev(empty)
    out0 = br0.forward(d0["centers"], d0["scales"], d0["quats"], br0.pack(d0["weights"]))
    torch.cuda.synchronize()
    assert br0.status() == 0 and float(out0["rgb"].abs().max()) == 0.0


def test_batch_with_contact_slots_and_tile_order():
    """The batched call with the paper's contact-point model, feature slots and the tile-centre
    order: every item against the oracle (colour, T and the slot map)."""
    base = synth.CONFIGS["contact"].replace(slot_dim=16, tile_sort=8)
    sizes = [(48, 40, 10), (40, 32, 14), (56, 24, 6)]
    cfgs = [base.replace(width=w, height=h, K=k, n_views=1) for w, h, k in sizes]
    cat, items, scenes = synth.make_batch(cfgs, 90)
    cat = dict(cat, scales=(cat["scales"] * 2.0).astype(np.float32))
    scenes = [dict(sc, scales=(sc["scales"] * 2.0).astype(np.float32)) for sc in scenes]
    K = cat["centers"].shape[0]
    br = BatchRenderer(base, items, K, precision="fp32")
    d = to_dev(cat)
    out = br.forward(d["centers"], d["scales"], d["quats"], br.pack(d["weights"]))
    torch.cuda.synchronize()
    assert br.status() == 0
    for i, (c, sc, it) in enumerate(zip(cfgs, scenes, items)):
        rgb_o, T_o, F_o = oracle.render(c, sc, [it[2]])
        assert np.abs(br.split(out["rgb"])[i].cpu().numpy().reshape(-1, 3) - rgb_o).max() < 1e-4, i
        assert np.abs(br.split(out["trans"])[i].cpu().numpy().reshape(-1) - T_o).max() < 1e-4, i
        f = br.split(out["feat"])[i].cpu().numpy().reshape(-1, 16)
        assert np.abs(f - F_o).max() < 1e-4, i
