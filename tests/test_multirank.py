"""The multi-rank (one process per GPU) host logic of the benchmark, on CPU with gloo and two
ranks: each rank renders its own views (weak scaling), the job's time is the slowest rank's,
the sharded renders together equal one render of all the views, and the backward's one
exchange (the sum all-reduce of the per-primitive gradients) gives the gradient of the whole
job. Rendering here is the FP64 oracle on a tiny image (what needs no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2606_03877_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wl = synth.CONFIGS["prec"].replace(width=24, height=16, K=10, n_views=2)
        scene = synth.make_scene(wl, 0)
        cams = synth.make_cameras(wl, first_view_seed=bench.rank_view_seed(rank, wl.n_views))
        rgb, trans, _ = oracle.render(wl, scene, cams, n_threads=1)
        # gather every rank's images (the test's check only; the benchmark has no collective on
        # the data path)
        t = torch.from_numpy(rgb)
        parts = [torch.empty_like(t) for _ in range(ws)]
        dist.all_gather(parts, t)
        slowest = bench.max_over_ranks(10.0 * (rank + 1), ws)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.concatenate([p.numpy() for p in parts], axis=0))
        np.save(os.path.join(out_dir, f"time{rank}.npy"), np.array([slowest]))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing(tmp_path):
    ws, port = 2, _free_port()
    mp.start_processes(_worker, args=(ws, port, str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    full_cfg = synth.CONFIGS["prec"].replace(width=24, height=16, K=10, n_views=2 * ws)
    scene = synth.make_scene(full_cfg, 0)
    ref, _, _ = oracle.render(full_cfg, scene, synth.make_cameras(full_cfg), n_threads=1)
    for r in range(ws):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert np.array_equal(got, ref)  # rank r's views are views [2r, 2r + 2) of the job
        assert float(np.load(tmp_path / f"time{r}.npy")[0]) == 20.0  # every rank sees the max


def test_job_throughput_and_seeds():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rays_per_s(1000, 4, 5, 2000.0) == pytest.approx(10000.0)
    seeds = [set(range(bench.rank_view_seed(r, 8), bench.rank_view_seed(r, 8) + 8)) for r in range(4)]
    assert all(not (a & b) for i, a in enumerate(seeds) for b in seeds[i + 1:])
    assert bench.rank_scene_seed(1) == 32 and bench.rank_scene_seed(0) == 0


def test_hit_capacity_per_workload():
    """Hit records reserved per ray: 16 for the 1024-primitive scene (about eight hits per ray
    at 1080p, more at low resolution), 8 otherwise, or the explicit --hit-capacity."""
    import sys
    import types
    sys.path.insert(0, ROOT)
    import bench
    auto = types.SimpleNamespace(hit_capacity=0.0)
    assert bench.hit_capacity(auto, synth.CONFIGS["stress"]) == 16.0
    assert bench.hit_capacity(auto, synth.CONFIGS["prec"]) == 8.0
    assert bench.hit_capacity(types.SimpleNamespace(hit_capacity=12.0), synth.CONFIGS["prec"]) == 12.0


def _grad_worker(rank, ws, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wl = synth.CONFIGS["prec"].replace(width=12, height=10, K=6, n_views=1)
        scene = synth.make_scene(wl, 0)
        scene = dict(scene, scales=(scene["scales"] * 3.0))
        cams = synth.make_cameras(wl, first_view_seed=bench.rank_view_seed(rank, wl.n_views))
        g = synth.make_grad((ws, wl.height * wl.width, 3), seed=9)[rank]
        ref = oracle.render_backward(wl, scene, cams, oracle.all_pixels(cams), g, None, None)
        P = ref["d_weights"].shape[1]
        flat, views = bench.grad_buffers(wl.K, P)
        for k, v in views.items():
            v.copy_(torch.from_numpy(np.asarray(ref[k], dtype=np.float32)))
        bench.allreduce_grads(flat, ws)
        np.save(os.path.join(out_dir, f"grad{rank}.npy"), flat.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_gradient_allreduce_is_the_job_gradient(tmp_path):
    """Data-parallel backward: rank r renders view r with its share of dL/dC; after the sum
    all-reduce every rank holds the gradient of the loss over both views (the oracle's, one
    process, both cameras)."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ws, port = 2, _free_port()
    mp.start_processes(_grad_worker, args=(ws, port, str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    wl = synth.CONFIGS["prec"].replace(width=12, height=10, K=6, n_views=ws)
    scene = synth.make_scene(wl, 0)
    scene = dict(scene, scales=(scene["scales"] * 3.0))
    cams = synth.make_cameras(wl)
    g = synth.make_grad((ws, wl.height * wl.width, 3), seed=9).reshape(-1, 3)
    ref = oracle.render_backward(wl, scene, cams, oracle.all_pixels(cams), g, None, None)
    want = np.concatenate([np.asarray(ref[k], dtype=np.float64).reshape(-1)
                           for k in ("d_weights", "d_centers", "d_scales", "d_quats")])
    assert np.abs(want).max() > 0
    for r in range(ws):
        got = np.load(tmp_path / f"grad{r}.npy").astype(np.float64)
        assert np.allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
