"""The multi-rank (one process per GPU) host logic of the benchmark, on CPU with gloo and two
ranks: each rank renders its own views (weak scaling, no data-path collective), the job's time
is the slowest rank's, and the sharded renders together equal one render of all the views.
Rendering here is the FP64 oracle on a tiny image (what needs no GPU)."""
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
