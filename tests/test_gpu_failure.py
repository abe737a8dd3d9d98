"""Failure detection on the GPU without a fault: the bounded wait every persistent tensor-core
kernel uses gives up on a barrier that nothing arrives at, reports MLPS_ERR_TIMEOUT through the
status word, and the device renders correctly right afterwards."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2606_03877_gb300 import _lib, synth
from paper_2606_03877_gb300.render import Renderer

from helpers import psnr, scaled_scene, to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports_timeout():
    scratch = torch.empty(4096, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lib.mlps_selftest_bounded_wait(50000, scratch)  # 50 ms
    st = _lib.mlps_read_status(scratch)  # synchronises
    dt = time.perf_counter() - t0
    assert st == _lib.MLPS_ERR_TIMEOUT
    assert 0.04 < dt < 5.0, dt  # it waited about its limit, then ended
    assert _lib.mlps_read_status(scratch) == _lib.MLPS_OK  # read and cleared
    # the context is usable: a BF16 render right afterwards matches the oracle
    cfg = synth.CONFIGS["prec"].replace(width=48, height=40, K=8, n_views=1)
    scene = scaled_scene(cfg, 51, 2.0)
    cams = synth.make_cameras(cfg, first_view_seed=51)
    r = Renderer(cfg, precision="bf16")
    d = to_dev(scene)
    out = r.forward(d["centers"], d["scales"], d["quats"], r.pack(d["weights"]), cams)
    torch.cuda.synchronize()
    assert r.status() == 0
    rgb_o, _, _ = oracle.render(cfg, scene, cams)
    assert psnr(out["rgb"].cpu().numpy().reshape(-1, 3), rgb_o) >= 45.0
