"""CPU-only checks of the C ABI: the library builds, loads and exports every declared symbol,
and its host-side shape/validation logic agrees with the documented layouts. No CUDA work is
enqueued here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_03877_gb300 import _lib, build, synth
from paper_2606_03877_gb300.render import make_config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return _lib.load(path)


def _declared():
    txt = open(os.path.join(ROOT, "include", "mlps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mlps_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.exported_symbols())


def test_abi_version_and_status_strings(lib):
    assert _lib.mlps_abi_version() == 7
    for s in range(8):
        assert _lib.mlps_status_string(s)
    assert _lib.mlps_status_string(4) == "hit capacity overflow"


@pytest.mark.parametrize("name", ["pr1", "diff", "prec", "stress"])
def test_param_count_and_stride(lib, name):
    c = synth.CONFIGS[name]
    cfg = make_config(c)
    assert _lib.mlps_param_count(cfg) == c.n_params
    assert _lib.mlps_input_dim(cfg) == c.input_dim
    assert _lib.mlps_weight_stride(cfg) % 256 == 0
    assert _lib.mlps_weight_stride(cfg) >= 4 * c.n_params
    sb, tb = _lib.mlps_workspace_size(cfg, c.K, _lib.cameras(synth.make_cameras(c)), c.n_views)
    assert sb > 0 and tb > 0 and sb % 256 == 0 and tb % 256 == 0


def test_config_validation(lib):
    base = synth.CONFIGS["prec"]
    bad = [("samples", 0), ("samples", 129), ("max_hits_per_ray", 0), ("max_hits_per_ray", 65),
           ("hidden_layers", 0), ("feat_dim", 33), ("t_eps", -1.0), ("hit_capacity_per_ray", 0.0),
           ("precision", 7)]
    for field, val in bad:
        cfg = make_config(base)
        setattr(cfg, field, val)
        assert _lib.mlps_check_config(cfg) == _lib.MLPS_ERR_INVALID_ARGUMENT, field
    cfg = make_config(base)
    cfg.hidden_width = 48
    assert _lib.mlps_check_config(cfg) == _lib.MLPS_ERR_UNSUPPORTED
    for wave in (-1, 65):
        cfg = make_config(base)
        cfg.early_stop_wave = wave
        assert _lib.mlps_check_config(cfg) == _lib.MLPS_ERR_INVALID_ARGUMENT
    cfg = make_config(base, early_stop_wave=4)
    assert _lib.mlps_check_config(cfg) == _lib.MLPS_OK
    cfg.slot_dim = 8
    assert _lib.mlps_check_config(cfg) == _lib.MLPS_ERR_UNSUPPORTED


def test_camera_validation(lib):
    c = synth.CONFIGS["prec"]
    cfg = make_config(c)
    cams = synth.make_cameras(c.replace(n_views=2))
    cams[1] = dict(cams[1], width=100)
    with pytest.raises(_lib.MlpsError) as e:
        _lib.mlps_workspace_size(cfg, 10, _lib.cameras(cams), 2)
    assert e.value.status == _lib.MLPS_ERR_UNSUPPORTED
    cams = synth.make_cameras(c.replace(n_views=1))
    cams[0] = dict(cams[0], fx=float("nan"))
    with pytest.raises(_lib.MlpsError):
        _lib.mlps_workspace_size(cfg, 10, _lib.cameras(cams), 1)
    with pytest.raises(_lib.MlpsError):
        _lib.mlps_workspace_size(cfg, 10, _lib.cameras(synth.make_cameras(c.replace(n_views=1))), 65)


def test_library_fails_loudly_when_missing(tmp_path):
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_sample_pixels_uniform_over_views():
    c = synth.CONFIGS["prec"]
    p = synth.sample_pixels(c, 4000, seed=3)
    assert len(p) == 4000 and len(np.unique(p, axis=0)) == 4000
    counts = np.bincount(p[:, 0], minlength=c.n_views)
    assert counts.min() > 0.7 * 4000 / c.n_views


def test_batch_workspace_matches_single_scene_layout(lib):
    """A batch whose items all render the whole scene at one resolution is the single-scene
    multi-view call: same workspace."""
    c = synth.CONFIGS["prec"].replace(width=320, height=200, n_views=3)
    cfg = make_config(c)
    cams = synth.make_cameras(c)
    single = _lib.mlps_workspace_size(cfg, c.K, _lib.cameras(cams), 3)
    items = _lib.batch_items([(0, c.K, cam) for cam in cams])
    assert _lib.mlps_batch_workspace_size(cfg, c.K, items, 3) == single


def test_batch_item_validation(lib):
    c = synth.CONFIGS["prec"].replace(width=64, height=48, n_views=2)
    cfg = make_config(c)
    cams = synth.make_cameras(c)
    ok = _lib.batch_items([(0, 10, cams[0]), (10, 20, cams[1])])
    sb, tb = _lib.mlps_batch_workspace_size(cfg, 30, ok, 2)
    assert sb > 0 and tb > 0
    for bad in ([(0, 10, cams[0]), (25, 10, cams[1])], [(-1, 5, cams[0])], [(0, -2, cams[0])]):
        with pytest.raises(_lib.MlpsError) as e:
            _lib.mlps_batch_workspace_size(cfg, 30, _lib.batch_items(bad), len(bad))
        assert e.value.status == _lib.MLPS_ERR_INVALID_ARGUMENT
    # mixed resolutions are allowed in a batch
    big = dict(cams[1], width=128, height=96, cx=64.0, cy=48.0)
    _lib.mlps_batch_workspace_size(cfg, 30, _lib.batch_items([(0, 10, cams[0]), (10, 20, big)]), 2)


def test_device_table_workspace_and_validation(lib):
    """A device-table batch is sized as a host table whose items all sit at the caps; the host
    checks the caps and the item count (the items themselves are checked on the device)."""
    c = synth.CONFIGS["prec"].replace(width=80, height=64, n_views=3)
    cfg = make_config(c)
    cams = synth.make_cameras(c)
    host = _lib.mlps_batch_workspace_size(cfg, 90, _lib.batch_items([(0, 30, cam) for cam in cams]), 3)
    assert _lib.mlps_batch_workspace_size_dev(cfg, 90, 3, _lib.batch_caps(80, 64, 30)) == host
    for n, caps in ((3, (0, 64, 30)), (3, (80, -1, 30)), (3, (80, 64, -1)), (0, (80, 64, 30)),
                    (65, (80, 64, 30)), (3, (20000, 64, 30))):
        with pytest.raises(_lib.MlpsError) as e:
            _lib.mlps_batch_workspace_size_dev(cfg, 90, n, _lib.batch_caps(*caps))
        assert e.value.status == _lib.MLPS_ERR_INVALID_ARGUMENT
    # a null item table is refused before any launch
    scene = _lib.MlpsScene(0, None, None, None, None)
    st = lib.mlps_render_batch_forward_dev(ctypes.byref(cfg), ctypes.byref(scene), None, 3,
                                           ctypes.byref(_lib.batch_caps(80, 64, 30)), None, None, None, None, 0,
                                           None, 0, None)
    assert st == _lib.MLPS_ERR_INVALID_ARGUMENT


def test_selftest_bounded_wait_validates_on_the_host(lib):
    """Argument errors come back before any launch (no GPU needed)."""
    assert lib.mlps_selftest_bounded_wait(1000, None, 4096, None) == _lib.MLPS_ERR_INVALID_ARGUMENT
    assert lib.mlps_selftest_bounded_wait(0, ctypes.c_void_p(256), 4096, None) == _lib.MLPS_ERR_INVALID_ARGUMENT
    assert lib.mlps_selftest_bounded_wait(2000000, ctypes.c_void_p(256), 4096, None) == \
        _lib.MLPS_ERR_INVALID_ARGUMENT
    assert lib.mlps_selftest_bounded_wait(1000, ctypes.c_void_p(256), 128, None) == _lib.MLPS_ERR_INVALID_ARGUMENT
    assert lib.mlps_selftest_bounded_wait(1000, ctypes.c_void_p(260), 4096, None) == _lib.MLPS_ERR_INVALID_ARGUMENT


def test_contact_mode_validation(lib):
    """Contact-point mode (Sec. 3.2) takes one sample per hit; its forward and backward run in
    every precision."""
    c = synth.CONFIGS["contact"]
    assert _lib.mlps_check_config(make_config(c)) == _lib.MLPS_OK
    assert _lib.mlps_check_config(make_config(c.replace(samples=2))) == _lib.MLPS_ERR_INVALID_ARGUMENT
    cfg = make_config(c)
    cfg.contact = 2
    assert _lib.mlps_check_config(cfg) == _lib.MLPS_ERR_INVALID_ARGUMENT
    for prec in ("bf16", "fp8"):  # forward on the tensor cores (32-wide hidden layers padded to 64)
        assert _lib.mlps_check_config(make_config(c, prec)) == _lib.MLPS_OK
    assert _lib.mlps_param_count(make_config(c)) == 72 * 32 + 32 + 32 * 32 + 32 + 32 * 4 + 4


def test_mlp_groups_validation(lib):
    base = synth.CONFIGS["prec"]
    for g, want in ((1, _lib.MLPS_ERR_INVALID_ARGUMENT), (7, _lib.MLPS_ERR_INVALID_ARGUMENT),
                    (2, _lib.MLPS_OK), (3, _lib.MLPS_OK), (4, _lib.MLPS_OK), (5, _lib.MLPS_OK),
                    (6, _lib.MLPS_ERR_UNSUPPORTED)):  # BF16 groups also keep their A operand in TMEM
        assert _lib.mlps_check_config(make_config(base, "bf16", mlp_groups=g)) == want, g
    for g in (2, 6):  # E4M3 keeps its operands in shared memory: up to six groups
        assert _lib.mlps_check_config(make_config(base, "fp8", mlp_groups=g)) == _lib.MLPS_OK, g
    # wider models and feature heads run with their default only
    assert _lib.mlps_check_config(make_config(synth.CONFIGS["stress"], "bf16", mlp_groups=3)) == \
        _lib.MLPS_ERR_UNSUPPORTED
    assert _lib.mlps_check_config(make_config(synth.CONFIGS["stress"], "bf16", mlp_groups=2)) == _lib.MLPS_OK
    # the FP32 path has no groups; the field is accepted and ignored
    assert _lib.mlps_check_config(make_config(base, "fp32", mlp_groups=3)) == _lib.MLPS_OK


def test_training_entry_points_validate_on_the_host(lib):
    """mlps_loss_workspace_size / mlps_loss / mlps_adam_step reject bad arguments before any
    device work (no GPU needed)."""
    ok = _lib.loss_desc(2, 45, 70, 8, None, 0.2, 0)
    assert _lib.mlps_loss_workspace_size(ok) == 256 + ((9 * 2 * 45 * 70 * 4 + 255) // 256) * 256
    for bad in (_lib.loss_desc(0, 45, 70), _lib.loss_desc(1, 45, 70, 0), _lib.loss_desc(1, 45, 70, 8, None, 1.5),
                _lib.loss_desc(1, 45, 70, 8, None, 0.2, -1)):
        assert _lib.mlps_loss_workspace_size(bad) == 0
    with pytest.raises(_lib.MlpsError) as e:
        _lib.mlps_loss(ok, None, None, None, None, None, None, None, None, 0)
    assert e.value.status == _lib.MLPS_ERR_INVALID_ARGUMENT
    with pytest.raises(_lib.MlpsError) as e:  # no groups
        _lib.mlps_adam_step([], 0.9, 0.999, 1e-15, 1)
    assert e.value.status == _lib.MLPS_ERR_INVALID_ARGUMENT
    g = _lib.MlpsAdamGroup(None, None, None, None, None, 10, 1e-3, 0)  # n > 0 without pointers
    with pytest.raises(_lib.MlpsError) as e:
        _lib.mlps_adam_step([g], 0.9, 0.999, 1e-15, 1)
    assert e.value.status == _lib.MLPS_ERR_INVALID_ARGUMENT
    g0 = _lib.MlpsAdamGroup(None, None, None, None, None, 0, 1e-3, 0)
    for args in ((1.0, 0.999, 1e-15, 1), (0.9, 0.999, 1e-15, 0)):  # beta1 = 1, step 0
        with pytest.raises(_lib.MlpsError) as e:
            _lib.mlps_adam_step([g0], *args)
        assert e.value.status == _lib.MLPS_ERR_INVALID_ARGUMENT


def test_slot_and_tile_order_config_validation(lib):
    c = synth.CONFIGS["contact"]
    assert _lib.mlps_check_config(make_config(c.replace(slot_dim=512))) == _lib.MLPS_OK
    assert _lib.mlps_check_config(make_config(c.replace(slot_dim=6))) == _lib.MLPS_ERR_UNSUPPORTED
    assert _lib.mlps_check_config(make_config(c.replace(slot_dim=4096))) == _lib.MLPS_ERR_INVALID_ARGUMENT
    assert _lib.mlps_param_count(make_config(c.replace(slot_dim=512))) == c.n_mlp_params + 4 * 512
    cfg = make_config(c.replace(tile_sort=8))
    assert cfg.tile_sort == 1 and cfg.tile == 8 and _lib.mlps_check_config(cfg) == _lib.MLPS_OK
    cfg.tile_sort = 2
    assert _lib.mlps_check_config(cfg) == _lib.MLPS_ERR_INVALID_ARGUMENT
