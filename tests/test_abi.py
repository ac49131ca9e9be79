"""The C-ABI library builds, loads without a GPU, and exports every symbol include/xg.h
declares; its host-only argument checks work.  No call here touches a GPU."""
import ctypes
import os
import re

import pytest

from paper_2403_04116_gb300 import binding as B
from paper_2403_04116_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "xg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.lib()


def test_header_declares_the_binding_names():
    assert _declared() == sorted(B.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(build.LIB)
    for name in _declared():
        assert hasattr(raw, name), name


def test_workspace_bytes_host_checks(lib):
    cfg = B.XgConfig(16, 16, 0.2, 0, 1 << 20)
    small = B.xg_workspace_bytes(cfg, 1000, 2, 64, 64)
    big = B.xg_workspace_bytes(cfg, 1000, 4, 64, 64)
    assert 0 < small < big
    assert B.xg_workspace_bytes(cfg, 0, 1, 64, 64) == 0
    assert B.xg_workspace_bytes(cfg, 10, 1, 0, 64) == 0
    assert B.xg_workspace_bytes(B.XgConfig(32, 32, 0.2, 0, 100, 2, 0), 10, 1, 64, 64) > 0
    for bad in (B.XgConfig(12, 16, 0.2, 0, 100), B.XgConfig(32, 32, 0.2, 0, 100, 1, 0),
                B.XgConfig(16, 16, 0.0, 0, 100), B.XgConfig(16, 16, 0.2, 0, 0),
                B.XgConfig(16, 16, float("nan"), 0, 100), B.XgConfig(16, 16, 0.2, 100, 100),
                B.XgConfig(16, 16, 0.2, 0, 100, 3, 0), B.XgConfig(16, 8, 0.2, 0, 100, 4, 0)):
        assert B.xg_workspace_bytes(bad, 10, 1, 64, 64) == 0


def test_pairs_cost_one_index_each(lib):
    # the pairs are written once, as 4-byte Gaussian indices at their final place: no key
    # array and no second buffer, so pair capacity costs exactly 4 bytes a pair
    def ws(cap, tile=(16, 16), W=64):
        return B.xg_workspace_bytes(B.XgConfig(tile[0], tile[1], 0.2, 0, cap), 1000, 3, W, W)
    for tile, W in (((16, 16), 64), ((8, 8), 1024), ((32, 16), 512)):
        assert ws((1 << 20) + 4096, tile, W) - ws(1 << 20, tile, W) == 4 * 4096
        assert ws((1 << 24) + 64, tile, W) - ws(1 << 24, tile, W) == 4 * 64


def test_workspace_of_a_scan_rendered_in_passes(lib):
    def ws(V, per_pass):
        return B.xg_workspace_bytes(B.XgConfig(16, 16, 0.2, 0, 1 << 20, 2, per_pass), 1000, V, 64, 64)
    # per-pass arrays follow the views of one pass; only the 64-byte camera table grows
    one_pass = ws(8, 0)
    assert ws(8, 8) == ws(8, 100) == one_pass
    assert ws(360, 8) - one_pass == pytest.approx(64 * 352, abs=512)
    assert ws(360, 8) < ws(360, 16) < ws(360, 0)
    assert ws(8, -1) == 0


def test_select_views_rejects_a_null_frame(lib):
    with pytest.raises(B.XgError) as e:
        B.xg_frame_select_views(None, 0)
    assert e.value.code == B.XG_ERR_INVALID_ARG


def test_frame_create_rejects_bad_arguments_before_touching_the_device(lib):
    from paper_2403_04116_gb300.synth import View
    cfg = B.XgConfig(16, 16, 0.2, 0, 1000)
    good = View(1000.0, 1500.0, 1.0, 1.0, 0.0, 64, 64)
    cases = [
        [View(1000.0, 1500.0, 1.0, 1.0, 0.0, 64, 64), View(1000.0, 1500.0, 1.0, 1.0, 0.5, 32, 64)],  # sizes differ
        [View(-1.0, 1500.0, 1.0, 1.0, 0.0, 64, 64)],
        [View(1000.0, 1500.0, 0.0, 1.0, 0.0, 64, 64)],
        [View(1000.0, 1500.0, 1.0, 1.0, float("inf"), 64, 64)],
        [View(1000.0, 1500.0, 1.0, 1.0, 0.0, 5000, 64)],
    ]
    for views in cases:
        with pytest.raises(B.XgError) as e:
            B.xg_frame_create(cfg, 10, views, 0, 1 << 30, 0)
        assert e.value.code == B.XG_ERR_INVALID_ARG
    # a missing or short workspace is refused
    with pytest.raises(B.XgError) as e:
        B.xg_frame_create(cfg, 10, [good], 0, 1 << 30, 0)
    assert e.value.code == B.XG_ERR_WORKSPACE
    with pytest.raises(B.XgError) as e:
        B.xg_frame_create(cfg, 10, [good], 256, 16, 0)
    assert e.value.code == B.XG_ERR_WORKSPACE


def test_status_strings(lib):
    assert B.xg_status_str(B.XG_OK) == "ok"
    assert "capacity" in B.xg_status_str(B.XG_ERR_CAPACITY)


def test_fdk_argument_checks_before_any_device_work(lib):
    from paper_2403_04116_gb300.synth import View, circular_views
    views = circular_views(8, 32, 32)
    vol = B.XgVolume(16, 16, 16, 0, 1.0)
    assert B.xg_fdk_workspace_bytes(8, 32, 32) > 8 * 32 * 32 * 4
    assert B.xg_fdk_workspace_bytes(0, 32, 32) == 0
    bad = list(views)
    bad[3] = View(900.0, 1500.0, 1.0, 1.0, 0.3, 32, 32)  # another scanner distance
    for vs, v, code in ((bad, vol, B.XG_ERR_INVALID_ARG), (views, B.XgVolume(0, 16, 16, 0, 1.0), B.XG_ERR_INVALID_ARG),
                        (views, vol, B.XG_ERR_WORKSPACE)):
        with pytest.raises(B.XgError) as e:
            B.xg_fdk(vs, 1 << 20, v, 1 << 20, 0, 0, 0)
        assert e.value.code == code
