"""Binning paths that the small parity scenes do not reach, bit-exact against the FP32
replica (the same expected index as test_gpu_parity.py: the replica's per-view tile lists
laid out in (tile, view) order):

* tile grids larger than one group of the pair scatter (2,048 tiles, whole rows): 8x8
  tiles on 512x512 (4,096 tiles, two groups of 32 rows) and on 1024x512 (8,192 tiles,
  four groups of 16 rows);
* Gaussian counts that are not a multiple of 4, so the sorted entries of every view after
  the first start off a 16-byte boundary (the radix scatter loads those chunks directly
  instead of by bulk copy), and views cut into many units of sorted entries;
* Gaussians as large as the scene (a fifth to a half of its side): most cover hundreds of
  the 1,024 tiles of a view, so the pair scatter takes every unit's entries in many chunks
  of a few entries each;
* culled entries (key 0) among the sorted ones, in a scene whose depths share their top
  byte (the entry sort's last pass is then a copy) and in one whose depths cross 512 mm (it
  is not);
* a scan whose last pass has fewer views but more radix blocks than a full pass: 36 views,
  19 per pass (608 blocks) and a last pass of 17 (612 blocks); every view equals the same
  view rendered by a frame of its own, and the last one equals the replica.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2403_04116_gb300 import binding as B  # noqa: E402
from paper_2403_04116_gb300 import synth  # noqa: E402
from paper_2403_04116_gb300.render import Frame, FrameConfig  # noqa: E402
from paper_2403_04116_gb300.synth import View  # noqa: E402
from tests.gpu_util import run_forward, to_device  # noqa: E402
from tests.test_gpu_parity import _expected_index  # noqa: E402

pytestmark = pytest.mark.gpu

# (Gaussians, views, W, H, tile, workload id)
CASES = {
    "two_groups_512_8x8": (20_001, 3, 512, 512, (8, 8), 21),
    "four_groups_1024x512_8x8": (12_003, 2, 1024, 512, (8, 8), 22),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2403_04116_gb300 import build
    build.build()
    oracle.lib()


@pytest.mark.parametrize("name", sorted(CASES))
def test_large_tile_grids_bit_exact(name):
    n, V, W, H, tile, cid = CASES[name]
    g = synth.gaussians(n, synth.scene_side_mm(min(W, H)), synth.rng(cid, 0))
    views = synth.circular_views(V, W, H, first_rad=0.1 * cid)
    gpu = run_forward(g, views, tile)
    f = gpu["frame"]
    T = f.tiles_per_view
    assert T > 2048  # more than one group of tile rows
    reps, idx = _expected_index(g, views, tile)
    assert gpu["status"].code == B.XG_OK
    assert gpu["M"] == idx["M"] > 100_000
    np.testing.assert_array_equal(gpu["key_tile"], idx["key_tile"])
    np.testing.assert_array_equal(gpu["value"], idx["value"])
    np.testing.assert_array_equal(gpu["range"], idx["range"])
    for v, r in enumerate(reps):
        np.testing.assert_array_equal(gpu["image"][v].view(np.uint32), r["image"].view(np.uint32))
        np.testing.assert_array_equal(gpu["last"][v].view(np.uint32), r["last"])


def test_scene_sized_gaussians_bit_exact():
    n, V, W, tile, cid = 2_001, 2, 256, (8, 8), 24
    g = synth.gaussians(n, synth.scene_side_mm(W), synth.rng(cid, 0), log_scale=(-1.6, -0.7))
    views = synth.circular_views(V, W, W, first_rad=0.3)
    gpu = run_forward(g, views, tile)
    reps, idx = _expected_index(g, views, tile)
    assert gpu["status"].code == B.XG_OK
    assert gpu["M"] == idx["M"] > 300 * n * V  # hundreds of tiles per Gaussian on average
    np.testing.assert_array_equal(gpu["key_tile"], idx["key_tile"])
    np.testing.assert_array_equal(gpu["value"], idx["value"])
    np.testing.assert_array_equal(gpu["range"], idx["range"])
    for v, r in enumerate(reps):
        np.testing.assert_array_equal(gpu["image"][v].view(np.uint32), r["image"].view(np.uint32))


@pytest.mark.parametrize("sod,side", [(1000.0, 42.7), (600.0, 200.0)])
def test_culled_entries_and_the_depth_span(sod, side):
    n, V, W, tile, cid = 6_001, 3, 128, (16, 16), 25
    g = synth.gaussians(n, side, synth.rng(cid, 0))
    g["opacity"][::3] = 0.003  # below 1/255: culled in projection, depth key 0
    views = [View(sod, 1100.0, 1.0, 1.0, 0.4 * k, W, W) for k in range(V)]
    gpu = run_forward(g, views, tile)
    depth = gpu["depth"].reshape(V, n)
    live = depth[depth > 0]
    assert (depth == 0).sum() >= n // 3 * V and live.size > 1000
    crosses = bool(live.min() < 512.0 <= live.max())
    assert crosses == (sod < 1000.0)  # the first scene's depths share the top byte of their bits
    reps, idx = _expected_index(g, views, tile)
    assert gpu["status"].code == B.XG_OK
    assert gpu["M"] == idx["M"] > 10_000
    np.testing.assert_array_equal(gpu["key_tile"], idx["key_tile"])
    np.testing.assert_array_equal(gpu["value"], idx["value"])
    np.testing.assert_array_equal(gpu["range"], idx["range"])
    for v, r in enumerate(reps):
        np.testing.assert_array_equal(gpu["image"][v].view(np.uint32), r["image"].view(np.uint32))


def test_ragged_pass_with_more_radix_blocks():
    # 37 radix tiles per view: enough for ceil(608 / 19) = 32 and ceil(608 / 17) = 36 CTAs per
    # view (a pass's CTAs never outnumber its tiles)
    n, V, W, VPP = 75_001, 36, 96, 19
    g = synth.gaussians(n, synth.scene_side_mm(W), synth.rng(23, 0))
    views = synth.circular_views(V, W, W)
    dev = to_device(g)
    cfg = FrameConfig(16, 16)
    f = Frame(n, views, cfg, 1 << 23, views_per_pass=VPP)
    image = torch.full((V, W, W), -1.0, device="cuda")
    for first in (0, VPP):
        nv = f.select(first)
        assert nv == (VPP if first == 0 else V - VPP)
        f.project(*dev)
        f.bin_sort()
        f.render_fwd(image[first:first + nv])
        assert f.status().code == B.XG_OK
    f.select(0)
    for v in (0, 18, 19, 27, 35):
        one = Frame(n, [views[v]], cfg, 1 << 21)
        one.project(*dev)
        one.bin_sort()
        img = torch.empty(1, W, W, device="cuda")
        one.render_fwd(img)
        assert one.status().code == B.XG_OK
        assert torch.equal(img[0], image[v]), v
    rep = oracle.replica_full(g, views[35], (16, 16))
    np.testing.assert_array_equal(image[35].cpu().numpy().view(np.uint32), rep["image"].view(np.uint32))


def _length_bucket(n: np.ndarray) -> np.ndarray:
    """Four buckets per octave of list length: 0 for an empty list, else 1 + 4 floor(log2 n)
    + the two bits below the leading one."""
    n = n.astype(np.int64)
    out = np.zeros(n.shape, np.int64)
    nz = n > 0
    lead = np.floor(np.log2(np.where(nz, n, 1))).astype(np.int64)
    frac = np.where(lead >= 2, (n >> np.maximum(lead - 2, 0)) & 3, (n << np.maximum(2 - lead, 0)) & 3)
    out[nz] = 1 + 4 * lead[nz] + frac[nz]
    return out


@pytest.mark.parametrize("views_n,tile", [(50, (16, 8)), (7, (8, 8))])
def test_work_order_is_longest_first_permutation(views_n, tile):
    """The compositing work items: every (view, tile) exactly once, by non-increasing bucket
    of list length (more items than the ordering CTA's threads times its unroll)."""
    n, W, cid = 8_000, 256, 26
    g = synth.gaussians(n, synth.scene_side_mm(W), synth.rng(cid, 0))
    views = synth.circular_views(views_n, W, W)
    gpu = run_forward(g, views, tile)
    f = gpu["frame"]
    T = int(f.layout.tiles_per_view)
    items = views_n * T
    order = f.array("order").cpu().numpy().view(np.uint32).astype(np.int64)
    assert order.size == items and (items > 8 * 1024) == (views_n == 50)
    np.testing.assert_array_equal(np.sort(order), np.arange(items))
    v, t = order // T, order % T
    rng = gpu["range"].astype(np.int64)
    length = rng[v * f.range_stride + t, 1] - rng[v * f.range_stride + t, 0]
    b = _length_bucket(length)
    assert (np.diff(b) <= 0).all()
    assert b[0] == _length_bucket(np.array([length.max()]))[0] and length.max() > 0
