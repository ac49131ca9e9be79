"""Pins of the FP32 replica (the bit-exact reference for the GPU's index work).

The replica is checked against the FP64 oracle and against properties of the method:
its exp/log against NumPy, its images against the oracle within the FP32 budget, its
tile lists against brute-force invariants, and the fact that tiles are pure
acceleration: the image must not depend on the tile size at all.
"""
import numpy as np
import pytest

import oracle
from paper_2403_04116_gb300 import synth
from paper_2403_04116_gb300.synth import View


def test_exp_accuracy(oracle_lib):
    x = np.concatenate([np.linspace(-80, 0, 400001, dtype=np.float32), np.float32([0.0, -1e-30, -5.54, 1e-7])])
    y = oracle.replica_exp(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    assert np.max(np.abs(y / ref - 1)) < 4e-7  # degree-6 Taylor bound 1.2e-7 plus float rounding
    assert oracle.replica_exp(np.float32([0.0]))[0] == 1.0


def test_exp_at_the_reduction_boundaries(oracle_lib):
    # x log2 e within a few ulps of k + 1/2: the remainder is near +-ln2/2, the polynomial's
    # worst case, and rint switches k there.  Every float in a window around each boundary
    # above the clamp at x = -80 (k = -114 .. 0): within the error bound of FP64 exp, and
    # non-decreasing across the switch
    xs = []
    for k in range(-114, 1):
        c = np.float32((k - 0.5) / np.log2(np.e))
        b = c.view(np.uint32).astype(np.int64)
        xs.append(np.arange(b - 40, b + 41).astype(np.uint32).view(np.float32))
    for x in xs:
        x = np.sort(x)
        y = oracle.replica_exp(x)
        ref = np.exp(x.astype(np.float64))
        assert np.max(np.abs(y.astype(np.float64) / ref - 1)) < 4e-7
        assert np.all(np.diff(y.astype(np.float64)) >= 0), x[0]


def test_log_accuracy(oracle_lib):
    x = np.concatenate([np.linspace(1, 255, 200001, dtype=np.float32), np.float32([1.0, 1.4142135, 1.4142137, 2])])
    y = oracle.replica_log(x).astype(np.float64)
    assert np.max(np.abs(y - np.log(x.astype(np.float64)))) < 2e-6
    assert oracle.replica_log(np.float32([1.0]))[0] == 0.0


def _config0(n=10_000, W=128, angle=0.0, cid=0):
    gen = synth.rng(cid, 0)
    g = synth.gaussians(n, synth.scene_side_mm(W), gen)
    return g, synth.circular_views(1, W, W, first_rad=angle)[0]


@pytest.mark.parametrize("angle", [0.0, 2.1])
def test_replica_matches_fp64_oracle(oracle_lib, angle):
    g, v = _config0(angle=angle)
    rep = oracle.replica_full(g, v)
    ref = oracle.render64(g, v)
    amb = ref["ambiguous"] != 0
    err = np.abs(rep["image"].astype(np.float64) - ref["image"])
    assert np.max(err[~amb]) <= 1e-4
    assert np.max(err) <= 1e-2
    same = rep["ncontrib"].astype(np.int64) == ref["ncontrib"]
    assert np.all(same[~amb])
    assert amb.mean() < 0.05
    assert rep["ncontrib"].max() > 50  # the workload blends deep stacks


def test_image_independent_of_tile_size(oracle_lib):
    g, v = _config0(n=4000, W=96, cid=3)
    base = oracle.replica_full(g, v, tile=(96, 96))
    for tile in [(8, 8), (16, 16), (32, 16)]:
        r = oracle.replica_full(g, v, tile=tile)
        np.testing.assert_array_equal(r["image"], base["image"])
        np.testing.assert_array_equal(r["ncontrib"], base["ncontrib"])
        np.testing.assert_array_equal(r["tfinal"], base["tfinal"])


def test_tile_lists_are_consistent(oracle_lib):
    g, v = _config0(n=3000, W=64, cid=4)
    r = oracle.replica_full(g, v, tile=(16, 16))
    rng, lst, cnt, depth = r["range"], r["list"], r["count"], r["depth"]
    assert int((rng[:, 1] - rng[:, 0]).astype(np.int64).sum()) == r["M"] == int(cnt.astype(np.int64).sum())
    np.testing.assert_array_equal(np.bincount(lst, minlength=len(cnt)), cnt)
    dbits = depth.view(np.uint32)
    for t in range(rng.shape[0]):
        b, e = rng[t]
        seg = lst[b:e]
        key = dbits[seg].astype(np.uint64) << np.uint64(32) | seg.astype(np.uint64)
        assert np.all(np.diff(key.astype(np.int64)) > 0)
        tx, ty = t % 4, t // 4
        rc = r["rect"][seg]
        assert np.all((rc[:, 0] <= tx) & (tx <= rc[:, 2]) & (rc[:, 1] <= ty) & (ty <= rc[:, 3]))


def test_tile_rect_contains_every_included_pixel(oracle_lib):
    gen = np.random.default_rng(5)
    W = H = 48
    side = synth.scene_side_mm(W)
    g = synth.gaussians(60, side, gen, log_scale=(-3.0, -1.5), opacity=(0.01, 0.99))
    v = View(1000.0, 1500.0, 1.0, 1.0, 0.4, W, H)
    p32 = oracle.replica_project(g, v, tile=(8, 8))
    p64 = oracle.project64(g, v)
    yy, xx = np.mgrid[0:H, 0:W]
    for k in range(60):
        if not p64[k, 0]:
            continue
        dx, dy = p64[k, 4] - (xx + 0.5), p64[k, 5] - (yy + 0.5)
        a, b, c = p64[k, 9:12]
        alpha = g["opacity"][k] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
        inside = alpha >= 1 / 255
        if not inside.any():
            continue
        assert p32["count"][k] > 0
        x0, y0, x1, y1 = p32["rect"][k]
        ys, xs = np.nonzero(inside)
        assert np.all((xs // 8 >= x0) & (xs // 8 <= x1) & (ys // 8 >= y0) & (ys // 8 <= y1))


def test_nonfinite_and_degenerate_inputs_are_culled(oracle_lib):
    gen = np.random.default_rng(6)
    g = synth.gaussians(8, 40.0, gen)
    g["mean"][0, 1] = np.nan
    g["scale"][2, 2] = np.inf
    g["quat"][:, 3] = 0.0
    g["opacity"][4] = 0.001  # below 1/255: can never contribute
    g["mean"][0, 5] = 2000.0  # behind the source (t_z < 0 at angle 0)
    v = View(1000.0, 1500.0, 1.0, 1.0, 0.0, 64, 64)
    p = oracle.replica_project(g, v)
    assert p["nonfinite"] == 2
    assert np.all(p["count"][[1, 2, 3, 4, 5]] == 0)
    assert np.all(p["rec"][[1, 2, 3, 4, 5]] == 0)
    assert np.all(p["count"][[0, 6, 7]] > 0)
