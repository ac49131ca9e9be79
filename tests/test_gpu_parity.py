"""Parity of the CUDA path (through the C ABI) with the oracle.

* index work -- records, depth keys, tile rectangles, counts, sorted pairs, tile ranges,
  contributor counts and last-contributor positions -- bit-exact against the FP32 replica;
* pixel values within 1e-4 absolute of the FP64 oracle (pixels where a blending decision
  sits within rounding of its threshold are allowed 1e-2, and counted);
* gradients within 1e-3 relative (1e-6 absolute floor) of the FP64 oracle's, plus the
  FP32 rounding allowance GRAD_TERM_REL * (sum of |per-pixel terms| behind the gradient):
  a gradient is a sum of per-pixel terms of both signs, and FP32 evaluates each term to a
  relative accuracy of about 3e-5 at worst (the transmittance is recovered by up to ~200
  successive divisions), so a sum that cancels to far below its terms cannot be held to
  1e-3 of itself by any FP32 implementation.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2403_04116_gb300 import binding as B  # noqa: E402
from paper_2403_04116_gb300 import synth  # noqa: E402
from paper_2403_04116_gb300.synth import View  # noqa: E402
from tests.gpu_util import (NAMES, PIXEL_STATS, grad_compare, merge_stats, run_backward, run_forward,  # noqa: E402
                            to_device)

pytestmark = pytest.mark.gpu

PIXEL_TOL = 1e-4
AMBIGUOUS_TOL = 1e-2
# pixels beyond 1e-4 of the FP64 oracle (all of them flagged ambiguous), as a fraction
OVER_TOL_FRAC_MAX = 1e-3
# Fraction of the gradients of these small scenes, under a random +-1 upstream gradient (the
# input that maximises cancellation), that must meet 1e-3 relative / 1e-6 absolute on their
# own, without the FP32 term allowance
STRICT_FRAC_MIN = 0.99


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2403_04116_gb300 import build
    build.build()
    oracle.lib()


# small cases: (Gaussians, views, W, H, tile, workload id)
CASES = {
    "one_view_128": (10_000, 1, 128, 128, (16, 16), 0),
    "ragged_5views_8x8": (3_000, 5, 100, 75, (8, 8), 10),
    "ragged_3views_32x16": (3_000, 3, 100, 75, (32, 16), 11),
    "tall_2views_16x32": (2_000, 2, 40, 90, (16, 32), 12),
}


def _case(name):
    n, V, W, H, tile, cid = CASES[name]
    g = synth.gaussians(n, synth.scene_side_mm(W), synth.rng(cid, 0))
    views = synth.circular_views(V, W, H, first_rad=0.1 * cid)
    return g, views, tile


def _expected_index(g, views, tile):
    """The frame's sorted pairs and ranges built from the replica's per-view tile lists: the
    (view, tile) lists laid out in (tile, view) order, keyed view * S + tile with S the power
    of two >= T."""
    reps = [oracle.replica_full(g, v, tile) for v in views]
    T = reps[0]["range"].shape[0]
    S = 1 << int(np.ceil(np.log2(T))) if T > 1 else 1
    key_tile, value, key_depth = [], [], []
    ranges = np.zeros((len(views) * S, 2), np.uint32)
    base = 0
    for t in range(T):
        for v, r in enumerate(reps):
            a, b = (int(x) for x in r["range"][t])
            if b <= a:
                continue
            lst = r["list"][a:b]
            key_tile.append(np.full(b - a, v * S + t, np.uint32))
            value.append(lst.astype(np.int32))
            key_depth.append(r["depth"].view(np.uint32)[lst])
            ranges[v * S + t] = (base, base + b - a)
            base += b - a
    return reps, {"key_tile": np.concatenate(key_tile), "value": np.concatenate(value),
                  "key_depth": np.concatenate(key_depth), "range": ranges, "M": base}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    g, views, tile = _case(request.param)
    gpu = run_forward(g, views, tile)
    reps, idx = _expected_index(g, views, tile)
    return {"name": request.param, "g": g, "views": views, "tile": tile, "gpu": gpu, "reps": reps, "idx": idx}


def test_project_bit_exact(case):
    gpu, reps, n = case["gpu"], case["reps"], case["g"]["intensity"].shape[0]
    for v, r in enumerate(reps):
        sl = slice(v * n, (v + 1) * n)
        np.testing.assert_array_equal(gpu["count"][sl].view(np.uint32), r["count"])
        np.testing.assert_array_equal(gpu["records"][sl].view(np.uint32), r["rec"].view(np.uint32))
        np.testing.assert_array_equal(gpu["depth"][sl].view(np.uint32), r["depth"].view(np.uint32))
        np.testing.assert_array_equal(gpu["rect"][sl], r["rect"])


def test_bin_sort_bit_exact(case):
    gpu, idx = case["gpu"], case["idx"]
    assert gpu["status"].code == B.XG_OK
    assert gpu["M"] == idx["M"] > 0
    np.testing.assert_array_equal(gpu["key_tile"], idx["key_tile"])
    np.testing.assert_array_equal(gpu["key_depth"], idx["key_depth"])
    np.testing.assert_array_equal(gpu["value"], idx["value"])
    np.testing.assert_array_equal(gpu["range"], idx["range"])


def test_render_fwd_bit_exact_against_replica(case):
    gpu, reps = case["gpu"], case["reps"]
    for v, r in enumerate(reps):
        np.testing.assert_array_equal(gpu["ncontrib"][v].view(np.uint32), r["ncontrib"])
        np.testing.assert_array_equal(gpu["last"][v].view(np.uint32), r["last"])
        np.testing.assert_array_equal(gpu["image"][v].view(np.uint32), r["image"].view(np.uint32))
        np.testing.assert_array_equal(gpu["tfinal"][v].view(np.uint32), r["tfinal"].view(np.uint32))


def test_render_fwd_against_fp64_oracle(case):
    gpu = case["gpu"]
    over, flagged = 0, 0
    for v, view in enumerate(case["views"]):
        ref = oracle.render64(case["g"], view)
        amb = ref["ambiguous"] != 0
        err = np.abs(gpu["image"][v].astype(np.float64) - ref["image"])
        assert err[~amb].max(initial=0.0) <= PIXEL_TOL
        assert err.max() <= AMBIGUOUS_TOL
        assert np.array_equal(gpu["ncontrib"][v][~amb], ref["ncontrib"][~amb])
        over += int((err > PIXEL_TOL).sum())
        flagged += int(amb.sum())
    PIXEL_STATS.append({"what": f"small case {case['name']}", "pixels": gpu["image"].size, "flagged": flagged,
                        "over_tol": over})
    assert over <= OVER_TOL_FRAC_MAX * gpu["image"].size


def _grad_check(gpu, ora, what, mag):
    rec = grad_compare(gpu, ora, mag, what)
    assert rec["bad_widened"] == 0, f"{what}: {rec['bad_widened']} of {rec['checked']} outside tolerance"
    return rec


def _upstream(views, g, gen, pixels=None):
    """+-1 upstream gradient (a sum-L1 loss), zero on pixels whose decisions are ambiguous."""
    Gs = []
    for view in views:
        G = gen.choice([-1.0, 1.0], size=(view.height, view.width))
        amb = oracle.render64(g, view, pixels=pixels)["ambiguous"]
        G[amb != 0] = 0.0
        Gs.append(G)
    return np.stack(Gs)


@pytest.mark.parametrize("name", ["ragged_5views_8x8", "tall_2views_16x32"])
def test_render_bwd_against_fp64_oracle(name):
    g, views, tile = _case(name)
    gen = np.random.default_rng(21)
    G = _upstream(views, g, gen)
    fwd = run_forward(g, views, tile)
    gpu = run_backward(fwd, G)
    ref = None
    n = g["intensity"].shape[0]
    VN = n * len(views)
    recs2d = []
    for v, view in enumerate(views):
        ref = oracle.grad64(g, view, G[v], out=ref)
        g2 = ref["g2d"]
        gpu2 = gpu["g2d"][:, v * n:(v + 1) * n]
        for k, what in enumerate(("u_x", "u_y", "conic_a", "conic_b", "conic_c", "opacity", "intensity")):
            recs2d.append(_grad_check(gpu2[k], g2[k], f"{name} view {v} d/d{what}", ref["mag2d"][k]))
    assert gpu["g2d"].shape == (7, VN)
    recs = [_grad_check(gpu[k], ref[k], f"{name} {k}", ref["mag"][k]) for k in NAMES]
    for tot in (merge_stats(recs2d, f"{name} 2-D gradients"), merge_stats(recs, f"{name} parameter gradients")):
        assert tot["checked"] > 1000
        assert tot["strict_frac"] >= STRICT_FRAC_MIN, tot


def test_autograd_function_matches_abi():
    from paper_2403_04116_gb300.render import FrameConfig, Renderer, render
    g, views, tile = _case("ragged_3views_32x16")
    dev = [t.clone().requires_grad_(True) for t in to_device(g)]
    r = Renderer(views, FrameConfig(*tile))
    img = render(r, *dev)
    G = torch.randn_like(img)
    (img * G).sum().backward()
    fwd = run_forward(g, views, tile)
    np.testing.assert_array_equal(img.detach().cpu().numpy(), fwd["image"])
    ref = run_backward(fwd, G.cpu().numpy())
    for t, k in zip(dev, NAMES):
        # float atomics accumulate in a run-dependent order: equal up to rounding
        got = t.grad.cpu().numpy()
        np.testing.assert_allclose(got, ref[k], rtol=1e-4, atol=1e-5 * np.abs(ref[k]).max())


# ------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------

def _scene(mean, scale, quat, opac, inten):
    n = len(opac)
    return {"mean": np.asarray(mean, np.float32).reshape(3, n), "scale": np.asarray(scale, np.float32).reshape(3, n),
            "quat": np.asarray(quat, np.float32).reshape(4, n), "opacity": np.asarray(opac, np.float32),
            "intensity": np.asarray(inten, np.float32)}


def test_lone_gaussian_peak():
    g = _scene(np.zeros(3), np.full(3, 2.0), [1, 0, 0, 0], [0.37], [0.8])
    view = View(1000.0, 1500.0, 1.0, 1.0, 0.7, 33, 33)
    out = run_forward(g, [view])
    assert out["image"][0, 16, 16] == pytest.approx(0.37 * 0.8, abs=2e-6)
    ref = oracle.render64(g, view)
    assert np.abs(out["image"][0] - ref["image"]).max() <= PIXEL_TOL


def test_everything_culled():
    g = _scene([[2000.0, 1500.0], [0, 0], [0, 0]], np.ones((3, 2)), np.tile([1.0, 0, 0, 0], (2, 1)).T, [0.5, 0.5],
               [1, 1])
    view = View(1000.0, 1500.0, 1.0, 1.0, 0.0, 64, 48)
    out = run_forward(g, [view])
    assert out["M"] == 0 and out["status"].code == B.XG_OK
    assert not out["image"].any() and not out["ncontrib"].any()
    assert np.all(out["tfinal"] == 1.0)
    gr = run_backward(out, np.ones((1, 48, 64)))
    assert all(not gr[k].any() for k in NAMES)


def test_capacity_overflow_is_reported_and_recoverable():
    g, views, tile = _case("ragged_3views_32x16")
    out = run_forward(g, views, tile, capacity=1000)
    assert out["status"].code == B.XG_ERR_CAPACITY
    need = int(out["status"].pairs)
    assert need > 1000
    assert not out["image"].any()
    gr = run_backward(out, np.ones(out["image"].shape))
    assert all(not gr[k].any() for k in NAMES)
    ok = run_forward(g, views, tile, capacity=need)
    assert ok["status"].code == B.XG_OK and ok["M"] == need


def test_nonfinite_gaussians_are_skipped_and_counted():
    g, views, tile = _case("ragged_5views_8x8")
    g = {k: v.copy() for k, v in g.items()}
    g["mean"][1, 17] = np.nan
    g["quat"][2, 99] = np.inf
    g["opacity"][1234] = np.nan
    out = run_forward(g, views, tile)
    assert out["status"].nonfinite == 3
    rep = oracle.replica_full(g, views[2], tile)
    np.testing.assert_array_equal(out["image"][2].view(np.uint32), rep["image"].view(np.uint32))


def test_single_pixel_detector_and_single_gaussian():
    g = _scene([0.1, -0.2, 0.05], [0.5, 0.7, 0.6], [0.9, 0.1, -0.3, 0.2], [0.6], [0.9])
    view = View(1000.0, 1500.0, 1.0, 1.0, 1.0, 1, 1)
    out = run_forward(g, [view], tile=(8, 8))
    ref = oracle.render64(g, view)
    assert abs(out["image"][0, 0, 0] - ref["image"][0, 0]) <= PIXEL_TOL


def test_large_detector_few_gaussians():
    W = H = 2048
    g = synth.gaussians(500, synth.scene_side_mm(W), synth.rng(13, 0), log_scale=(-4.0, -3.0))
    view = synth.circular_views(1, W, H, first_rad=0.3)[0]
    out = run_forward(g, [view], tile=(16, 16))
    assert out["status"].code == B.XG_OK and out["M"] > 65536
    rep = oracle.replica_full(g, view, (16, 16))
    np.testing.assert_array_equal(out["ncontrib"][0].view(np.uint32), rep["ncontrib"])
    np.testing.assert_array_equal(out["image"][0].view(np.uint32), rep["image"].view(np.uint32))


def test_views_in_one_frame_equal_separate_frames():
    g, views, tile = _case("ragged_5views_8x8")
    together = run_forward(g, views, tile)
    for v, view in enumerate(views):
        alone = run_forward(g, [view], tile)
        np.testing.assert_array_equal(together["image"][v], alone["image"][0])
        np.testing.assert_array_equal(together["last"][v], alone["last"][0])


def test_tile_shape_batch_and_pixels_per_thread_do_not_change_the_image():
    g, views, _ = _case("ragged_3views_32x16")
    base = run_forward(g, views, (16, 16))
    for tile, batch, ppt in [((8, 8), 64, 1), ((32, 16), 128, 1), ((8, 32), 256, 2), ((32, 8), 64, 2),
                             ((16, 16), 128, 1), ((32, 32), 256, 2), ((16, 16), 64, 4), ((32, 32), 128, 4),
                             ((8, 16), 256, 4)]:
        other = run_forward(g, views, tile, batch=batch, ppt=ppt)
        np.testing.assert_array_equal(other["image"], base["image"])
        np.testing.assert_array_equal(other["ncontrib"], base["ncontrib"])
        np.testing.assert_array_equal(other["tfinal"], base["tfinal"])


@pytest.mark.parametrize("ppt", [1, 2, 4])
def test_backward_pixels_per_thread_variants_agree(ppt):
    g, views, tile = _case("tall_2views_16x32")
    G = np.random.default_rng(5).choice([-1.0, 1.0], size=(len(views), views[0].height, views[0].width))
    a = run_backward(run_forward(g, views, tile, batch=64, ppt=ppt), G)
    b = run_backward(run_forward(g, views, (16, 16), batch=256, ppt=1 if ppt != 1 else 2), G)
    for k in NAMES:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-4, atol=1e-5 * np.abs(b[k]).max())
