"""Pins of the oracle outputs that set the GPU tests' tolerances.

The FP64 oracle returns, beside the image and the gradients, two things that decide how
strictly the CUDA path is judged:

* the ambiguity flags of each pixel: bit 1 when some Gaussian's opacity sits within 1e-4
  (relative) of the 1/255 inclusion threshold, bit 2 when the transmittance after a
  Gaussian sits within 1e-3 of the 1e-4 stop, bit 4 when two consecutive contributors lie
  within 2^-22 (relative) in depth (Eq. 10 and the thresholds of the blending it follows);
* the term magnitudes: ``mag2d``, per Gaussian and per 2-D quantity, the sum over pixels of
  |each pixel's term|, and ``mag``, the same magnitudes carried to the parameters through
  the absolute value of the linear backward map of Eq. 7-9.

A mistake in either (a flag that never fires, a margin far too wide, a magnitude that
double counts) would loosen every GPU test without failing any, so they are pinned here
against facts that do not come from the oracle: hand-built scenes whose decisions sit at
a chosen distance from each threshold, the triangle inequality, the sign-definite
intensity term, the decomposition of a sum over pixels into single-pixel calls, and a
finite-difference Jacobian of the projection.
"""
import numpy as np
import pytest

import oracle
from paper_2403_04116_gb300 import synth
from paper_2403_04116_gb300.synth import View

# odd detector: the principal point (W/2, H/2) is the centre of pixel (16, 16), and every
# point on the central ray (the x axis at angle 0) projects exactly there
W = H = 33
CENTRE = 16 * W + 16


def _view(angle=0.0):
    return View(1000.0, 1500.0, 1.0, 1.0, angle, W, H)


def _scene(xs, opac, inten=None, scale=2.0):
    """Isotropic Gaussians on the central ray at x = xs (depth t_z = 1000 - x)."""
    n = len(xs)
    mean = np.zeros((3, n))
    mean[0] = xs
    quat = np.zeros((4, n))
    quat[0] = 1.0
    return {"mean": mean, "scale": np.full((3, n), scale), "quat": quat, "opacity": np.asarray(opac, float),
            "intensity": np.asarray(inten if inten is not None else [0.5] * n, float)}


def _flags(g):
    return int(oracle.render64(g, _view())["ambiguous"].reshape(-1)[CENTRE])


# ------------------------------------------------------------------------------------------
# ambiguity flags
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("rel,flagged", [(1e-6, True), (-1e-6, True), (5e-5, True), (1e-2, False),
                                         (-1e-2, False), (3e-4, False)])
def test_alpha_threshold_flag(oracle_lib, rel, flagged):
    """A lone Gaussian seen at its centre has opacity o exactly there; o = (1 + rel)/255 is
    flagged (bit 1) within the 1e-4 relative margin of the 1/255 threshold, not outside."""
    f = _flags(_scene([0.0], [(1.0 + rel) / 255.0]))
    assert bool(f & 1) == flagged, f
    assert f & ~1 == 0


@pytest.mark.parametrize("rel,flagged", [(1e-6, True), (-1e-6, True), (5e-4, True), (1e-2, False),
                                         (-1e-2, False), (3e-3, False)])
def test_transmittance_stop_flag(oracle_lib, rel, flagged):
    """A front Gaussian clamped at 0.99 and a second of opacity 0.5 leave T = 0.005; a
    third of opacity 0.98 - 0.02 rel behind them leaves 1e-4 (1 + rel), flagged (bit 2)
    within the 1e-3 margin of the stop.  Whether the third one is blended follows the
    sign of rel."""
    g = _scene([20.0, 10.0, 0.0], [0.995, 0.5, 0.98 - 0.02 * rel])
    f = _flags(g)
    assert bool(f & 2) == flagged, f
    assert f & ~2 == 0
    r = oracle.render64(g, _view())
    assert int(r["ncontrib"].reshape(-1)[CENTRE]) == (3 if rel > 0 else 2)
    want_t = 0.005 * (1e-4 * (1 + rel) / 0.005 if rel > 0 else 1.0)
    assert abs(r["tfinal"].reshape(-1)[CENTRE] / want_t - 1.0) < 1e-12


@pytest.mark.parametrize("rel,flagged", [(1e-7, True), (2e-7, True), (1e-6, False), (1e-2, False)])
def test_depth_tie_flag(oracle_lib, rel, flagged):
    """Two contributors on the same ray whose depths differ by rel (relative) are flagged
    (bit 4) within 2^-22 = 2.4e-7, where FP32 depth keys may tie or swap."""
    x2 = 1000.0 - 1000.0 * (1.0 + rel)  # t_z = 1000 (1 + rel), behind the first
    f = _flags(_scene([0.0, x2], [0.3, 0.3]))
    assert bool(f & 4) == flagged, f
    assert f & ~4 == 0


def test_unambiguous_scene_has_no_flags(oracle_lib):
    f = _flags(_scene([20.0, 0.0, -20.0], [0.3, 0.4, 0.5]))
    assert f == 0


# ------------------------------------------------------------------------------------------
# term magnitudes
# ------------------------------------------------------------------------------------------

def _random_case(seed, n=60, Wd=40):
    g = synth.gaussians(n, synth.scene_side_mm(Wd), synth.rng(90 + seed, 0), log_scale=(-3.0, -2.0))
    g = {k: v.astype(np.float64) for k, v in g.items()}
    views = synth.circular_views(2, Wd, Wd, first_rad=0.4 + seed)
    return g, views


@pytest.mark.parametrize("seed", [0, 1])
def test_magnitudes_bound_the_sums(oracle_lib, seed):
    """|sum of terms| <= sum of |terms|: mag2d >= |g2d| for every 2-D quantity and mag >=
    |gradient| for every parameter (accumulated over views)."""
    g, views = _random_case(seed)
    gen = np.random.default_rng(seed)
    out = None
    for v in views:
        G = gen.choice([-1.0, 1.0], size=(v.height, v.width))
        out = oracle.grad64(g, v, G, out=out)
        assert (out["mag2d"] >= np.abs(out["g2d"]) * (1 - 1e-12)).all()
        assert (out["mag2d"] > 0).sum() > 20  # the scene is not empty
    for k in ("mean", "scale", "quat", "opacity", "intensity"):
        assert (out["mag"][k] >= np.abs(out[k]) * (1 - 1e-12)).all(), k


def test_intensity_magnitude_equals_sum_for_nonnegative_upstream(oracle_lib):
    """With G >= 0 every intensity term G alpha T is >= 0, so its magnitude equals its sum,
    for the 2-D quantity and for the parameter."""
    g, views = _random_case(2)
    gen = np.random.default_rng(5)
    G = gen.uniform(0.0, 1.0, size=(views[0].height, views[0].width))
    out = oracle.grad64(g, views[0], G)
    np.testing.assert_array_equal(out["mag2d"][6], out["g2d"][6])
    np.testing.assert_allclose(out["mag"]["intensity"], out["intensity"], rtol=1e-14, atol=0)
    # and with G <= 0 the magnitude is minus the sum
    out = oracle.grad64(g, views[0], -G)
    np.testing.assert_array_equal(out["mag2d"][6], -out["g2d"][6])


def test_magnitudes_decompose_over_pixels(oracle_lib):
    """mag2d over a set of pixels equals the sum over single-pixel calls of |g2d|: a pixel
    holds one term per Gaussian, so for one pixel the magnitude is the absolute value of
    the sum.  A double-counted or dropped pixel breaks the equality."""
    g, views = _random_case(3)
    v = views[1]
    gen = np.random.default_rng(6)
    G = gen.choice([-1.0, 1.0], size=(v.height, v.width))
    pix = np.sort(gen.choice(v.width * v.height, size=150, replace=False)).astype(np.int32)
    whole = oracle.grad64(g, v, G, pixels=pix)
    acc = np.zeros_like(whole["mag2d"])
    for p in pix:
        one = oracle.grad64(g, v, G, pixels=np.array([p], np.int32))
        np.testing.assert_array_equal(one["mag2d"], np.abs(one["g2d"]))
        acc += np.abs(one["g2d"])
    assert (whole["mag2d"] > 0).sum() > 20
    np.testing.assert_allclose(whole["mag2d"], acc, rtol=1e-12, atol=1e-300)


def _projection_jacobian(g, k, view):
    """d(u_x, u_y, a, b, c, opacity, intensity)/d(mean, scale, quat, opacity, intensity) of
    Gaussian k by central differences of the oracle's projection (7 x 12)."""
    params = [("mean", r) for r in range(3)] + [("scale", r) for r in range(3)] + [("quat", r) for r in range(4)]
    J = np.zeros((7, 12))
    for col, (key, r) in enumerate(params):
        h = 1e-5 * max(1.0, abs(g[key][r, k]))
        vals = []
        for s in (1.0, -1.0):
            gp = {kk: vv.copy() for kk, vv in g.items()}
            gp[key][r, k] += s * h
            pr = oracle.project64(gp, view)[k]
            vals.append(np.array([pr[4], pr[5], pr[9], pr[10], pr[11]]))
        J[:5, col] = (vals[0] - vals[1]) / (2 * h)
    J[5, 10] = 1.0  # opacity and intensity reach the blending unchanged
    J[6, 11] = 1.0
    return J


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_pixel_magnitude_by_hand(oracle_lib, seed):
    """One Gaussian, one pixel: each 2-D gradient is a single term t_q, so mag2d = |t_q|,
    and the parameter magnitude is sum_q |dq/dtheta| |t_q| with the Jacobian dq/dtheta of
    the projection taken by central differences (independent of the oracle's chain rule);
    the gradient itself is sum_q dq/dtheta t_q."""
    gen = np.random.default_rng(40 + seed)
    v = View(1000.0, 1500.0, 1.0, 1.0, gen.uniform(0, 2 * np.pi), W, H)
    side = synth.scene_side_mm(W)
    q = gen.normal(size=4)
    g = {"mean": gen.uniform(-0.2, 0.2, size=(3, 1)) * side, "scale": np.exp(gen.uniform(-2.5, -1.5, size=(3, 1))) * side,
         "quat": (q / np.linalg.norm(q) * gen.uniform(0.7, 1.4)).reshape(4, 1), "opacity": np.array([0.4]),
         "intensity": np.array([0.7])}
    pr = oracle.project64(g, v)[0]
    x, y = int(pr[4]), int(pr[5])  # the pixel holding the projected centre, off its centre
    pix = np.array([y * W + x], np.int32)
    G = np.zeros((H, W))
    G[y, x] = -1.0
    out = oracle.grad64(g, v, G, pixels=pix)
    t = out["g2d"][:, 0]
    assert np.count_nonzero(t) == 7
    np.testing.assert_array_equal(out["mag2d"][:, 0], np.abs(t))
    J = _projection_jacobian(g, 0, v)
    want_mag = np.abs(J).T @ np.abs(t)
    want_grad = J.T @ t
    got_mag = np.concatenate([out["mag"][k].reshape(-1) for k in ("mean", "scale", "quat", "opacity", "intensity")])
    got_grad = np.concatenate([out[k].reshape(-1) for k in ("mean", "scale", "quat", "opacity", "intensity")])
    scale = np.abs(want_mag).max()
    np.testing.assert_allclose(got_mag, want_mag, rtol=1e-5, atol=1e-7 * scale)
    np.testing.assert_allclose(got_grad, want_grad, rtol=1e-5, atol=1e-7 * scale)


@pytest.mark.parametrize("rel,flagged", [(1e-8, True), (1e-7, True), (1e-5, False), (1e-2, False)])
def test_depth_tie_with_the_candidate_after_the_stop(oracle_lib, rel, flagged):
    """Three Gaussians take T to 1.5e-4, a fourth (opacity 0.5) would take it below 1e-4 and
    stops the blend; a fifth lies behind the fourth by rel in depth.  Within 2^-22 of the
    stopper's depth a float32 depth order may put the fifth first (and blend it instead), so
    the pixel is flagged; farther behind it is not."""
    x_stop = -10.0
    x_next = 1000.0 - (1000.0 - x_stop) * (1.0 + rel)
    g = _scene([20.0, 10.0, x_stop, x_next], [0.995, 0.985, 0.5, 0.2])
    f = _flags(g)
    assert bool(f & 4) == flagged, f
    assert f & ~4 == 0
    assert int(oracle.render64(g, _view())["ncontrib"].reshape(-1)[CENTRE]) == 2


def test_flags_cover_every_decision_the_fp32_replica_takes_differently(oracle_lib):
    """On a full view of the 50,000-Gaussian training scene (256 x 256), the FP32 replica of
    the kernels' decision sequence and the FP64 oracle blend the same number of Gaussians at
    every pixel the oracle does not flag."""
    g = synth.gaussians(50_000, synth.scene_side_mm(256), synth.rng(1, 0))
    view = synth.circular_views(50, 256, 256)[0]
    rep = oracle.replica_full(g, view, (16, 16))
    ref = oracle.render64(g, view)
    amb = ref["ambiguous"] != 0
    assert 0 < amb.mean() < 0.2
    np.testing.assert_array_equal(rep["ncontrib"].astype(np.int64)[~amb], ref["ncontrib"][~amb])
