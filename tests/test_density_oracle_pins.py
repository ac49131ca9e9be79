"""Pins of the adaptive-density-control oracle (oracle/density64.py) against facts outside
it: SciPy's quaternion rotation, hand-built cases for every rule, the sample covariance of
split centres, closed-form statistics."""
import numpy as np
import pytest

from oracle import density64 as D


def _params(n, nf=3, seed=0):
    gen = np.random.default_rng(seed)
    q = gen.normal(size=(4, n))
    return {"mean": gen.normal(size=(3, n)).astype(np.float32), "log_scale": gen.uniform(-3, 0, size=(3, n)).astype(np.float32),
            "quat": q.astype(np.float32), "opacity_logit": gen.normal(size=n).astype(np.float32),
            "features": gen.normal(size=(nf, n)).astype(np.float32)}


def test_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    q = np.random.default_rng(1).normal(size=(4, 50))
    R = D.quat_to_rot64(q)
    want = Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], axis=1)).as_matrix()
    np.testing.assert_allclose(R, want, atol=1e-12)


def test_statistics_closed_form():
    g = np.zeros((3, 2, 2))
    g[0, 0] = (3, 4)      # norm 5
    g[1, 0] = (0, 1)      # norm 1
    g[2, 0] = (6, 8)      # norm 10, but not visible
    g[0, 1] = (1, 1)
    vis = np.array([[True, False], [True, False], [False, False]])
    acc, den = D.densify_stats64(g, vis, scale=2.0)
    np.testing.assert_allclose(acc, [12.0, 0.0])
    np.testing.assert_array_equal(den, [2, 0])


def test_every_rule_by_hand():
    p = _params(7)
    p["log_scale"][:] = -2.0
    p["opacity_logit"][:] = 0.0
    acc = np.array([0.1, 5.0, 5.0, 5.0, 5.0, 0.1, 0.0], np.float32)
    den = np.array([1, 1, 1, 1, 1, 1, 0])
    p["log_scale"][1, 2] = -0.5          # 2: large, high gradient -> split
    p["opacity_logit"][3] = -9.0         # 3: transparent -> pruned (though its gradient is high)
    p["log_scale"][0, 5] = 3.0           # 5: too large in the world -> pruned
    out = D.densify64(p, acc, den, np.zeros((2, 3, 7)), grad_thresh=1.0, size_log_thresh=-1.0,
                      prune_logit=-5.0, max_log_size=2.0)
    # 0 kept; 1 kept + clone; 2 -> two children; 3 pruned; 4 kept + clone; 5 pruned; 6 kept (never seen)
    np.testing.assert_array_equal(out["src"], [0, 1, 1, 2, 2, 4, 4, 6])
    np.testing.assert_array_equal(out["kind"], [0, 0, 1, 2, 2, 0, 1, 0])
    # a child: scales divided by 1.6, centre = parent's with zero noise, the rest copied
    np.testing.assert_allclose(out["log_scale"][:, 3], p["log_scale"][:, 2] - np.log(1.6), rtol=1e-12)
    np.testing.assert_allclose(out["mean"][:, 3], p["mean"][:, 2], rtol=1e-7)
    np.testing.assert_array_equal(out["quat"][:, 3], p["quat"][:, 2])
    np.testing.assert_array_equal(out["features"][:, 4], p["features"][:, 2])
    # the threshold is inclusive: accum / denom == grad_thresh densifies
    out = D.densify64(p, np.full(7, 2.0, np.float32), np.full(7, 2), np.zeros((2, 3, 7)), 1.0, 5.0, -50.0)
    assert (out["kind"] == 1).sum() == 7


def test_children_sample_the_gaussian():
    n = 20000
    p = _params(1, seed=2)
    p = {k: np.repeat(v, n, axis=-1) for k, v in p.items()}
    z = np.random.default_rng(3).normal(size=(2, 3, n))
    out = D.densify64(p, np.ones(n, np.float32), np.ones(n), z, 0.5, -10.0, -50.0)
    assert out["mean"].shape == (3, 2 * n)
    R = D.quat_to_rot64(p["quat"][:, :1])[0]
    S = np.diag(np.exp(p["log_scale"][:, 0].astype(np.float64)))
    cov = R @ S @ S @ R.T
    d = out["mean"] - p["mean"][:, :1].astype(np.float64)
    np.testing.assert_allclose(d.mean(axis=1), 0.0, atol=0.03 * np.sqrt(np.diag(cov)).max())
    np.testing.assert_allclose(np.cov(d), cov, atol=0.05 * np.abs(cov).max())


def test_opacity_reset():
    lo = np.array([-8.0, -4.0, 0.0, 3.0], np.float32)
    np.testing.assert_array_equal(D.opacity_reset64(lo, -4.59512), np.float32([-8.0, -4.59512, -4.59512, -4.59512]))
