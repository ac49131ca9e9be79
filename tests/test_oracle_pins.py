"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* geometry: the projection equals a ray/detector-plane intersection of the cone-beam
  scanner (Sec. 3.3); the EWA covariance equals J_num Sigma J_num^T for the numerical
  Jacobian of that exact map, with Sigma built from SciPy's quaternion rotation;
* closed forms: a lone isotropic Gaussian's image, two Gaussians on the central ray
  (front-to-back order of Eq. 10), a stack that hits the transmittance stop;
* invariants: with unit intensities I = 1 - T; T in [1e-4, 1]; the image is unchanged
  when the scene and the scanner rotate together, or when the Gaussians are permuted;
* gradients: central finite differences of the oracle's own forward pass; the sum of
  intensity gradients equals 1 - T; quaternion gradients are orthogonal to q.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2403_04116_gb300 import synth
from paper_2403_04116_gb300.synth import View


def _view(angle=0.0, W=33, H=33, sod=1000.0, sdd=1500.0, pu=1.0, pv=1.0):
    return View(sod, sdd, pu, pv, angle, W, H)


def _scene(mean, scale, quat, opac, inten):
    n = len(opac)
    return {"mean": np.asarray(mean, float).reshape(3, n), "scale": np.asarray(scale, float).reshape(3, n),
            "quat": np.asarray(quat, float).reshape(4, n), "opacity": np.asarray(opac, float),
            "intensity": np.asarray(inten, float)}


def _ray_plane_projection(mu, v: View):
    """Where the ray from the source through mu meets the detector, in detector pixels."""
    a = v.angle_rad
    src = v.sod_mm * np.array([math.cos(a), math.sin(a), 0.0])
    nrm = -np.array([math.cos(a), math.sin(a), 0.0])  # detector normal, towards the detector
    e_u = np.array([-math.sin(a), math.cos(a), 0.0])
    e_v = np.array([0.0, 0.0, -1.0])
    det_c = src + v.sdd_mm * nrm
    d = mu - src
    X = src + d * (v.sdd_mm / (d @ nrm))
    return np.array([v.width / 2 + (X - det_c) @ e_u / v.pitch_u_mm,
                     v.height / 2 + (X - det_c) @ e_v / v.pitch_v_mm])


def _random_scene(n, side, gen, log_scale=(-3.0, -2.0), opac=(0.05, 0.5)):
    g = synth.gaussians(n, side, gen, log_scale=log_scale, opacity=opac)
    return {k: v.astype(np.float64) for k, v in g.items()}


# ------------------------------------------------------------------------------------------
# geometry
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("angle", [0.0, 0.3, 1.7, 3.9, -2.2])
def test_mean_projection_is_ray_detector_intersection(oracle_lib, angle):
    gen = np.random.default_rng(1)
    v = _view(angle, W=64, H=48, pu=0.8, pv=1.3)
    n = 50
    mu = gen.uniform(-30, 30, size=(3, n))
    g = _scene(mu, np.ones((3, n)), np.tile([1.0, 0, 0, 0], (n, 1)).T, np.full(n, 0.5), np.ones(n))
    pr = oracle.project64(g, v)
    for k in range(n):
        np.testing.assert_allclose(pr[k, 4:6], _ray_plane_projection(mu[:, k], v), rtol=0, atol=1e-9)
        src = v.sod_mm * np.array([math.cos(angle), math.sin(angle), 0.0])
        # t_z is the depth of mu along the source's viewing direction
        np.testing.assert_allclose(pr[k, 3], (mu[:, k] - src) @ -src / v.sod_mm, atol=1e-9)


def test_isocentre_projects_to_principal_point(oracle_lib):
    for a in np.linspace(-3, 3, 7):
        v = _view(a, W=40, H=30)
        g = _scene(np.zeros(3), np.ones(3), [1, 0, 0, 0], [0.5], [1.0])
        pr = oracle.project64(g, v)
        np.testing.assert_allclose(pr[0, 4:6], [20.0, 15.0], atol=1e-12)
        assert pr[0, 3] == pytest.approx(1000.0)


@pytest.mark.parametrize("angle", [0.0, 0.9, 2.5, -1.2])
def test_ewa_covariance_matches_numerical_jacobian(oracle_lib, angle):
    gen = np.random.default_rng(7)
    v = _view(angle, W=64, H=64, pu=0.9, pv=1.1)
    n = 20
    mu = gen.uniform(-20, 20, size=(3, n))
    s = gen.uniform(0.3, 3.0, size=(3, n))
    q = gen.normal(size=(4, n)) * gen.uniform(0.5, 2.0, size=n)  # unnormalised on purpose
    g = _scene(mu, s, q, np.full(n, 0.5), np.ones(n))
    pr = oracle.project64(g, v)
    h = 1e-4
    for k in range(n):
        Jn = np.zeros((2, 3))
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            Jn[:, c] = (_ray_plane_projection(mu[:, k] + e, v) - _ray_plane_projection(mu[:, k] - e, v)) / (2 * h)
        R = Rotation.from_quat([q[1, k], q[2, k], q[3, k], q[0, k]]).as_matrix()  # SciPy is scalar-last
        Sigma = R @ np.diag(s[:, k] ** 2) @ R.T
        S2 = Jn @ Sigma @ Jn.T + 0.3 * np.eye(2)
        got = np.array([[pr[k, 6], pr[k, 7]], [pr[k, 7], pr[k, 8]]])
        np.testing.assert_allclose(got, S2, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(np.array([[pr[k, 9], pr[k, 10]], [pr[k, 10], pr[k, 11]]]) @ got, np.eye(2),
                                   atol=1e-10)


# ------------------------------------------------------------------------------------------
# closed forms of the blend
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("angle", [0.0, 1.1, 4.0])
def test_lone_isotropic_gaussian_closed_form(oracle_lib, angle):
    v = _view(angle, W=33, H=33)
    s, o, i = 2.0, 0.37, 0.8
    q = Rotation.random(random_state=3).as_quat()
    g = _scene(np.zeros(3), np.full(3, s), [q[3], q[0], q[1], q[2]], [o], [i])
    r = oracle.render64(g, v)
    var = (1500.0 * s / 1000.0) ** 2 + 0.3
    yy, xx = np.mgrid[0:33, 0:33]
    d2 = (xx + 0.5 - 16.5) ** 2 + (yy + 0.5 - 16.5) ** 2
    a = o * np.exp(-0.5 * d2 / var)
    expect = np.where(a >= 1 / 255, i * a, 0.0)
    np.testing.assert_allclose(r["image"], expect, rtol=1e-12, atol=1e-15)
    assert r["image"][16, 16] == pytest.approx(o * i, rel=1e-15)
    np.testing.assert_array_equal(r["ncontrib"], (a >= 1 / 255).astype(np.int32))
    np.testing.assert_allclose(r["tfinal"], np.where(a >= 1 / 255, 1 - a, 1.0), rtol=1e-12)


def test_alpha_threshold_boundary(oracle_lib):
    v = _view(0.0, W=33, H=33)
    s = 2.0
    var = (1.5 * s) ** 2 + 0.3
    d2 = 3.0 ** 2  # pixel (19, 16) is 3 px from the centre pixel's centre
    for factor, inside in [(1.001, 1), (0.999, 0)]:
        o = factor / 255.0 / math.exp(-0.5 * d2 / var)
        g = _scene(np.zeros(3), np.full(3, s), [1, 0, 0, 0], [o], [1.0])
        r = oracle.render64(g, v)
        assert r["ncontrib"][16, 19] == inside


def test_two_gaussians_on_central_ray_blend_front_to_back(oracle_lib):
    v = _view(0.0)
    # source on +x: x = +5 is nearer to it than x = -5; index order is the reverse
    far, near = (-5.0, 0.6, 0.3), (5.0, 0.25, 0.9)
    g = _scene([[far[0], near[0]], [0, 0], [0, 0]], np.full((3, 2), 1.5), np.tile([1.0, 0, 0, 0], (2, 1)).T,
               [far[1], near[1]], [far[2], near[2]])
    r = oracle.render64(g, v)
    expect = near[1] * near[2] + (1 - near[1]) * far[1] * far[2]
    assert r["image"][16, 16] == pytest.approx(expect, rel=1e-14)
    assert r["tfinal"][16, 16] == pytest.approx((1 - near[1]) * (1 - far[1]), rel=1e-14)


def test_transmittance_stop(oracle_lib):
    v = _view(0.0)
    K = 20
    xs = np.linspace(-10, 10, K)
    g = _scene([xs, np.zeros(K), np.zeros(K)], np.full((3, K), 1.0), np.tile([1.0, 0, 0, 0], (K, 1)).T,
               np.full(K, 0.5), np.ones(K))
    r = oracle.render64(g, v)
    # 0.5^13 = 1.2e-4 stays above the 1e-4 floor, the 14th Gaussian would take T to 6.1e-5
    assert r["ncontrib"][16, 16] == 13
    assert r["tfinal"][16, 16] == pytest.approx(0.5 ** 13, rel=1e-14)
    assert r["image"][16, 16] == pytest.approx(1 - 0.5 ** 13, rel=1e-14)


# ------------------------------------------------------------------------------------------
# invariants on random scenes
# ------------------------------------------------------------------------------------------

def test_unit_intensity_image_is_one_minus_transmittance(oracle_lib):
    gen = synth.rng(90, 0)
    v = _view(0.4, W=48, H=40)
    g = _random_scene(400, synth.scene_side_mm(48), gen, opac=(0.05, 0.9))
    g["intensity"][:] = 1.0
    r = oracle.render64(g, v)
    np.testing.assert_allclose(r["image"], 1 - r["tfinal"], atol=1e-13)
    assert np.all(r["tfinal"] >= 1e-4) and np.all(r["tfinal"] <= 1.0)
    assert r["ncontrib"].max() > 13  # the stop rule was exercised


def test_image_bounds_and_nonincreasing_transmittance(oracle_lib):
    gen = synth.rng(91, 0)
    v = _view(2.0, W=40, H=40)
    g = _random_scene(300, synth.scene_side_mm(40), gen, opac=(0.05, 0.95))
    r = oracle.render64(g, v)
    assert np.all(r["image"] >= 0) and np.all(r["image"] <= g["intensity"].max() + 1e-15)
    # adding Gaussians can only lower the transmittance of a pixel that did not stop early
    g2 = {k: np.concatenate([g[k], g[k][..., :50]], axis=-1) for k in g}
    g2["mean"][:, -50:] += 0.01
    r2 = oracle.render64(g2, v)
    ok = (r["ncontrib"] < 12) & (r2["ncontrib"] < 12)
    assert np.all(r2["tfinal"][ok] <= r["tfinal"][ok] + 1e-15)


def test_rotating_scene_and_scanner_together(oracle_lib):
    gen = synth.rng(92, 0)
    g = _random_scene(200, synth.scene_side_mm(40), gen)
    beta = 0.7
    Rz = Rotation.from_euler("z", beta)
    g_rot = {k: v.copy() for k, v in g.items()}
    g_rot["mean"] = Rz.as_matrix() @ g["mean"]
    q = Rotation.from_quat(np.stack([g["quat"][1], g["quat"][2], g["quat"][3], g["quat"][0]], 1))
    qr = (Rz * q).as_quat()
    g_rot["quat"] = np.stack([qr[:, 3], qr[:, 0], qr[:, 1], qr[:, 2]])
    r0 = oracle.render64(g, _view(0.3, W=40, H=40))
    r1 = oracle.render64(g_rot, _view(0.3 + beta, W=40, H=40))
    np.testing.assert_allclose(r1["image"], r0["image"], atol=1e-10)
    np.testing.assert_array_equal(r1["ncontrib"], r0["ncontrib"])


def test_permuting_gaussians_leaves_image(oracle_lib):
    gen = synth.rng(93, 0)
    g = _random_scene(300, synth.scene_side_mm(40), gen)
    perm = gen.permutation(300)
    gp = {k: v[..., perm] for k, v in g.items()}
    v = _view(1.3, W=40, H=40)
    np.testing.assert_array_equal(oracle.render64(gp, v)["image"], oracle.render64(g, v)["image"])


def test_pixel_subset_matches_full_render(oracle_lib):
    gen = synth.rng(94, 0)
    g = _random_scene(300, synth.scene_side_mm(40), gen)
    v = _view(0.5, W=40, H=40)
    full = oracle.render64(g, v)
    pix = np.array([0, 17, 820, 821, 1599])
    sub = oracle.render64(g, v, pixels=pix)
    np.testing.assert_array_equal(sub["image"].reshape(-1)[pix], full["image"].reshape(-1)[pix])


# ------------------------------------------------------------------------------------------
# gradients
# ------------------------------------------------------------------------------------------

def _loss(g, v, G):
    r = oracle.render64(g, v)
    return float((r["image"] * G).sum()), r["ncontrib"]


def test_gradients_match_central_differences(oracle_lib):
    gen = np.random.default_rng(11)
    W = H = 32
    side = synth.scene_side_mm(W)
    n = 6
    g = {"mean": gen.uniform(-0.25, 0.25, (3, n)) * side, "scale": gen.uniform(0.08, 0.2, (3, n)) * side,
         "quat": gen.normal(size=(4, n)), "opacity": gen.uniform(0.3, 0.8, n),
         "intensity": gen.uniform(0.2, 1.0, n)}
    v = _view(0.8, W=W, H=H)
    G = gen.normal(size=(H, W))
    an = oracle.grad64(g, v, G)
    eps = 1e-4
    checked = 0
    for key, rows in (("mean", 3), ("scale", 3), ("quat", 4), ("opacity", 1), ("intensity", 1)):
        for k in range(n):
            for r in range(rows):
                idx = (r, k) if rows > 1 else (k,)
                gp = {kk: vv.copy() for kk, vv in g.items()}
                gm = {kk: vv.copy() for kk, vv in g.items()}
                gp[key][idx] += eps
                gm[key][idx] -= eps
                lp, np_ = _loss(gp, v, G)
                lm, nm = _loss(gm, v, G)
                if not np.array_equal(np_, nm):
                    continue  # a blending decision flipped inside the stencil
                fd = (lp - lm) / (2 * eps)
                assert an[key][idx] == pytest.approx(fd, rel=2e-5, abs=1e-7), (key, idx)
                checked += 1
    assert checked >= 60


def test_intensity_gradients_sum_to_one_minus_transmittance(oracle_lib):
    gen = synth.rng(95, 0)
    g = _random_scene(300, synth.scene_side_mm(40), gen)
    v = _view(0.2, W=40, H=40)
    r = oracle.render64(g, v)
    an = oracle.grad64(g, v, np.ones((40, 40)))
    assert an["intensity"].sum() == pytest.approx((1 - r["tfinal"]).sum(), rel=1e-12)


def test_quaternion_gradient_orthogonal_to_q(oracle_lib):
    gen = synth.rng(96, 0)
    g = _random_scene(200, synth.scene_side_mm(40), gen)
    g["quat"] *= gen.uniform(0.5, 2.0, size=200)
    v = _view(1.0, W=40, H=40)
    an = oracle.grad64(g, v, gen.normal(size=(40, 40)))
    dots = (an["quat"] * g["quat"]).sum(0)
    scale = np.abs(an["quat"]).sum(0) * np.abs(g["quat"]).sum(0) + 1e-300
    assert np.all(np.abs(dots) <= 1e-12 * scale)


def test_phantom_sphere_chord(oracle_lib):
    # synth's ray integrals: a unit-density sphere at the isocentre, central ray chord = 2 R
    ph = {"centre": np.zeros((1, 3)), "axes": np.full((1, 3), 10.0), "rot": np.eye(3)[None], "density": [1.0]}
    v = _view(0.6)
    img = synth.phantom_line_integrals(ph, v)
    assert img[16, 16] == pytest.approx(20.0, rel=1e-9)
    # off-centre pixel: chord 2 sqrt(R^2 - r_perp^2), r_perp the ray's distance to the centre
    src, d = synth.detector_rays(v)
    r_perp = np.linalg.norm(np.cross(-src, d[16, 20]))
    assert img[16, 20] == pytest.approx(2 * math.sqrt(100 - r_perp ** 2), rel=1e-9)
