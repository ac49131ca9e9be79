"""Pins of the FDK oracle (oracle/fdk64.py): the ramp kernel's closed form and zero DC
response, and reconstructions of exactly projected spheres (density, position, and the
empty surroundings), which fix the weights, the filter scale, the back-projection factor
and the orientation of the geometry."""
import math

import numpy as np
import pytest

from oracle import fdk64 as F
from paper_2403_04116_gb300 import synth


def test_ramp_kernel_closed_form():
    tau = 0.7
    h = F.ramp_kernel64(2048, tau)
    c = 2047
    assert h[c] == pytest.approx(1 / (4 * tau * tau))
    assert h[c + 1] == h[c - 1] == pytest.approx(-1 / (math.pi ** 2 * tau * tau))
    assert h[c + 2] == 0.0 and h[c + 3] == pytest.approx(-1 / (9 * math.pi ** 2 * tau * tau))
    # sum_n h = 1/(4 tau^2) - (2 / (pi^2 tau^2)) sum_odd 1/n^2 = 0 (sum_odd 1/n^2 = pi^2 / 8)
    assert abs(h.sum()) < 1e-3 / (tau * tau)


def _scan(W, V):
    return synth.circular_views(V, W, W)


@pytest.mark.parametrize("centre", [(0.0, 0.0, 0.0), (0.15, -0.1, 0.05)])
def test_sphere_reconstruction(centre):
    W, V, n = 64, 120, 40
    side = synth.scene_side_mm(W)
    vox = side / n
    c = np.asarray(centre) * side
    R = 0.3 * side
    ph = synth.sphere_phantom(c, R, density=1.0)
    views = _scan(W, V)
    proj = np.stack([synth.phantom_line_integrals(ph, v) for v in views])
    vol = F.fdk64(proj, views, (n, n, n), vox)
    Z, Y, X = F.voxel_centres((n, n, n), vox)
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    inside, outside = r < 0.7 * R, (r > 1.3 * R) & (np.abs(Z) < 0.4 * side)
    assert vol[inside].mean() == pytest.approx(1.0, abs=0.03)
    assert np.abs(vol[inside] - 1.0).max() < 0.15
    assert np.abs(vol[outside]).mean() < 0.02
    # the reconstruction sits where the sphere is: centre of mass within half a voxel
    w = np.clip(vol, 0, None) * (r < 1.5 * R)
    com = np.array([(w * X).sum(), (w * Y).sum(), (w * Z).sum()]) / w.sum()
    np.testing.assert_allclose(com, c, atol=0.5 * vox)


def test_phantom_density_voxelisation():
    ph = synth.sphere_phantom((1.0, -2.0, 0.5), 10.0, density=0.7)
    d = synth.phantom_density(ph, (40, 40, 40), 1.0)
    # volume of the voxelised sphere ~ 4/3 pi r^3
    assert (d > 0).sum() == pytest.approx(4 / 3 * math.pi * 1000, rel=0.03)
    assert d.max() == pytest.approx(0.7)
