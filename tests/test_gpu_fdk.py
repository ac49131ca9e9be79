"""FDK reconstruction on the device against the FP64 oracle (same projections, same
geometry), and the reconstruction of an exactly projected sphere."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fdk64 as F  # noqa: E402
from paper_2403_04116_gb300 import binding as B  # noqa: E402
from paper_2403_04116_gb300 import synth  # noqa: E402
from paper_2403_04116_gb300.render import _stream_handle  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib(build_if_missing=True)


def _fdk_gpu(proj, views, shape, voxel):
    V, H, W = proj.shape
    nb = B.xg_fdk_workspace_bytes(V, W, H)
    raw = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ws = raw[(-raw.data_ptr()) % 256:][:nb]
    p = torch.from_numpy(np.ascontiguousarray(proj, np.float32)).cuda()
    out = torch.full(shape, float("nan"), device="cuda")
    B.xg_fdk(views, p.data_ptr(), B.XgVolume(shape[2], shape[1], shape[0], 0, voxel), out.data_ptr(),
             ws.data_ptr(), nb, _stream_handle())
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("W,H,V,shape", [(64, 64, 90, (40, 40, 40)), (48, 37, 60, (20, 33, 27))])
def test_fdk_matches_the_oracle(W, H, V, shape):
    side = synth.scene_side_mm(W)
    ph = synth.ellipsoid_phantom(4, side, synth.rng(70, W))
    views = synth.circular_views(V, W, H)
    proj = np.stack([synth.phantom_line_integrals(ph, v) for v in views]).astype(np.float32)
    voxel = side / 40
    want = F.fdk64(proj, views, shape, voxel)
    got = _fdk_gpu(proj, views, shape, voxel)
    assert np.isfinite(got).all()
    assert np.abs(got - want).max() <= 2e-5 * np.abs(want).max() + 1e-6


def test_fdk_off_centre_sphere():
    W, V, n = 64, 120, 40
    side = synth.scene_side_mm(W)
    vox = side / n
    c = np.array([0.15, -0.1, 0.05]) * side
    R = 0.3 * side
    views = synth.circular_views(V, W, W)
    proj = np.stack([synth.phantom_line_integrals(synth.sphere_phantom(c, R), v) for v in views])
    vol = _fdk_gpu(proj, views, (n, n, n), vox)
    Z, Y, X = F.voxel_centres((n, n, n), vox)
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    assert vol[r < 0.7 * R].mean() == pytest.approx(1.0, abs=0.03)
    assert np.abs(vol[(r > 1.3 * R) & (np.abs(Z) < 0.4 * side)]).mean() < 0.02
