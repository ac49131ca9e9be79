"""Parity at the benchmark's full size and in its launch configuration.

Workload: 50,000 Gaussians uniform in the scanned cuboid, 50 views over 360 degrees,
256 x 256 detector, the L1 loss against ellipsoid-phantom projections; the step is the
autotuned, graph-captured batched step that bench.py times.  Checked on samples the
oracles can compute:

* three views: every index quantity (contributor counts, last positions, transmittance)
  and the image bit-exact against the FP32 replica, the tile lists too;
* 4096 random pixels of every view: within 1e-4 of the FP64 oracle (ambiguous ones 1e-2);
* the gradients of 40 random Gaussians (480 parameters): within tolerance of the FP64
  oracle, with the same upstream gradient on both sides.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2403_04116_gb300 import synth  # noqa: E402
from paper_2403_04116_gb300.batch import GraphedStep, autotune  # noqa: E402
from tests.gpu_util import NAMES, to_device  # noqa: E402

pytestmark = pytest.mark.gpu

N, V, W = 50_000, 50, 256
GRAD_RTOL, GRAD_ATOL, GRAD_TERM_REL = 1e-3, 1e-6, 3e-5


@pytest.fixture(scope="module")
def workload():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2403_04116_gb300 import build
    build.build()
    side = synth.scene_side_mm(W)
    g = synth.gaussians(N, side, synth.rng(1, 0))
    views = synth.circular_views(V, W, W)
    ph = synth.ellipsoid_phantom(10, side, synth.rng(1, 1))
    target = synth.phantom_targets(ph, views)
    dev = to_device(g)
    tdev = torch.from_numpy(target).cuda()
    tuned = autotune(N, views, dev, tdev)
    step = GraphedStep(N, views, tuned.config(), tuned.pair_capacity)
    step.load(dev, tdev)
    step.capture()
    step.replay()
    torch.cuda.synchronize()
    return {"g": g, "views": views, "target": target, "step": step, "tuned": tuned, "dev": dev}


def test_sampled_views_bit_exact_against_replica(workload):
    step, tuned = workload["step"], workload["tuned"]
    tile = (tuned.tile_w, tuned.tile_h)
    f = step.frame
    image = step.image.cpu().numpy()
    tfin = f.array("tfinal").cpu().numpy().reshape(V, W, W)
    last = f.array("last").cpu().numpy().view(np.uint32).reshape(V, W, W)
    rng = f.array("range").cpu().numpy().view(np.uint32).reshape(V, f.range_stride, 2)[:, :f.tiles_per_view]
    val = f.array("value").cpu().numpy()
    for v in (0, 17, 49):
        rep = oracle.replica_full(workload["g"], workload["views"][v], tile)
        np.testing.assert_array_equal(image[v].view(np.uint32), rep["image"].view(np.uint32))
        np.testing.assert_array_equal(tfin[v].view(np.uint32), rep["tfinal"].view(np.uint32))
        np.testing.assert_array_equal(last[v], rep["last"])
        lens = rng[v, :, 1].astype(np.int64) - rng[v, :, 0]
        np.testing.assert_array_equal(lens, (rep["range"][:, 1].astype(np.int64) - rep["range"][:, 0]))
        nz = lens > 0
        for t in np.nonzero(nz)[0][::7]:
            a, b = rng[v, t]
            c, d = rep["range"][t]
            np.testing.assert_array_equal(val[a:b], rep["list"][c:d])


def test_sampled_pixels_against_fp64_oracle(workload):
    image = workload["step"].image.cpu().numpy()
    gen = np.random.default_rng(3)
    over = 0
    for v, view in enumerate(workload["views"]):
        pix = np.sort(gen.choice(W * W, size=4096, replace=False))
        ref = oracle.render64(workload["g"], view, pixels=pix)
        got = image[v].reshape(-1)[pix].astype(np.float64)
        want = ref["image"].reshape(-1)[pix]
        amb = ref["ambiguous"].reshape(-1)[pix] != 0
        err = np.abs(got - want)
        assert err[~amb].max() <= 1e-4, (v, err[~amb].max())
        assert err.max() <= 1e-2
        over += int((err > 1e-4).sum())
    assert over <= 1e-3 * V * 4096


def test_sampled_gradients_against_fp64_oracle(workload):
    g, views, step = workload["g"], workload["views"], workload["step"]
    gen = np.random.default_rng(4)
    sample = np.sort(gen.choice(N, size=40, replace=False))
    # the pixels where the sampled Gaussians can contribute, per view
    G = np.zeros((V, W, W))
    pix_of = []
    yy, xx = np.mgrid[0:W, 0:W]
    for v, view in enumerate(views):
        pr = oracle.project64({k: g[k][..., sample] for k in g}, view)
        mask = np.zeros((W, W), bool)
        for k in range(len(sample)):
            if not pr[k, 0]:
                continue
            dx, dy = pr[k, 4] - (xx + 0.5), pr[k, 5] - (yy + 0.5)
            a, b, c = pr[k, 9:12]
            mask |= g["opacity"][sample[k]] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)) >= 1 / 255
        pix = np.nonzero(mask.reshape(-1))[0].astype(np.int32)
        pix_of.append(pix)
        ref = oracle.render64(g, view, pixels=pix)
        # the summed-L1 gradient (+-1) from the oracle's own image, zero where a decision is
        # ambiguous; unscaled, so gradients sit well above the 1e-6 absolute floor
        Gv = np.zeros(W * W)
        Gv[pix] = np.sign(ref["image"].reshape(-1)[pix] - workload["target"][v].reshape(-1)[pix])
        Gv[pix[ref["ambiguous"].reshape(-1)[pix] != 0]] = 0.0
        G[v] = Gv.reshape(W, W)
    ora = None
    for v, view in enumerate(views):
        ora = oracle.grad64(g, view, G[v], pixels=pix_of[v], out=ora)
    f = step.frame
    grads = tuple(torch.empty_like(t) for t in workload["dev"])
    f.render_bwd(workload["dev"], torch.from_numpy(G.astype(np.float32)).cuda(), grads)
    torch.cuda.synchronize()
    checked = 0
    for t, k in zip(grads, NAMES):
        got = t.cpu().numpy()[..., sample].astype(np.float64)
        want = ora[k][..., sample]
        mag = ora["mag"][k][..., sample]
        bad = np.abs(got - want) > GRAD_RTOL * np.abs(want) + GRAD_ATOL + GRAD_TERM_REL * mag
        assert not bad.any(), (k, got[bad][:4], want[bad][:4])
        checked += want.size
    assert checked == 40 * 12
    assert np.count_nonzero(np.abs(ora["mean"][:, sample]) > 1e-3) > 60  # gradients well above the floor
