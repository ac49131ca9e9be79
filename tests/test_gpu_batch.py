"""The batched, graph-captured step and the plain one-view-per-launch form compute the
same images as direct calls (bit for bit) and the same gradients (up to the order of float
atomics); replays pick up new inputs; the autotuner's choice does not change results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2403_04116_gb300 import synth  # noqa: E402
from paper_2403_04116_gb300.batch import GraphedStep, PlainSteps, autotune, size_pairs  # noqa: E402
from paper_2403_04116_gb300.render import FrameConfig  # noqa: E402
from tests.gpu_util import NAMES, run_backward, run_forward, to_device  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2403_04116_gb300 import build
    build.build()


def _scene(cid=41, n=4000, V=6, W=96, H=80):
    side = synth.scene_side_mm(W)
    g = synth.gaussians(n, side, synth.rng(cid, 0))
    views = synth.circular_views(V, W, H, first_rad=0.2)
    ph = synth.ellipsoid_phantom(10, side, synth.rng(cid, 1))
    target = torch.from_numpy(synth.phantom_targets(ph, views)).cuda()
    return g, views, target


def _close(a, b):
    np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5 * max(np.abs(b).max(), 1e-30))


def test_graphed_step_matches_direct_calls_and_replays_new_inputs():
    g, views, target = _scene()
    cfg = FrameConfig(16, 16)
    dev = to_device(g)
    cap = size_pairs(dev[4].shape[0], views, cfg, dev)
    step = GraphedStep(dev[4].shape[0], views, cfg, cap)
    step.load(dev, target)
    step.capture()
    for trial in range(2):
        if trial == 1:  # new contents, same graph
            g = {k: v.copy() for k, v in g.items()}
            g["mean"] += np.float32(0.5)
            g["opacity"] *= np.float32(0.9)
            step.load(to_device(g))
        step.replay()
        torch.cuda.synchronize()
        ref = run_forward(g, views, (16, 16))
        np.testing.assert_array_equal(step.image.cpu().numpy(), ref["image"])
        G = np.sign(ref["image"] - target.cpu().numpy()) / ref["image"].size
        grads = run_backward(ref, G.astype(np.float32))
        for t, k in zip(step.grads, NAMES):
            _close(t.cpu().numpy(), grads[k])


def test_graph_with_host_transfers_matches_the_device_step():
    """capture_host: the inputs copied from pinned host tensors inside the graph (targets
    overlapped with the forward pass) and the loss copied back give the device step's
    results, and a replay after the host tensors change sees the new contents."""
    g, views, target = _scene()
    cfg = FrameConfig(16, 16)
    dev = to_device(g)
    n = dev[4].shape[0]
    step = GraphedStep(n, views, cfg, size_pairs(n, views, cfg, dev))
    host = tuple(t.cpu().pin_memory() for t in dev)
    host_target = target.cpu().pin_memory()
    step.load(dev, target)
    step.capture()
    step.capture_host(host, host_target)
    for trial in range(2):
        if trial == 1:
            host[0].add_(0.5)
            step.load(tuple(t.cuda() for t in host))
        step.replay()
        torch.cuda.synchronize()
        image, loss = step.image.clone(), step.loss.clone()
        grads = [t.clone() for t in step.grads]
        step.image.zero_()
        step.replay_host()
        torch.cuda.current_stream().synchronize()
        assert torch.equal(step.image, image)
        assert float(step.host_loss[0]) == pytest.approx(float(loss), rel=1e-6)
        for a, b in zip(step.grads, grads):
            _close(a.cpu().numpy(), b.cpu().numpy())
    # pipelined: the step in its second loss slot is enqueued before the first one's loss is
    # read; both read the same host inputs, so both losses equal the device step's
    step.replay()
    torch.cuda.synchronize()
    loss = float(step.loss)
    step.replay_host(0)
    step.replay_host(1)
    assert step.loss_of(0) == pytest.approx(loss, rel=1e-6)
    assert step.loss_of(1) == pytest.approx(loss, rel=1e-6)


def test_plain_per_view_form_matches_batched():
    g, views, target = _scene(cid=42, V=4)
    cfg = FrameConfig(8, 8, batch=64)
    dev = to_device(g)
    n = dev[4].shape[0]
    step = GraphedStep(n, views, cfg, size_pairs(n, views, cfg, dev))
    step.load(dev, target)
    step.capture()
    step.replay()
    plain = PlainSteps(n, views, cfg, size_pairs(n, views[:1], cfg, dev, margin=2.0))
    grads = tuple(torch.empty_like(t) for t in dev)
    plain.run(dev, target, grads)
    torch.cuda.synchronize()
    for v in range(len(views)):
        np.testing.assert_array_equal(plain.images[v][0].cpu().numpy(), step.image[v].cpu().numpy())
    for a, b in zip(grads, step.grads):
        _close(a.cpu().numpy(), b.cpu().numpy())


def test_autotune_choice_keeps_the_image():
    g, views, target = _scene(cid=43, V=3)
    dev = to_device(g)
    n = dev[4].shape[0]
    best = autotune(n, views, dev, target, tiles=((8, 8), (16, 16)), batches=(64, 256), reps=2, use_cache=False)
    assert (best.tile_w, best.tile_h) in ((8, 8), (16, 16)) and best.batch in (64, 256) and best.ms > 0
    a = GraphedStep(n, views, best.config(), best.pair_capacity)
    b = GraphedStep(n, views, FrameConfig(32, 16, batch=128), size_pairs(n, views, FrameConfig(32, 16), dev))
    for s in (a, b):
        s.load(dev, target)
        s.capture()
        s.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.image.cpu().numpy(), b.image.cpu().numpy())


@pytest.mark.parametrize("tile,ppt", [((8, 8), 2), ((16, 16), 1), ((32, 16), 4)])
@pytest.mark.parametrize("batch", [64, 128, 256, 512])
def test_launch_forms_and_batches_give_identical_images(tile, ppt, batch):
    """Persistent blocks (warps taking work items from a counter) and one block per (view,
    tile), at every staging batch the configuration's shared memory allows: the same images
    bit for bit as the plain one-view-per-launch form, and the same gradients up to the
    order of float atomics."""
    g, views, target = _scene(cid=44, V=3)
    dev = to_device(g)
    n = dev[4].shape[0]
    ref_cfg = FrameConfig(8, 8, batch=64)
    plain = PlainSteps(n, views, ref_cfg, size_pairs(n, views[:1], ref_cfg, dev, margin=2.0))
    pgrads = tuple(torch.empty_like(t) for t in dev)
    plain.run(dev, target, pgrads)
    checked = 0
    for persistent in (0, 1):
        cfg = FrameConfig(*tile, batch=batch, pixels_per_thread=ppt, persistent=persistent)
        try:
            step = GraphedStep(n, views, cfg, size_pairs(n, views, cfg, dev))
        except ValueError:
            continue  # this batch needs more shared memory than one block has
        step.load(dev, target)
        step.capture()
        step.replay()
        torch.cuda.synchronize()
        for v in range(len(views)):
            np.testing.assert_array_equal(step.image[v].cpu().numpy(), plain.images[v][0].cpu().numpy())
        for a, b in zip(step.grads, pgrads):
            _close(a.cpu().numpy(), b.cpu().numpy())
        checked += 1
    if batch <= 128:
        assert checked == 2
