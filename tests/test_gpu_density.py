"""Adaptive density control on the device against its oracle: the plan (counts, order) and
the applied parameters and Adam moments (copies bit-exact, split centres within FP32
rounding), the gradient statistics against the FP64 rasterizer's gradients, the opacity
reset, and a short training run whose Gaussian count changes."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import density64 as D  # noqa: E402
from paper_2403_04116_gb300 import binding as B  # noqa: E402
from paper_2403_04116_gb300 import synth  # noqa: E402
from paper_2403_04116_gb300.render import Frame, FrameConfig, _stream_handle  # noqa: E402
from tests.gpu_util import to_device  # noqa: E402

pytestmark = pytest.mark.gpu
KEYS = ("mean", "log_scale", "quat", "opacity_logit", "features")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib(build_if_missing=True)


def _dev(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _set(d, nf):
    return B.XgParamSet(*(d[k].data_ptr() for k in KEYS), nf, 0, d["mean"].shape[1])


def _random_state(n, nf, seed):
    gen = np.random.default_rng(seed)
    p = {"mean": gen.normal(0, 30, size=(3, n)), "log_scale": gen.uniform(-3, 1.5, size=(3, n)),
         "quat": gen.normal(size=(4, n)), "opacity_logit": gen.normal(-2, 2, size=n),
         "features": gen.normal(size=(nf, n))}
    p = {k: v.astype(np.float32) for k, v in p.items()}
    m = {k: gen.normal(size=v.shape).astype(np.float32) for k, v in p.items()}
    v = {k: gen.uniform(0, 1, size=x.shape).astype(np.float32) for k, x in p.items()}
    accum = gen.exponential(1.0, size=n).astype(np.float32)
    denom = gen.integers(0, 4, size=n).astype(np.int32)
    return p, m, v, accum, denom, gen.normal(size=(2, 3, n)).astype(np.float32)


@pytest.mark.parametrize("n,nf", [(5000, 4), (1, 2), (70000, 16)])
def test_plan_and_apply_match_the_oracle(n, nf):
    p, m, v, accum, denom, z = _random_state(n, nf, seed=n)
    rules = dict(grad_thresh=0.5, size_log_thresh=0.0, prune_logit=-4.0, max_log_size=1.2)
    want = D.densify64(p, accum, denom, z, **rules)
    dp, dm, dv = ({k: _dev(x[k]) for k in KEYS} for x in (p, m, v))
    da, dd, dz = _dev(accum), _dev(denom, np.int32), _dev(z)
    R = B.XgDensityRules(rules["grad_thresh"], rules["size_log_thresh"], rules["prune_logit"], rules["max_log_size"])
    offsets = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.xg_densify_workspace_bytes() // 4 + 4, dtype=torch.int32, device="cuda")
    s = _stream_handle()
    B.xg_densify_plan(_set(dp, nf), da.data_ptr(), dd.data_ptr(), R, offsets.data_ptr(), ws.data_ptr(), s)
    n_new = int(offsets[n].item())
    assert n_new == len(want["src"])
    shapes = {"mean": (3,), "log_scale": (3,), "quat": (4,), "opacity_logit": (), "features": (nf,)}
    out = [{k: torch.full((*shp, n_new), float("nan"), device="cuda") for k, shp in shapes.items()} for _ in range(3)]
    B.xg_densify_apply(_set(dp, nf), _set(dm, nf), _set(dv, nf), da.data_ptr(), dd.data_ptr(), R, offsets.data_ptr(),
                       dz.data_ptr(), _set(out[0], nf), _set(out[1], nf), _set(out[2], nf), s)
    got = [{k: t.cpu().numpy() for k, t in o.items()} for o in out]
    src, kind = want["src"], want["kind"]
    copy, child = kind < 2, kind == 2
    for k in ("quat", "opacity_logit", "features"):
        np.testing.assert_array_equal(got[0][k], p[k][..., src])
    for k in ("mean", "log_scale"):
        np.testing.assert_array_equal(got[0][k][:, copy], p[k][:, src[copy]])
    if child.any():
        s_par = np.exp(p["log_scale"][:, src[child]].astype(np.float64))
        tol = 2e-6 * (np.abs(p["mean"][:, src[child]]) + 3 * s_par.max(axis=0) * 4) + 1e-6
        assert (np.abs(got[0]["mean"][:, child] - want["mean"][:, child]) <= tol).all()
        np.testing.assert_allclose(got[0]["log_scale"][:, child], want["log_scale"][:, child], atol=3e-7)
    for st, mom in ((got[1], m), (got[2], v)):
        for k in KEYS:
            kept = kind == 0
            np.testing.assert_array_equal(st[k][..., kept], mom[k][..., src[kept]])
            assert (st[k][..., ~kept] == 0).all()
    if n > 1000:
        assert {0, 1, 2} <= set(kind.tolist()) and n_new != n


def test_statistics_match_the_fp64_gradients():
    W = H = 48
    n = 1500
    side = synth.scene_side_mm(W)
    g = synth.gaussians(n, side, synth.rng(51, 0))
    views = synth.circular_views(2, W, H, first_rad=0.3)
    gen = np.random.default_rng(5)
    G = np.zeros((2, H, W))
    grads, mags, vis = [], [], []
    for vi, view in enumerate(views):
        r = oracle.render64(g, view)
        Gv = gen.choice([-1.0, 1.0], size=(H, W))
        Gv[r["ambiguous"] != 0] = 0.0
        G[vi] = Gv
        o = oracle.grad64(g, view, Gv)
        grads.append(o["g2d"][0:2].T)
        mags.append(o["mag2d"][0:2].T)
        vis.append(oracle.replica_project(g, view, (16, 16))["count"] > 0)
    scale = 3.0
    want_acc, want_den = D.densify_stats64(np.stack(grads), np.stack(vis), scale)
    tol = (np.stack(vis) * (1e-3 * np.linalg.norm(np.stack(grads), axis=-1) + 1e-6 +
                            3e-5 * np.linalg.norm(np.stack(mags), axis=-1))).sum(axis=0) * scale
    dev = to_device(g)
    f = Frame(n, views, FrameConfig(16, 16), 1 << 18)
    f.project(*dev)
    f.bin_sort()
    img = torch.empty(2, H, W, device="cuda")
    f.render_fwd(img)
    f.render_bwd(dev, _dev(G), tuple(torch.empty_like(t) for t in dev))
    acc = torch.full((n,), 1.0, device="cuda")  # accumulates onto what is there
    den = torch.full((n,), 2, dtype=torch.int32, device="cuda")
    B.xg_densify_stats(f.handle, scale, acc.data_ptr(), den.data_ptr(), _stream_handle())
    np.testing.assert_array_equal(den.cpu().numpy(), want_den + 2)
    got = acc.cpu().numpy().astype(np.float64) - 1.0
    assert (np.abs(got - want_acc) <= tol + 1e-6).all()
    assert want_acc.max() > 1.0


def test_opacity_reset_matches_the_oracle():
    lo = np.random.default_rng(0).normal(-3, 3, size=1000).astype(np.float32)
    t = _dev(lo)
    m, v = _dev(np.ones(1000)), _dev(np.ones(1000))
    reset = math.log(0.01 / 0.99)
    B.xg_opacity_reset(t.data_ptr(), m.data_ptr(), v.data_ptr(), 1000, reset, _stream_handle())
    np.testing.assert_array_equal(t.cpu().numpy(), D.opacity_reset64(lo, reset))
    assert not m.cpu().numpy().any() and not v.cpu().numpy().any()


def test_training_with_density_control_changes_the_count_and_learns():
    from paper_2403_04116_gb300.train import TrainConfig, Trainer, config3, raw_from_activated
    side, tr_v, tr_t, te_v, te_t, g = config3(4000, 128, seed_id=62)
    cfg = TrainConfig(views_per_step=8, position_scale=side, decay_steps=400, densify=True, densify_from=50,
                      densify_interval=50, densify_until=351, opacity_reset_interval=200, grad_thresh=2e-4)
    raw = raw_from_activated(g, cfg.n_features, np.random.default_rng(1))
    tr = Trainer(raw, tr_v, torch.from_numpy(tr_t).cuda(), cfg, FrameConfig(16, 16))
    te = torch.from_numpy(te_t).cuda()
    before = tr.psnr(te_v, te).mean()
    tr.capture()
    tr.train(400, check_every=100)
    torch.cuda.synchronize()
    after = tr.psnr(te_v, te).mean()
    assert tr.n != 4000 and tr.p["mean"].shape == (3, tr.n)
    assert math.isfinite(after) and after > before + 1.0, (before, after, tr.n)
