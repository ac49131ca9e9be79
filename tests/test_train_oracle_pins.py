"""Pins of the FP64 training-step oracle (oracle/train64.py) against facts outside it:
closed forms of SSIM, finite differences of the loss, torch.optim.Adam, the definitions of
the activations and of PSNR."""
import numpy as np
import pytest

from oracle import train64 as T


def test_window_is_a_normalised_gaussian():
    w = T.gaussian_window()
    assert w.shape == (11,) and w.sum() == pytest.approx(1.0)
    assert w[5] / w[6] == pytest.approx(np.exp(1 / 4.5))
    np.testing.assert_allclose(w, w[::-1])


def test_ssim_of_an_image_with_itself_is_one_and_stationary():
    gen = np.random.default_rng(0)
    x = gen.uniform(0, 1, size=(2, 20, 23))
    r = T.loss_l1_ssim64(x, x, gamma=0.2)
    assert r["ssim"] == pytest.approx(1.0, abs=1e-12)
    assert r["loss"] == pytest.approx(0.0, abs=1e-12)
    assert np.abs(r["grad"]).max() < 1e-12


def test_ssim_of_constant_images_closed_form():
    a, b = 0.3, 0.7
    x = np.full((1, 30, 30), a)
    y = np.full((1, 30, 30), b)
    S = T.ssim_map64(x, y)["S"]
    # away from the zero-padded border the variances vanish and SSIM = (2ab + C1) / (a^2 + b^2 + C1)
    assert S[0, 15, 15] == pytest.approx((2 * a * b + T.C1) / (a * a + b * b + T.C1), rel=1e-12)


def test_ssim_of_affine_copy_interior():
    # y = s x + t in a region far from the border: sigma_xy = s sigma_x^2, sigma_y^2 = s^2 sigma_x^2
    gen = np.random.default_rng(1)
    x = gen.uniform(0.2, 0.8, size=(1, 40, 40))
    s, t = 0.5, 0.1
    y = s * x + t
    m = T.ssim_map64(x, y)
    w = m["w"]
    from scipy.ndimage import correlate1d

    def blur(a):
        return correlate1d(correlate1d(a, w, axis=-1, mode="constant"), w, axis=-2, mode="constant")
    mx = blur(x)
    vx = blur(x * x) - mx * mx
    my = s * mx + t
    want = (2 * mx * my + T.C1) * (2 * s * vx + T.C2) / ((mx * mx + my * my + T.C1) * (vx + s * s * vx + T.C2))
    np.testing.assert_allclose(m["S"][0, 10:30, 10:30], want[0, 10:30, 10:30], rtol=1e-10)


def test_loss_gradient_matches_central_differences():
    gen = np.random.default_rng(2)
    y = gen.uniform(0, 1, size=(2, 9, 12))
    x = np.clip(y + gen.normal(0, 0.2, size=y.shape), 0, 1)
    g = T.loss_l1_ssim64(x, y, gamma=0.2)["grad"]
    eps = 1e-6
    for idx in [(0, 0, 0), (0, 4, 5), (1, 8, 11), (1, 3, 0), (0, 6, 9)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (T.loss_l1_ssim64(xp, y)["loss"] - T.loss_l1_ssim64(xm, y)["loss"]) / (2 * eps)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    gen = np.random.default_rng(3)
    p0 = gen.normal(size=50)
    grads = [gen.normal(size=50) for _ in range(6)]
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = T.adam64(p, g, m, v, t, 1e-2)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_adam_first_step_and_decay_schedule():
    g = np.array([3.0, -0.5, 1e-3])
    p, _, _ = T.adam64(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.1)
    np.testing.assert_allclose(p, -0.1 * np.sign(g), rtol=1e-9)
    # exponential decay: lr at step T is lr_final, halfway the geometric mean
    for t, want in [(1000, 1.9e-6), (500, np.sqrt(1.9e-4 * 1.9e-6))]:
        q, _, _ = T.adam64(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), t, 1.9e-4, lr_final=1.9e-6,
                           decay_steps=1000)
        mhat = (1 - 0.9) / (1 - 0.9 ** t)
        vhat = (1 - 0.999) / (1 - 0.999 ** t)
        assert -q[0] == pytest.approx(want * mhat / np.sqrt(vhat), rel=1e-9)


def test_activation_chain_rule_matches_central_differences():
    gen = np.random.default_rng(4)
    n, nf = 7, 5
    ls, ol, f = gen.normal(size=(3, n)), gen.normal(size=n), gen.normal(size=(nf, n))
    lam = gen.uniform(0.5, 1.5, size=nf)
    gs, go, gi = gen.normal(size=(3, n)), gen.normal(size=n), gen.normal(size=n)

    def L(ls_, ol_, f_):
        s, o, i = T.activate64(ls_, ol_, f_, lam)
        return (gs * s).sum() + (go * o).sum() + (gi * i).sum()
    a_ls, a_ol, a_f = T.activate_bwd64(ls, ol, f, lam, gs, go, gi)
    eps = 1e-6
    for arr, grad in ((ls, a_ls), (ol, a_ol), (f, a_f)):
        for idx in [tuple(0 for _ in arr.shape), tuple(d - 1 for d in arr.shape)]:
            ap, am = arr.copy(), arr.copy()
            ap[idx] += eps
            am[idx] -= eps
            args_p = [ap if a is arr else a for a in (ls, ol, f)]
            args_m = [am if a is arr else a for a in (ls, ol, f)]
            assert grad[idx] == pytest.approx((L(*args_p) - L(*args_m)) / (2 * eps), rel=1e-6, abs=1e-9)
    s, o, i = T.activate64(ls, ol, f, lam)
    np.testing.assert_allclose(i, 1 / (1 + np.exp(-(lam[:, None] * f).sum(0))))


def test_psnr_definition():
    x = np.zeros((2, 4, 4))
    y = x.copy()
    y[0] += 0.1
    y[1, 0, 0] = 1.0
    np.testing.assert_allclose(T.psnr64(x, y), [20.0, -10 * np.log10(1 / 16)])
