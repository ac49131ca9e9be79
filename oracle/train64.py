"""FP64 oracle of the training step around the rasterizer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the benchmark's CPU baseline may import this module.  Plain NumPy /
SciPy in float64, written from the definitions:

* activations of the radiative Gaussian model (Sec. 3.1): scale = exp(s),
  opacity = sigmoid(o), intensity = RIRF(f) = sigmoid(sum_k lambda_k f_k) (Eq. 3, the
  weights applied as an inner product), and their chain rule;
* the training objective of Eq. 11, (1 - gamma) L1 + gamma (1 - SSIM), SSIM as defined by
  Wang et al. with an 11-tap Gaussian window of sigma 1.5, zero padding, C1 = 0.01^2,
  C2 = 0.03^2, and its gradient with respect to the rendered image;
* Adam (beta1, beta2, eps, bias correction) with the exponential learning-rate decay of
  Sec. 4.1;
* PSNR with peak 1.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate1d

C1 = 0.01 ** 2
C2 = 0.03 ** 2


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def activate64(log_scale, opacity_logit, features, lam):
    """scale[3, n], opacity[n], intensity[n] from the raw parameters (float64)."""
    log_scale, opacity_logit, features, lam = (np.asarray(a, np.float64) for a in
                                               (log_scale, opacity_logit, features, lam))
    return np.exp(log_scale), sigmoid(opacity_logit), sigmoid(lam @ features)


def activate_bwd64(log_scale, opacity_logit, features, lam, g_scale, g_opacity, g_intensity):
    """dL/dlog_scale, dL/dopacity_logit, dL/dfeatures from the activated gradients."""
    log_scale, opacity_logit, features, lam = (np.asarray(a, np.float64) for a in
                                               (log_scale, opacity_logit, features, lam))
    o = sigmoid(opacity_logit)
    i = sigmoid(lam @ features)
    gz = np.asarray(g_intensity, np.float64) * i * (1 - i)
    return (np.asarray(g_scale, np.float64) * np.exp(log_scale), np.asarray(g_opacity, np.float64) * o * (1 - o),
            np.outer(lam, gz))


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    d = np.arange(size) - size // 2
    w = np.exp(-d * d / (2 * sigma * sigma))
    return w / w.sum()


def _blur(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Separable Gaussian blur of every view, zero outside the image."""
    a = correlate1d(a, w, axis=-1, mode="constant", cval=0.0)
    return correlate1d(a, w, axis=-2, mode="constant", cval=0.0)


def ssim_map64(x: np.ndarray, y: np.ndarray) -> dict:
    """SSIM map of images x, y ([V, H, W]) and the partial derivatives of each map value."""
    w = gaussian_window()
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _blur(x, w), _blur(y, w)
    sxx = _blur(x * x, w) - mx * mx
    syy = _blur(y * y, w) - my * my
    sxy = _blur(x * y, w) - mx * my
    n1, n2 = 2 * mx * my + C1, 2 * sxy + C2
    d1, d2 = mx * mx + my * my + C1, sxx + syy + C2
    S = n1 * n2 / (d1 * d2)
    return {"S": S, "mx": mx, "my": my, "dS_dmx": 2 * my * n2 / (d1 * d2) - S * 2 * mx / d1,
            "dS_dsxx": -S / d2, "dS_dsxy": 2 * n1 / (d1 * d2), "w": w}


def loss_l1_ssim64(x: np.ndarray, y: np.ndarray, gamma: float = 0.2) -> dict:
    """Eq. 11 over all pixels of all views, and its gradient with respect to x."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    P = x.size
    m = ssim_map64(x, y)
    # d mean(S) / dx(q) = (1/P) [w * A + 2 x (w * B) + y (w * C)]   (w symmetric, zero padded)
    A = m["dS_dmx"] - 2 * m["mx"] * m["dS_dsxx"] - m["my"] * m["dS_dsxy"]
    dS = (_blur(A, m["w"]) + 2 * x * _blur(m["dS_dsxx"], m["w"]) + y * _blur(m["dS_dsxy"], m["w"])) / P
    l1 = np.abs(x - y).mean()
    s = m["S"].mean()
    grad = (1 - gamma) * np.sign(x - y) / P - gamma * dS
    return {"loss": (1 - gamma) * l1 + gamma * (1 - s), "l1": l1, "ssim": s, "grad": grad, "map": m["S"]}


def adam64(param, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-15, lr_final=None,
           decay_steps: int = 0):
    """One Adam step taken as step number t (1-based); returns new (param, m, v)."""
    param, grad, m, v = (np.asarray(a, np.float64) for a in (param, grad, m, v))
    if decay_steps > 0:
        lr = lr * (lr_final / lr) ** min(t / decay_steps, 1.0)
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v


def psnr64(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """PSNR (peak 1) of each view of [V, ...] images."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mse = ((x - y) ** 2).reshape(x.shape[0], -1).mean(axis=1)
    return -10.0 * np.log10(mse)
