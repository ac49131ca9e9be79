"""Oracle of adaptive density control -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the benchmark's CPU baseline may import this module.

The paper adjusts the number of Gaussians with the adaptive control of 3D Gaussian
splatting (Sec. 3.2) without restating it.  This follows the published rules of that
method (Kerbl et al. 2023, Sec. 5), read as follows:

* statistics: after each step, every Gaussian visible in a view (touching at least one
  tile) adds the norm of its projected-centre gradient dL/du (times a caller-given
  scale) to ``accum`` and 1 to ``denom``;
* densify where accum / denom >= grad_thresh: a Gaussian whose largest scale is at most
  the size threshold is cloned (an identical copy), a larger one is split into two whose
  centres are drawn from the Gaussian itself (mu + R diag(s) z, z ~ N(0, I) supplied by the
  caller) and whose scales are s / 1.6;
* prune Gaussians whose opacity is below ``min_opacity`` or whose largest scale exceeds
  ``max_size`` (children are tested with their own scale);
* output order: for each source Gaussian in order, [itself if kept], [its clone],
  [child 0, child 1].

Parameters are raw (log-scales, opacity logits), and every integer decision is taken in
FP32 as the device takes it: the average by an IEEE FP32 division, compared with FP32
thresholds given in log / logit space.  The new geometry (split centres) is computed in
FP64.
"""
from __future__ import annotations

import numpy as np

SPLIT_FACTOR = 1.6


def densify_stats64(grad_u: np.ndarray, visible: np.ndarray, scale: float):
    """accum[n], denom[n] from per-view centre gradients grad_u[V, n, 2] and visibility[V, n]."""
    norms = np.sqrt((np.asarray(grad_u, np.float64) ** 2).sum(axis=-1))
    vis = np.asarray(visible, bool)
    return (np.where(vis, norms * scale, 0.0)).sum(axis=0), vis.sum(axis=0).astype(np.int64)


def quat_to_rot64(q: np.ndarray) -> np.ndarray:
    """Rotation matrices [n, 3, 3] of quaternions q[4, n] (w, x, y, z), normalised."""
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q, axis=0)
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], axis=-1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], axis=-1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=-1)], axis=-2)


def densify64(params: dict, accum, denom, normals, grad_thresh: float, size_log_thresh: float,
              prune_logit: float, max_log_size: float | None = None) -> dict:
    """One densify-and-prune step.  params: mean[3,n], log_scale[3,n], quat[4,n],
    opacity_logit[n], features[nf,n] (float32); normals[2, 3, n].  Returns the new
    parameters (float64 centres of children, float32 copies otherwise), ``src`` (source
    index of each output) and ``kind`` (0 kept, 1 clone, 2 child)."""
    f32 = np.float32
    ls = np.asarray(params["log_scale"], f32)
    ol = np.asarray(params["opacity_logit"], f32)
    acc = np.asarray(accum, f32)
    den = np.asarray(denom)
    with np.errstate(divide="ignore", invalid="ignore"):
        avg = np.where(den > 0, acc / den.astype(f32), f32(0))
    dens = avg >= f32(grad_thresh)
    maxls = ls.max(axis=0)
    big = maxls > f32(size_log_thresh)
    low = ol < f32(prune_logit)
    large = maxls > f32(max_log_size) if max_log_size is not None else np.zeros_like(low)
    ln_split = f32(np.log(SPLIT_FACTOR))
    child_large = ((maxls - ln_split) > f32(max_log_size)) if max_log_size is not None else np.zeros_like(low)
    split = dens & big
    keep = ~split & ~low & ~large
    clone = dens & ~big & ~low & ~large
    child = split & ~low & ~child_large

    R = quat_to_rot64(params["quat"])
    s = np.exp(np.asarray(ls, np.float64))
    mu = np.asarray(params["mean"], np.float64)
    z = np.asarray(normals, np.float64)
    src, kind, means, lsc = [], [], [], []
    for g in range(ol.shape[0]):
        if keep[g]:
            src.append(g), kind.append(0), means.append(mu[:, g]), lsc.append(np.asarray(ls[:, g], np.float64))
        if clone[g]:
            src.append(g), kind.append(1), means.append(mu[:, g]), lsc.append(np.asarray(ls[:, g], np.float64))
        if child[g]:
            for k in range(2):
                src.append(g), kind.append(2)
                means.append(mu[:, g] + R[g] @ (s[:, g] * z[k, :, g]))
                lsc.append(np.asarray(ls[:, g], np.float64) - np.log(SPLIT_FACTOR))
    src = np.asarray(src, np.int64)
    out = {"src": src, "kind": np.asarray(kind, np.int64),
           "mean": np.stack(means, axis=1) if means else np.zeros((3, 0)),
           "log_scale": np.stack(lsc, axis=1) if lsc else np.zeros((3, 0))}
    for k in ("quat", "opacity_logit", "features"):
        out[k] = np.asarray(params[k])[..., src]
    return out


def opacity_reset64(opacity_logit, reset_logit: float) -> np.ndarray:
    """Opacities capped at sigmoid(reset_logit), in logit space (FP32 minimum)."""
    return np.minimum(np.asarray(opacity_logit, np.float32), np.float32(reset_logit))
