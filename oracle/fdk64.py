"""FP64 oracle of FDK cone-beam reconstruction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the benchmark's CPU baseline may import this module.

The paper's downstream use of rendered projections is CT reconstruction (Sec. 4, Table 2).
This is the Feldkamp-Davis-Kress algorithm for a full circular scan with a flat detector,
in the scanner geometry of Eq. 12 (source at L_SO (cos a, sin a, 0), detector columns
along (-sin a, cos a, 0), rows along (0, 0, -1), pixel (x, y) centred at (x + 1/2, y + 1/2)
pixels from the detector corner), written from the method's three steps:

1. weight: P_w(p, zeta) = P(p, zeta) D / sqrt(D^2 + p^2 + zeta^2), with D = L_SO and (p, zeta)
   the pixel centre scaled to the plane through the rotation axis (tau = pitch L_SO / L_SD);
2. filter every detector row with the ramp (Ram-Lak) kernel sampled at tau:
   h[0] = 1 / (4 tau^2), h[n odd] = -1 / (pi^2 n^2 tau^2), h[n even] = 0, Q = tau (h * P_w);
3. back-project: f(mu) = (dbeta / 2) sum over views of U^2 Q(p, zeta), U = D / t_z, the
   voxel's projection (p, zeta) = U (t_x, t_y) with t = M_ext mu, sampled bilinearly (zero
   outside the detector); dbeta = 2 pi / V for V views evenly spaced over the circle.

The volume is [nz][ny][nx]; voxel (i, j, k) is centred at
((i + 1/2 - nx/2) s, (j + 1/2 - ny/2) s, (k + 1/2 - nz/2) s), s the voxel size in mm.
"""
from __future__ import annotations

import math

import numpy as np


def ramp_kernel64(n: int, tau: float) -> np.ndarray:
    """h[-(n-1) .. n-1] of the discrete ramp filter, index n - 1 holding h[0]."""
    k = np.arange(-(n - 1), n)
    h = np.zeros(k.size)
    h[k == 0] = 1.0 / (4.0 * tau * tau)
    odd = (k % 2) != 0
    h[odd] = -1.0 / (math.pi ** 2 * k[odd].astype(np.float64) ** 2 * tau * tau)
    return h


def filter_view64(proj: np.ndarray, view) -> np.ndarray:
    """Steps 1 and 2 for one projection [H, W] (float64)."""
    H, W = proj.shape
    D = view.sod_mm
    tau_u = view.pitch_u_mm * view.sod_mm / view.sdd_mm
    tau_v = view.pitch_v_mm * view.sod_mm / view.sdd_mm
    p = (np.arange(W) + 0.5 - W / 2.0) * tau_u
    z = (np.arange(H) + 0.5 - H / 2.0) * tau_v
    pw = np.asarray(proj, np.float64) * (D / np.sqrt(D * D + p[None, :] ** 2 + z[:, None] ** 2))
    h = ramp_kernel64(W, tau_u)
    # Toeplitz matrix T[k, x] = h[x - k]: Q = tau (P_w @ T)
    idx = np.arange(W)[None, :] - np.arange(W)[:, None] + (W - 1)
    return tau_u * (pw @ h[idx])


def voxel_centres(shape, voxel_mm: float):
    nz, ny, nx = shape
    x = (np.arange(nx) + 0.5 - nx / 2.0) * voxel_mm
    y = (np.arange(ny) + 0.5 - ny / 2.0) * voxel_mm
    z = (np.arange(nz) + 0.5 - nz / 2.0) * voxel_mm
    return np.meshgrid(z, y, x, indexing="ij")  # Z, Y, X each [nz, ny, nx]


def bilinear64(img: np.ndarray, xi: np.ndarray, yi: np.ndarray) -> np.ndarray:
    """img sampled at continuous pixel indices (pixel (x, y) centred at index (x, y)), 0 outside."""
    H, W = img.shape
    x0 = np.floor(xi).astype(np.int64)
    y0 = np.floor(yi).astype(np.int64)
    fx, fy = xi - x0, yi - y0
    out = np.zeros(xi.shape)
    for dy, wy in ((0, 1.0 - fy), (1, fy)):
        for dx, wx in ((0, 1.0 - fx), (1, fx)):
            xx, yy = x0 + dx, y0 + dy
            ok = (xx >= 0) & (xx < W) & (yy >= 0) & (yy < H)
            out[ok] += (wx * wy)[ok] * img[yy[ok], xx[ok]]
    return out


def fdk64(projections: np.ndarray, views, shape, voxel_mm: float) -> np.ndarray:
    """The reconstructed volume [nz, ny, nx] (float64) from projections [V, H, W]."""
    Z, Y, X = voxel_centres(shape, voxel_mm)
    vol = np.zeros(shape)
    dbeta = 2.0 * math.pi / len(views)
    for proj, v in zip(projections, views):
        Q = filter_view64(proj, v)
        H, W = Q.shape
        D = v.sod_mm
        c, s = math.cos(v.angle_rad), math.sin(v.angle_rad)
        tx = -s * X + c * Y
        ty = -Z
        tz = D - (c * X + s * Y)
        U = D / tz
        tau_u = v.pitch_u_mm * v.sod_mm / v.sdd_mm
        tau_v = v.pitch_v_mm * v.sod_mm / v.sdd_mm
        xi = U * tx / tau_u + W / 2.0 - 0.5
        yi = U * ty / tau_v + H / 2.0 - 0.5
        vol += U * U * bilinear64(Q, xi, yi)
    return vol * (dbeta / 2.0)
