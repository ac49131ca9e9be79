"""Seeded synthetic inputs shaped like X-Gaussian's circular cone-beam scans.

This module is shared by the tests, the benchmark and the smoke check, on both the
CUDA side and the oracle side.  It holds none of the rasterizer's arithmetic: it draws
random Gaussian attributes, lays out scan angles, and integrates density along straight
rays through an analytic ellipsoid phantom (the stand-in for the CT-derived projections
of the paper's Sec. 4.1, whose datasets are not available here).

Conventions (paper Sec. 3.3, Eq. 12): the world origin is the centre of the scanned
object; the source orbits in the z = 0 plane at distance ``sod_mm``; the detector is
``sdd_mm`` from the source.  Angles are in radians.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SOD_MM = 1000.0
SDD_MM = 1500.0
PITCH_MM = 1.0
SEED_BASE = 0x5847_0000


@dataclass(frozen=True)
class View:
    """One cone-beam projection: scanner distances (mm), detector pitch (mm), azimuth (rad), detector size (px)."""

    sod_mm: float
    sdd_mm: float
    pitch_u_mm: float
    pitch_v_mm: float
    angle_rad: float
    width: int
    height: int


def rng(config_id: int, stream: int) -> np.random.Generator:
    """Independent generator for (workload id, sub-stream): 0 = Gaussians, 1 = phantom, 2 = sampling."""
    ss = np.random.SeedSequence(SEED_BASE + config_id)
    return np.random.default_rng(ss.spawn(stream + 1)[stream])


def scene_side_mm(width: int, pitch_mm: float = PITCH_MM, sod_mm: float = SOD_MM, sdd_mm: float = SDD_MM) -> float:
    """Side of the scanned cuboid: half the field of view at the rotation centre."""
    return 0.5 * width * pitch_mm * sod_mm / sdd_mm


def gaussians(n: int, side_mm: float, gen: np.random.Generator,
              log_scale=(-5.0, -3.0), opacity=(0.05, 0.5), intensity=(0.0, 1.0)) -> dict:
    """Random activated Gaussians, structure-of-arrays, float32.

    means uniform in the cube [-side/2, side/2]^3, per-axis log-scales uniform in
    ``log_scale`` (in units of the cube side), quaternions (w, x, y, z) uniform on S^3,
    opacity and intensity uniform.
    """
    mean = (gen.uniform(-0.5, 0.5, size=(3, n)) * side_mm).astype(np.float32)
    scale = (np.exp(gen.uniform(log_scale[0], log_scale[1], size=(3, n))) * side_mm).astype(np.float32)
    q = gen.normal(size=(4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    quat = q.astype(np.float32)
    opac = gen.uniform(opacity[0], opacity[1], size=n).astype(np.float32)
    inten = gen.uniform(intensity[0], intensity[1], size=n).astype(np.float32)
    return {"mean": mean, "scale": scale, "quat": quat, "opacity": opac, "intensity": inten}


def circular_views(n_views: int, width: int, height: int, span_rad: float = 2.0 * math.pi,
                   sod_mm: float = SOD_MM, sdd_mm: float = SDD_MM, pitch_mm: float = PITCH_MM,
                   first_rad: float = 0.0) -> list[View]:
    """``n_views`` projections at equal angular steps of ``span_rad / n_views``."""
    return [View(sod_mm, sdd_mm, pitch_mm, pitch_mm, first_rad + span_rad * k / n_views, width, height)
            for k in range(n_views)]


# ----------------------------------------------------------------------------------------
# analytic phantom: sum of homogeneous ellipsoids, projected by exact ray integrals
# ----------------------------------------------------------------------------------------

def ellipsoid_phantom(n_ell: int, side_mm: float, gen: np.random.Generator) -> dict:
    """Random ellipsoids inside the cube: centres in 0.6 of it, semi-axes 5-25 % of the side."""
    centre = gen.uniform(-0.3, 0.3, size=(n_ell, 3)) * side_mm
    axes = gen.uniform(0.05, 0.25, size=(n_ell, 3)) * side_mm
    q = gen.normal(size=(n_ell, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    rot = np.stack([_rot_from_unit_quat(qq) for qq in q])
    density = gen.uniform(0.1, 1.0, size=n_ell)
    return {"centre": centre, "axes": axes, "rot": rot, "density": density}


def _rot_from_unit_quat(q):
    # Rodrigues form: rotation by angle 2*acos(w) about (x, y, z) / |(x, y, z)|.
    w, v = q[0], q[1:]
    s = np.linalg.norm(v)
    if s == 0.0:
        return np.eye(3)
    k = v / s
    ang = 2.0 * math.atan2(s, w)
    kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * kx + (1.0 - math.cos(ang)) * (kx @ kx)


def detector_rays(view: View):
    """Source point (3,) and unit ray directions (H, W, 3) to every pixel centre.

    The source sits at sod*(cos a, sin a, 0); the detector plane is perpendicular to the
    source-origin line at distance sdd from the source; detector columns run along
    (-sin a, cos a, 0) and rows along (0, 0, -1); pixel (x, y) is centred at
    (x + 1/2, y + 1/2) pixels from the detector corner, the detector centre being at W/2, H/2.
    """
    a = view.angle_rad
    src = view.sod_mm * np.array([math.cos(a), math.sin(a), 0.0])
    toward = -np.array([math.cos(a), math.sin(a), 0.0])
    e_u = np.array([-math.sin(a), math.cos(a), 0.0])
    e_v = np.array([0.0, 0.0, -1.0])
    det_c = src + view.sdd_mm * toward
    xs = (np.arange(view.width) + 0.5 - view.width / 2.0) * view.pitch_u_mm
    ys = (np.arange(view.height) + 0.5 - view.height / 2.0) * view.pitch_v_mm
    pts = det_c[None, None, :] + xs[None, :, None] * e_u[None, None, :] + ys[:, None, None] * e_v[None, None, :]
    d = pts - src[None, None, :]
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    return src, d


def phantom_line_integrals(ph: dict, view: View) -> np.ndarray:
    """Sum over ellipsoids of density x chord length along each pixel's ray (float64, H x W)."""
    src, d = detector_rays(view)
    out = np.zeros(d.shape[:2])
    for c, ax, r, rho in zip(ph["centre"], ph["axes"], ph["rot"], ph["density"]):
        # map into the ellipsoid's unit-sphere frame: x_loc = R^T (x - c) / axes
        o = (r.T @ (src - c)) / ax
        dl = np.einsum("ij,hwj->hwi", r.T, d) / ax
        qa = np.einsum("hwi,hwi->hw", dl, dl)
        qb = 2.0 * np.einsum("hwi,i->hw", dl, o)
        qc = float(o @ o) - 1.0
        disc = qb * qb - 4.0 * qa * qc
        hit = disc > 0.0
        # chord parameter length |t1 - t0| = sqrt(disc)/qa, rays are unit length in world units
        out[hit] += rho * np.sqrt(disc[hit]) / qa[hit]
    return out


def phantom_density(ph: dict, shape, voxel_mm: float) -> np.ndarray:
    """Density of the phantom at the voxel centres of a [nz, ny, nx] volume centred on the
    origin (voxel (i, j, k) at ((i + 1/2 - nx/2) s, (j + 1/2 - ny/2) s, (k + 1/2 - nz/2) s))."""
    nz, ny, nx = shape
    axes = [(np.arange(m) + 0.5 - m / 2.0) * voxel_mm for m in (nx, ny, nz)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    pts = np.stack([X, Y, Z], axis=-1)
    out = np.zeros(shape)
    for c, ax, r, rho in zip(ph["centre"], ph["axes"], ph["rot"], ph["density"]):
        loc = np.einsum("ij,...j->...i", r.T, pts - c) / ax
        out[(loc * loc).sum(axis=-1) <= 1.0] += rho
    return out


def sphere_phantom(centre, radius: float, density: float = 1.0) -> dict:
    return {"centre": np.asarray([centre], np.float64), "axes": np.full((1, 3), float(radius)),
            "rot": np.eye(3)[None], "density": np.asarray([density], np.float64)}


def phantom_targets(ph: dict, views: list[View]) -> np.ndarray:
    """Projections of the phantom for every view, scaled by their common maximum to [0, 1]."""
    imgs = np.stack([phantom_line_integrals(ph, v) for v in views])
    m = imgs.max()
    return (imgs / m if m > 0 else imgs).astype(np.float32)


def projection_noise(images: np.ndarray, level: float, gen: np.random.Generator) -> np.ndarray:
    """Targets with additive zero-mean Gaussian noise of standard deviation ``level`` times
    each view's value range: the paper's measured projections carry 3 % noise (Sec. 4.1),
    whose model it does not state; this is the reading."""
    images = np.asarray(images, np.float64)
    flat = images.reshape(images.shape[0], -1)
    span = (flat.max(axis=1) - flat.min(axis=1)).reshape(-1, *([1] * (images.ndim - 1)))
    return images + gen.normal(0.0, 1.0, size=images.shape) * level * span
