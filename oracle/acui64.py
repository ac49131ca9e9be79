"""FP64 oracle of ACUI's grid initialisation (Sec. 3.3, Eq. 13) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the benchmark's CPU baseline may import this module.

A cuboid of S_1 x S_2 x S_3 mm centred on the origin is divided into an M_1 x M_2 x M_3
voxel grid; the Gaussian centres are the points (n_1 S_1 d / M_1, n_2 S_2 d / M_2,
n_3 S_3 d / M_3) for integers n_i with |n_i| <= [M_i / (2 d)] + 1, d the sampling interval
in voxels.  [.] is read as the floor.  Points are listed with n_1 slowest and n_3 fastest,
each n_i ascending.
"""
from __future__ import annotations

import math

import numpy as np


def half_count(M: int, d: float) -> int:
    """[M / (2 d)] + 1: the largest |n| on an axis of M voxels."""
    return math.floor(M / (2.0 * d)) + 1


def acui_count(size_mm, grid, d: float) -> int:
    return int(np.prod([2 * half_count(M, d) + 1 for M in grid]))


def acui_points64(size_mm, grid, d: float) -> np.ndarray:
    """The grid points of Eq. 13 as float64 [3, N] (x, y, z rows)."""
    axes = []
    for S, M in zip(size_mm, grid):
        c = half_count(M, d)
        n = np.arange(-c, c + 1, dtype=np.float64)
        axes.append(n * S * d / M)
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)])

