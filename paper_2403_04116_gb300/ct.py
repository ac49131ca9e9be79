"""CT reconstruction from projections: FDK (xg_fdk) over device tensors, and the 3-D PSNR
used to score a reconstruction against a known volume."""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B
from .render import _stream_handle


def fdk(projections: torch.Tensor, views, shape, voxel_mm: float, stream=None) -> torch.Tensor:
    """Volume [nz, ny, nx] reconstructed from projections [V, H, W] (CUDA float32) of a full
    circular scan with the given views (evenly spaced over 2 pi, one scanner)."""
    views = list(views)
    V, H, W = projections.shape
    if len(views) != V or projections.dtype != torch.float32 or not projections.is_cuda:
        raise ValueError("expected CUDA float32 projections [V, H, W] matching the views")
    nb = B.xg_fdk_workspace_bytes(V, W, H)
    if nb == 0:
        raise ValueError("invalid scan size")
    raw = torch.empty(nb + 256, dtype=torch.uint8, device=projections.device)
    ws = raw[(-raw.data_ptr()) % 256:][:nb]
    nz, ny, nx = shape
    out = torch.empty(nz, ny, nx, dtype=torch.float32, device=projections.device)
    p = projections.contiguous()
    B.xg_fdk(views, p.data_ptr(), B.XgVolume(nx, ny, nz, 0, float(voxel_mm)), out.data_ptr(), ws.data_ptr(), nb,
             _stream_handle(stream))
    return out


def psnr3d(volume: np.ndarray, truth: np.ndarray) -> float:
    """PSNR of a volume against the true one, the peak being the true volume's maximum."""
    v, t = np.asarray(volume, np.float64), np.asarray(truth, np.float64)
    mse = float(((v - t) ** 2).mean())
    return 10.0 * math.log10(float(t.max()) ** 2 / mse) if mse > 0 else float("inf")
