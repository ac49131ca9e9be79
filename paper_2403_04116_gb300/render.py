"""PyTorch front end: frames over caller-owned workspaces, and the autograd Function.

PyTorch provides device memory and streams only; every stage runs in ``libxg.so``.
Gaussian attributes enter activated (scale > 0, opacity in [0, 1]); apply exp / sigmoid /
the paper's RIRF sigmoid (Eq. 3) in torch before calling, so autograd covers them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import binding as B

NEAR_MM = 0.2
_NAMES = ("mean", "scale", "quat", "opacity", "intensity")


def _stream_handle(stream: torch.cuda.Stream | None = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def gaussians_struct(mean, scale, quat, opacity, intensity) -> B.XgGaussians:
    n = intensity.shape[0]
    for t, shape in ((mean, (3, n)), (scale, (3, n)), (quat, (4, n)), (opacity, (n,)), (intensity, (n,))):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape:
            raise ValueError(f"expected a contiguous CUDA float32 tensor of shape {shape}, got "
                             f"{tuple(t.shape)} {t.dtype} on {t.device}")
    return B.XgGaussians(mean.data_ptr(), scale.data_ptr(), quat.data_ptr(), opacity.data_ptr(),
                         intensity.data_ptr(), n)


@dataclass
class FrameConfig:
    tile_w: int = 16
    tile_h: int = 16
    near_mm: float = NEAR_MM
    batch: int = 64  # list entries whose records each compositing warp keeps in flight
    pixels_per_thread: int = 2  # pixels each compositing thread owns (1, 2 or 4)
    persistent: int = 0  # 1: as many blocks as fit, warps taking work items from a counter


class Frame:
    """One batch of views sharing a detector size, with its device workspace.

    ``pair_capacity`` bounds the (view, tile, Gaussian) pairs of one pass; the workspace is
    allocated once here and reused by every call, so a sequence of calls can be
    graph-captured.  With ``views_per_pass`` below the view count the per-pass arrays hold
    that many views, and :meth:`select` picks the window the next calls render; ``V`` is
    the number of views of the current pass.
    """

    def __init__(self, n: int, views, cfg: FrameConfig | None = None, pair_capacity: int = 1 << 22,
                 device: torch.device | str | None = None, stream: torch.cuda.Stream | None = None,
                 views_per_pass: int = 0):
        self.cfg = cfg or FrameConfig()
        self.views = list(views)
        self.n = int(n)
        self.n_scan = len(self.views)
        self.views_per_pass = min(views_per_pass, self.n_scan) if views_per_pass > 0 else self.n_scan
        self.V = self.views_per_pass
        self.first = 0
        self.W, self.H = self.views[0].width, self.views[0].height
        self.pair_capacity = int(pair_capacity)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._c = B.XgConfig(self.cfg.tile_w, self.cfg.tile_h, self.cfg.near_mm, self.cfg.batch, self.pair_capacity,
                             self.cfg.pixels_per_thread, self.views_per_pass, self.cfg.persistent, 0)
        nbytes = B.xg_workspace_bytes(self._c, self.n, self.n_scan, self.W, self.H)
        if nbytes == 0:
            raise ValueError("invalid frame configuration")
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        pad = (-raw.data_ptr()) % 256
        self.workspace = raw[pad:pad + nbytes]
        self._raw = raw
        self.handle = B.xg_frame_create(self._c, self.n, self.views, self.workspace.data_ptr(), nbytes,
                                        _stream_handle(stream))
        self.layout = B.xg_frame_layout(self.handle)
        self.tiles_x, self.tiles_y = self.layout.tiles_x, self.layout.tiles_y
        self.tiles_per_view = self.layout.tiles_per_view
        self.range_stride = self.layout.range_stride  # range entry of (view, tile): view * stride + tile

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            B.xg_frame_destroy(h)
            self.handle = None

    # ---- stages -------------------------------------------------------------------------
    def project(self, mean, scale, quat, opacity, intensity, stream=None) -> None:
        B.xg_project(self.handle, gaussians_struct(mean, scale, quat, opacity, intensity), _stream_handle(stream))

    def bin_sort(self, stream=None) -> None:
        B.xg_bin_sort(self.handle, _stream_handle(stream))

    def render_fwd(self, image: torch.Tensor, n_contrib: torch.Tensor | None = None, stream=None) -> None:
        self._check_image(image, torch.float32)
        if n_contrib is not None:
            self._check_image(n_contrib, torch.int32)
        B.xg_render_fwd(self.handle, image.data_ptr(), n_contrib.data_ptr() if n_contrib is not None else None,
                        _stream_handle(stream))

    def render_bwd(self, gaussians: tuple, grad_image: torch.Tensor, grads: tuple, stream=None) -> None:
        self._check_image(grad_image, torch.float32)
        g = gaussians_struct(*gaussians)
        for t, ref in zip(grads, gaussians):
            if t.shape != ref.shape or t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
                raise ValueError("gradient buffers must match the Gaussian tensors")
        out = B.XgGrads(*[t.data_ptr() for t in grads])
        B.xg_render_bwd(self.handle, g, grad_image.data_ptr(), out, _stream_handle(stream))

    def select(self, first_view: int) -> int:
        """Render views first_view .. first_view + V - 1 in the calls that follow; returns V."""
        self.V = B.xg_frame_select_views(self.handle, first_view)
        self.first = first_view
        return self.V

    def status(self, stream=None) -> B.XgDeviceStatus:
        return B.xg_frame_read_status(self.handle, _stream_handle(stream))

    def copy_status(self, out: torch.Tensor, stream=None) -> None:
        """Enqueue a copy of the device status into ``out`` (CUDA int64 tensor of 7 entries:
        code and reserved packed in the first, then the fields of ``xg_device_status``)."""
        if out.dtype != torch.int64 or not out.is_cuda or out.numel() < 7 or not out.is_contiguous():
            raise ValueError("expected a contiguous CUDA int64 tensor of at least 7 entries")
        B.xg_frame_copy_status(self.handle, out.data_ptr(), _stream_handle(stream))

    def set_timing(self, enable: bool) -> None:
        B.xg_frame_set_timing(self.handle, enable)

    def read_timing(self) -> dict:
        return B.xg_frame_read_timing(self.handle)

    def _check_image(self, t: torch.Tensor, dtype) -> None:
        if t.dtype != dtype or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (self.V, self.H, self.W):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor of shape {(self.V, self.H, self.W)}")

    # ---- inspection of intermediate arrays ------------------------------------------------
    def array(self, name: str) -> torch.Tensor:
        """A view of one workspace array (see ``xg_layout`` in include/xg.h)."""
        VN = self.V * self.n
        cap = self.pair_capacity
        P = self.V * self.H * self.W
        spec = {
            "records": (torch.float32, (VN, 8)), "depth": (torch.float32, (VN,)), "rect": (torch.int16, (VN, 4)),
            "count": (torch.int32, (VN,)), "value": (torch.int32, (cap,)),
            "range": (torch.int32, (self.V * self.range_stride, 2)), "tfinal": (torch.float32, (P,)),
            "last": (torch.int32, (P,)), "grad2d": (torch.float32, (VN, 8)),
            "order": (torch.int32, (self.V * self.layout.tiles_per_view,)),
        }
        dtype, shape = spec[name]
        off = getattr(self.layout, name)
        nbytes = math.prod(shape) * torch.empty((), dtype=dtype).element_size()
        return self.workspace[off:off + nbytes].view(dtype).view(shape)


class Renderer:
    """Renders a fixed list of views; grows its pair capacity on demand (outside graphs)."""

    def __init__(self, views, cfg: FrameConfig | None = None, pair_capacity: int | None = None,
                 check_capacity: bool = True):
        self.views = list(views)
        self.cfg = cfg or FrameConfig()
        self.pair_capacity = pair_capacity
        self.check_capacity = check_capacity
        self.frame: Frame | None = None

    def _frame(self, n: int, device) -> Frame:
        if self.frame is None or self.frame.n != n:
            cap = self.pair_capacity or max(1 << 16, 8 * n * len(self.views))
            self.frame = Frame(n, self.views, self.cfg, cap, device)
        return self.frame

    def forward(self, mean, scale, quat, opacity, intensity, n_contrib: torch.Tensor | None = None) -> torch.Tensor:
        n = intensity.shape[0]
        f = self._frame(n, intensity.device)
        f.project(mean, scale, quat, opacity, intensity)
        f.bin_sort()
        if self.check_capacity:
            st = f.status()
            if st.code == B.XG_ERR_CAPACITY:
                self.pair_capacity = int(st.pairs * 1.25) + 1024
                self.frame = None
                f = self._frame(n, intensity.device)
                f.project(mean, scale, quat, opacity, intensity)
                f.bin_sort()
                st = f.status()
            if st.code != B.XG_OK:
                raise B.XgError(st.code, "xg_bin_sort")
        image = torch.empty((f.V, f.H, f.W), dtype=torch.float32, device=intensity.device)
        f.render_fwd(image, n_contrib)
        return image

    def backward(self, gaussians: tuple, grad_image: torch.Tensor) -> tuple:
        grads = tuple(torch.empty_like(t) for t in gaussians)
        self.frame.render_bwd(gaussians, grad_image.contiguous(), grads)
        return grads


class XgRender(torch.autograd.Function):
    """image[V, H, W] = F_DRR(views, Gaussians) (Eq. 5); backward through xg_render_bwd.

    The renderer's frame keeps the sorted lists, tfinal and last of the latest forward
    call; backward must follow its own forward before the next forward on the same renderer.
    """

    @staticmethod
    def forward(ctx, renderer: Renderer, mean, scale, quat, opacity, intensity):
        ts = tuple(t.detach().contiguous() for t in (mean, scale, quat, opacity, intensity))
        image = renderer.forward(*ts)
        ctx.renderer = renderer
        ctx.save_for_backward(*ts)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        grads = ctx.renderer.backward(ctx.saved_tensors, grad_image)
        return (None, *grads)


def render(renderer: Renderer, mean, scale, quat, opacity, intensity) -> torch.Tensor:
    return XgRender.apply(renderer, mean, scale, quat, opacity, intensity)


def loss_l1_into(image: torch.Tensor, target: torch.Tensor, grad: torch.Tensor, loss: torch.Tensor,
                 scale: float | None = None, stream=None) -> None:
    """loss[0] = scale * sum|image - target|, grad = scale * sign(image - target) (one kernel)."""
    for t in (image, target, grad):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.shape != image.shape:
            raise ValueError("image, target and grad must be contiguous CUDA float32 tensors of one shape")
    if loss.dtype != torch.float32 or not loss.is_cuda or loss.numel() < 1:
        raise ValueError("loss must be a CUDA float32 tensor")
    count = image.numel()
    B.xg_loss_l1(image.data_ptr(), target.data_ptr(), count, float(scale if scale is not None else 1.0 / count),
                 grad.data_ptr(), loss.data_ptr(), _stream_handle(stream))


class L1Loss(torch.autograd.Function):
    """Mean absolute error (the L1 term of Eq. 11) with its gradient formed in the same kernel."""

    @staticmethod
    def forward(ctx, image, target):
        image = image.contiguous()
        target = target.detach().contiguous()
        grad = torch.empty_like(image)
        loss = torch.empty(1, dtype=torch.float32, device=image.device)
        loss_l1_into(image, target, grad, loss)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None
