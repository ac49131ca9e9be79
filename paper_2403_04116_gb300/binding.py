"""ctypes binding of ``include/xg.h``: same names, argument marshalling only.

Every computation happens in ``libxg.so``.  If the library has not been built, loading
fails loudly: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

XG_OK = 0
XG_ERR_INVALID_ARG = 1
XG_ERR_CAPACITY = 2
XG_ERR_CUDA = 3
XG_ERR_WORKSPACE = 4
XG_ERR_CHECK = 5

# Every symbol include/xg.h declares.
EXPORTS = ("xg_workspace_bytes", "xg_frame_create", "xg_frame_destroy", "xg_frame_select_views", "xg_fdk_workspace_bytes", "xg_fdk", "xg_densify_stats", "xg_densify_workspace_bytes",
           "xg_densify_plan", "xg_densify_apply", "xg_opacity_reset", "xg_acui_count", "xg_acui_points", "xg_frame_copy_status", "xg_project",
           "xg_bin_sort",
           "xg_render_fwd", "xg_render_bwd", "xg_frame_read_status", "xg_frame_layout", "xg_exp_check", "xg_loss_l1",
           "xg_frame_set_timing", "xg_frame_read_timing", "xg_activate", "xg_activate_bwd",
           "xg_loss_workspace_bytes", "xg_loss_l1_ssim", "xg_adam_step", "xg_psnr", "xg_sort_pairs_noalloc", "xg_sort_pairs_noalloc_status", "xg_fp32_peak",
           "xg_status_str")
XG_ADAM_MAX_GROUPS = 8
XG_NOALLOC_MAX_PAIRS = 1 << 20


class XgView(ctypes.Structure):
    _fields_ = [("sod_mm", ctypes.c_double), ("sdd_mm", ctypes.c_double), ("pitch_u_mm", ctypes.c_double),
                ("pitch_v_mm", ctypes.c_double), ("angle_rad", ctypes.c_double), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class XgGaussians(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("intensity", ctypes.c_void_p), ("n", ctypes.c_int64)]


class XgGrads(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("intensity", ctypes.c_void_p)]


class XgConfig(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("near_mm", ctypes.c_float),
                ("batch", ctypes.c_int32), ("pair_capacity", ctypes.c_int64), ("pixels_per_thread", ctypes.c_int32),
                ("views_per_pass", ctypes.c_int32), ("persistent", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class XgDeviceStatus(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("reserved", ctypes.c_int32), ("pairs", ctypes.c_int64),
                ("nonfinite", ctypes.c_int64), ("fwd_evaluated", ctypes.c_int64), ("fwd_contrib", ctypes.c_int64),
                ("bwd_evaluated", ctypes.c_int64), ("bwd_contrib", ctypes.c_int64)]


class XgKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class XgLayout(ctypes.Structure):
    _fields_ = [(name, ctypes.c_size_t) for name in
                ("status", "cameras", "records", "depth", "rect", "count", "value", "range", "tfinal", "last",
                 "grad2d")] + [
        ("tiles_per_view", ctypes.c_int64), ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32),
        ("sort_passes", ctypes.c_int32), ("range_stride", ctypes.c_int32), ("order", ctypes.c_size_t)]


class XgRawGaussians(ctypes.Structure):
    _fields_ = [("log_scale", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p), ("features", ctypes.c_void_p),
                ("lambda_", ctypes.c_void_p), ("n_features", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n", ctypes.c_int64)]


class XgAdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("count", ctypes.c_int64), ("lr", ctypes.c_float),
                ("lr_final", ctypes.c_float), ("decay_steps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class XgParamSet(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("log_scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("opacity_logit", ctypes.c_void_p), ("features", ctypes.c_void_p), ("n_features", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("n", ctypes.c_int64)]


class XgDensityRules(ctypes.Structure):
    _fields_ = [("grad_thresh", ctypes.c_float), ("size_log_thresh", ctypes.c_float),
                ("prune_logit", ctypes.c_float), ("max_log_size", ctypes.c_float)]


class XgVolume(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("voxel_mm", ctypes.c_double)]


class XgError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {xg_status_str(code)} ({code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load libxg.so (raises if it is absent and ``build_if_missing`` is false)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with paper_2403_04116_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.xg_workspace_bytes.argtypes = [ctypes.POINTER(XgConfig), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32]
    L.xg_workspace_bytes.restype = ctypes.c_size_t
    L.xg_frame_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(XgConfig), ctypes.c_int64,
                                  ctypes.POINTER(XgView), ctypes.c_int32, P, ctypes.c_size_t, P]
    L.xg_frame_create.restype = ctypes.c_int
    L.xg_acui_count.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), ctypes.c_double]
    L.xg_acui_count.restype = ctypes.c_int64
    L.xg_acui_points.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), ctypes.c_double, P,
                                 ctypes.c_int64, P]
    L.xg_acui_points.restype = ctypes.c_int
    L.xg_frame_copy_status.argtypes = [P, P, P]
    L.xg_frame_copy_status.restype = ctypes.c_int
    L.xg_frame_select_views.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    L.xg_frame_select_views.restype = ctypes.c_int
    L.xg_frame_destroy.argtypes = [P]
    L.xg_frame_destroy.restype = None
    L.xg_project.argtypes = [P, ctypes.POINTER(XgGaussians), P]
    L.xg_project.restype = ctypes.c_int
    L.xg_bin_sort.argtypes = [P, P]
    L.xg_bin_sort.restype = ctypes.c_int
    L.xg_render_fwd.argtypes = [P, P, P, P]
    L.xg_render_fwd.restype = ctypes.c_int
    L.xg_render_bwd.argtypes = [P, ctypes.POINTER(XgGaussians), P, ctypes.POINTER(XgGrads), P]
    L.xg_render_bwd.restype = ctypes.c_int
    L.xg_frame_read_status.argtypes = [P, ctypes.POINTER(XgDeviceStatus), P]
    L.xg_frame_read_status.restype = ctypes.c_int
    L.xg_frame_layout.argtypes = [P, ctypes.POINTER(XgLayout)]
    L.xg_frame_layout.restype = ctypes.c_int
    L.xg_loss_l1.argtypes = [P, P, ctypes.c_int64, ctypes.c_float, P, P, P]
    L.xg_loss_l1.restype = ctypes.c_int
    L.xg_exp_check.argtypes = [P, P, P, ctypes.c_int64, P]
    L.xg_exp_check.restype = ctypes.c_int
    L.xg_frame_set_timing.argtypes = [P, ctypes.c_int32]
    L.xg_frame_set_timing.restype = ctypes.c_int
    L.xg_frame_read_timing.argtypes = [P, ctypes.POINTER(XgKernelTime), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)]
    L.xg_frame_read_timing.restype = ctypes.c_int
    L.xg_activate.argtypes = [ctypes.POINTER(XgRawGaussians), P, P, P, P]
    L.xg_activate.restype = ctypes.c_int
    L.xg_activate_bwd.argtypes = [ctypes.POINTER(XgRawGaussians), P, P, P, P, P, P, P]
    L.xg_activate_bwd.restype = ctypes.c_int
    L.xg_loss_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.xg_loss_workspace_bytes.restype = ctypes.c_size_t
    L.xg_loss_l1_ssim.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, P, P, P,
                                  ctypes.c_size_t, P]
    L.xg_loss_l1_ssim.restype = ctypes.c_int
    L.xg_adam_step.argtypes = [ctypes.POINTER(XgAdamGroup), ctypes.c_int32, P, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, P]
    L.xg_adam_step.restype = ctypes.c_int
    L.xg_fdk_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.xg_fdk_workspace_bytes.restype = ctypes.c_size_t
    L.xg_fdk.argtypes = [ctypes.POINTER(XgView), ctypes.c_int32, P, ctypes.POINTER(XgVolume), P, P, ctypes.c_size_t, P]
    L.xg_fdk.restype = ctypes.c_int
    PS = ctypes.POINTER(XgParamSet)
    L.xg_densify_stats.argtypes = [P, ctypes.c_float, P, P, P]
    L.xg_densify_stats.restype = ctypes.c_int
    L.xg_densify_workspace_bytes.argtypes = []
    L.xg_densify_workspace_bytes.restype = ctypes.c_size_t
    L.xg_densify_plan.argtypes = [PS, P, P, ctypes.POINTER(XgDensityRules), P, P, P]
    L.xg_densify_plan.restype = ctypes.c_int
    L.xg_densify_apply.argtypes = [PS, PS, PS, P, P, ctypes.POINTER(XgDensityRules), P, P, PS, PS, PS, P]
    L.xg_densify_apply.restype = ctypes.c_int
    L.xg_opacity_reset.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_float, P]
    L.xg_opacity_reset.restype = ctypes.c_int
    L.xg_psnr.argtypes = [P, P, ctypes.c_int32, ctypes.c_int64, P, P]
    L.xg_psnr.restype = ctypes.c_int
    L.xg_sort_pairs_noalloc.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, P, P, P, P]
    L.xg_sort_pairs_noalloc.restype = ctypes.c_int
    L.xg_fp32_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_int64), P]
    L.xg_fp32_peak.restype = ctypes.c_int
    L.xg_sort_pairs_noalloc_status.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    L.xg_sort_pairs_noalloc_status.restype = ctypes.c_int
    L.xg_status_str.argtypes = [ctypes.c_int]
    L.xg_status_str.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(code: int, what: str) -> None:
    if code != XG_OK:
        raise XgError(code, what)


def xg_status_str(code: int) -> str:
    return lib().xg_status_str(code).decode()


def xg_workspace_bytes(cfg: XgConfig, n: int, n_views: int, width: int, height: int) -> int:
    return int(lib().xg_workspace_bytes(ctypes.byref(cfg), n, n_views, width, height))


def xg_frame_create(cfg: XgConfig, n: int, views, workspace: int, workspace_bytes: int, stream: int) -> int:
    arr = (XgView * len(views))(*[XgView(v.sod_mm, v.sdd_mm, v.pitch_u_mm, v.pitch_v_mm, v.angle_rad, v.width,
                                         v.height) for v in views])
    out = ctypes.c_void_p()
    _check(lib().xg_frame_create(ctypes.byref(out), ctypes.byref(cfg), n, arr, len(views), workspace,
                                 workspace_bytes, stream), "xg_frame_create")
    return out.value


def _acui_args(size_mm, grid):
    return (ctypes.c_double * 3)(*[float(x) for x in size_mm]), (ctypes.c_int32 * 3)(*[int(m) for m in grid])


def xg_acui_count(size_mm, grid, interval: float) -> int:
    return int(lib().xg_acui_count(*_acui_args(size_mm, grid), float(interval)))


def xg_acui_points(size_mm, grid, interval: float, mean_ptr: int, capacity: int, stream: int) -> None:
    _check(lib().xg_acui_points(*_acui_args(size_mm, grid), float(interval), mean_ptr, int(capacity), stream),
           "xg_acui_points")


def xg_frame_copy_status(frame: int, out_ptr: int, stream: int) -> None:
    _check(lib().xg_frame_copy_status(frame, out_ptr, stream), "xg_frame_copy_status")


def xg_frame_select_views(frame: int, first_view: int) -> int:
    got = ctypes.c_int32(0)
    _check(lib().xg_frame_select_views(frame, first_view, ctypes.byref(got)), "xg_frame_select_views")
    return got.value


def xg_frame_destroy(frame: int) -> None:
    lib().xg_frame_destroy(frame)


def xg_project(frame: int, g: XgGaussians, stream: int) -> None:
    _check(lib().xg_project(frame, ctypes.byref(g), stream), "xg_project")


def xg_bin_sort(frame: int, stream: int) -> None:
    _check(lib().xg_bin_sort(frame, stream), "xg_bin_sort")


def xg_render_fwd(frame: int, image: int, n_contrib: int | None, stream: int) -> None:
    _check(lib().xg_render_fwd(frame, image, n_contrib, stream), "xg_render_fwd")


def xg_render_bwd(frame: int, g: XgGaussians, grad_image: int, out: XgGrads, stream: int) -> None:
    _check(lib().xg_render_bwd(frame, ctypes.byref(g), grad_image, ctypes.byref(out), stream), "xg_render_bwd")


def xg_frame_read_status(frame: int, stream: int) -> XgDeviceStatus:
    s = XgDeviceStatus()
    _check(lib().xg_frame_read_status(frame, ctypes.byref(s), stream), "xg_frame_read_status")
    return s


def xg_frame_layout(frame: int) -> XgLayout:
    L = XgLayout()
    _check(lib().xg_frame_layout(frame, ctypes.byref(L)), "xg_frame_layout")
    return L


def xg_exp_check(x: int, y_scalar: int, y_packed: int, n: int, stream: int) -> None:
    _check(lib().xg_exp_check(x, y_scalar, y_packed, n, stream), "xg_exp_check")


def xg_loss_l1(image: int, target: int, count: int, scale: float, grad: int, loss: int, stream: int) -> None:
    _check(lib().xg_loss_l1(image, target, count, scale, grad, loss, stream), "xg_loss_l1")


def xg_frame_set_timing(frame: int, enable: bool) -> None:
    _check(lib().xg_frame_set_timing(frame, 1 if enable else 0), "xg_frame_set_timing")


def xg_frame_read_timing(frame: int) -> dict:
    """{kernel name: (launches, total ms)} since the previous read (waits for the events)."""
    out = (XgKernelTime * 32)()
    count = ctypes.c_int32()
    _check(lib().xg_frame_read_timing(frame, out, 32, ctypes.byref(count)), "xg_frame_read_timing")
    return {out[i].name.decode(): (int(out[i].launches), float(out[i].total_ms)) for i in range(count.value)}


def xg_sort_pairs_noalloc(key_tile: int, key_depth: int, value: int, count: int, tile_bits: int,
                          out_key_tile: int, out_key_depth: int, out_value: int, stream: int) -> None:
    _check(lib().xg_sort_pairs_noalloc(key_tile, key_depth, value, count, tile_bits, out_key_tile, out_key_depth,
                                       out_value, stream), "xg_sort_pairs_noalloc")


def xg_fp32_peak(packed: int, iters: int, sink: int, stream: int) -> int:
    """Enqueue one FMA-chain launch; returns the FP32 multiply-adds it performs."""
    ops = ctypes.c_int64(0)
    _check(lib().xg_fp32_peak(packed, iters, sink, ctypes.byref(ops), stream), "xg_fp32_peak")
    return int(ops.value)


def xg_sort_pairs_noalloc_status(stream: int) -> int:
    """Device-side code of the last allocation-free sort on the current device (waits for
    ``stream``): XG_OK or XG_ERR_CHECK."""
    code = ctypes.c_int32(-1)
    _check(lib().xg_sort_pairs_noalloc_status(stream, ctypes.byref(code)), "xg_sort_pairs_noalloc_status")
    return int(code.value)


def xg_activate(raw: XgRawGaussians, scale: int, opacity: int, intensity: int, stream: int) -> None:
    _check(lib().xg_activate(ctypes.byref(raw), scale, opacity, intensity, stream), "xg_activate")


def xg_activate_bwd(raw: XgRawGaussians, g_scale: int, g_opacity: int, g_intensity: int, g_log_scale: int,
                    g_opacity_logit: int, g_features: int, stream: int) -> None:
    _check(lib().xg_activate_bwd(ctypes.byref(raw), g_scale, g_opacity, g_intensity, g_log_scale, g_opacity_logit,
                                 g_features, stream), "xg_activate_bwd")


def xg_loss_workspace_bytes(n_views: int, width: int, height: int) -> int:
    return int(lib().xg_loss_workspace_bytes(n_views, width, height))


def xg_loss_l1_ssim(image: int, target: int, n_views: int, width: int, height: int, gamma: float, grad: int,
                    loss: int, workspace: int, workspace_bytes: int, stream: int) -> None:
    _check(lib().xg_loss_l1_ssim(image, target, n_views, width, height, gamma, grad, loss, workspace,
                                 workspace_bytes, stream), "xg_loss_l1_ssim")


def xg_adam_step(groups, step: int, beta1: float, beta2: float, eps: float, stream: int) -> None:
    arr = (XgAdamGroup * len(groups))(*groups)
    _check(lib().xg_adam_step(arr, len(groups), step, beta1, beta2, eps, stream), "xg_adam_step")


def xg_fdk_workspace_bytes(n_views: int, width: int, height: int) -> int:
    return int(lib().xg_fdk_workspace_bytes(n_views, width, height))


def xg_fdk(views, projections: int, vol: XgVolume, volume: int, workspace: int, nbytes: int, stream: int) -> None:
    arr = (XgView * len(views))(*[XgView(v.sod_mm, v.sdd_mm, v.pitch_u_mm, v.pitch_v_mm, v.angle_rad, v.width,
                                         v.height) for v in views])
    _check(lib().xg_fdk(arr, len(views), projections, ctypes.byref(vol), volume, workspace, nbytes, stream), "xg_fdk")


def xg_densify_stats(frame: int, scale: float, accum: int, denom: int, stream: int) -> None:
    _check(lib().xg_densify_stats(frame, scale, accum, denom, stream), "xg_densify_stats")


def xg_densify_workspace_bytes() -> int:
    return int(lib().xg_densify_workspace_bytes())


def xg_densify_plan(params: XgParamSet, accum: int, denom: int, rules: XgDensityRules, offsets: int, workspace: int,
                    stream: int) -> None:
    _check(lib().xg_densify_plan(ctypes.byref(params), accum, denom, ctypes.byref(rules), offsets, workspace, stream),
           "xg_densify_plan")


def xg_densify_apply(params: XgParamSet, m: XgParamSet, v: XgParamSet, accum: int, denom: int, rules: XgDensityRules,
                     offsets: int, normals: int, out: XgParamSet, out_m: XgParamSet, out_v: XgParamSet,
                     stream: int) -> None:
    _check(lib().xg_densify_apply(ctypes.byref(params), ctypes.byref(m), ctypes.byref(v), accum, denom,
                                  ctypes.byref(rules), offsets, normals, ctypes.byref(out), ctypes.byref(out_m),
                                  ctypes.byref(out_v), stream), "xg_densify_apply")


def xg_opacity_reset(opacity_logit: int, adam_m, adam_v, n: int, reset_logit: float, stream: int) -> None:
    _check(lib().xg_opacity_reset(opacity_logit, adam_m, adam_v, n, reset_logit, stream), "xg_opacity_reset")


def xg_psnr(image: int, target: int, n_views: int, pixels_per_view: int, psnr: int, stream: int) -> None:
    _check(lib().xg_psnr(image, target, n_views, pixels_per_view, psnr, stream), "xg_psnr")
