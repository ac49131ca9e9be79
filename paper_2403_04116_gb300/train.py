"""Training of the radiative Gaussian model on cone-beam projections (Sec. 3, Eq. 11; the
optimiser settings of Sec. 4.1), every step replayed from a CUDA graph.

A step takes one group of views (8 by default) and runs, all in libxg.so:
activate (exp, sigmoid, RIRF) -> project -> bin + sort -> composite -> (1 - gamma) L1 +
gamma (1 - SSIM) -> composite backward -> activation backward -> Adam.  Views are split
into fixed groups, one frame and one captured graph per group, replayed in turn.

    python -m paper_2403_04116_gb300.train [--steps 20000] [--gaussians 200000] ...

prints one JSON line: wall time, steps/s, training loss, held-out PSNR before and after.
``--densify`` turns on adaptive density control (clone / split / prune and the opacity
reset, by the published rules of 3D Gaussian splatting, which the paper adopts); without
it the number of Gaussians stays fixed.  ``--init acui`` starts from the ACUI grid of Eq. 13 (xg_acui_points) instead
of cuboid-uniform Gaussians; ``--noise 0.03`` adds the paper's 3 % projection noise to the
training targets (held-out PSNR is taken against the noise-free projections).
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B
from . import synth
from .batch import size_pairs
from .render import Frame, FrameConfig, _stream_handle

NAMES = ("mean", "log_scale", "quat", "opacity_logit", "features")


@dataclass
class TrainConfig:
    n_features: int = 16            # N_f (Sec. 4.4: 16 is on par with 32)
    gamma: float = 0.2              # Eq. 11
    views_per_step: int = 8
    lr_position: float = 1.9e-4     # times position_scale, decaying exponentially to lr_position_final
    lr_position_final: float = 1.9e-6
    position_scale: float = 1.0     # scene extent in mm
    lr_feature: float = 2e-3
    lr_opacity: float = 8e-3
    lr_scale: float = 5e-3
    lr_rotation: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    decay_steps: int = 20000
    # adaptive density control (3D Gaussian splatting's published defaults; readings for
    # X-ray: gradients of the projected centre in pixels are taken per view, scaled to
    # normalised device units (W / 2) and to a loss averaged over one view)
    densify: bool = False
    densify_from: int = 500
    densify_until: int = 15000
    densify_interval: int = 100
    opacity_reset_interval: int = 3000
    grad_thresh: float = 2e-4
    percent_dense: float = 0.01     # clone at or below, split above this fraction of the scene side
    min_opacity: float = 0.005
    max_size_fraction: float = 0.1  # prune Gaussians larger than this fraction of the scene side
    reset_opacity: float = 0.01
    seed: int = 0


def raw_from_activated(g: dict, n_features: int, gen: np.random.Generator) -> dict:
    """Raw parameters whose activations reproduce the given Gaussians (lambda = 1):
    log of the scales, logit of the opacities, features summing to logit(intensity)."""
    inten = np.clip(g["intensity"].astype(np.float64), 1e-4, 1 - 1e-4)
    op = np.clip(g["opacity"].astype(np.float64), 1e-6, 1 - 1e-6)
    z = np.log(inten / (1 - inten))
    noise = gen.normal(0, 0.01, size=(n_features, inten.size))
    noise -= noise.mean(axis=0, keepdims=True)
    return {"mean": g["mean"].astype(np.float32), "log_scale": np.log(g["scale"]).astype(np.float32),
            "quat": g["quat"].astype(np.float32), "opacity_logit": np.log(op / (1 - op)).astype(np.float32),
            "features": (z / n_features + noise).astype(np.float32)}


def acui_raw(side_mm: float, grid: int, interval: float, n_features: int, device="cuda") -> dict:
    """Raw parameters of ACUI's initial Gaussians: centres on the grid of Eq. 13 over a cube
    of side ``side_mm`` divided into ``grid``^3 voxels (generated on the device).  The paper
    sets only the centres; the rest follows the 3DGS lineage's defaults (a reading): an
    isotropic scale equal to the grid spacing (the distance to the nearest neighbours), the
    identity rotation, opacity 0.1, and zero features (intensity 1/2 with lambda = 1)."""
    size = (side_mm, side_mm, side_mm)
    dims = (grid, grid, grid)
    n = B.xg_acui_count(size, dims, interval)
    if n == 0:
        raise ValueError("invalid ACUI grid")
    mean = torch.empty(3, n, device=device)
    B.xg_acui_points(size, dims, interval, mean.data_ptr(), n, _stream_handle())
    h = side_mm * interval / grid
    quat = np.zeros((4, n), np.float32)
    quat[0] = 1.0
    return {"mean": mean.cpu().numpy(), "log_scale": np.full((3, n), math.log(h), np.float32), "quat": quat,
            "opacity_logit": np.full(n, math.log(0.1 / 0.9), np.float32),
            "features": np.zeros((n_features, n), np.float32)}


class Trainer:
    def __init__(self, raw: dict, views, targets: torch.Tensor, cfg: TrainConfig, frame_cfg: FrameConfig,
                 device="cuda", capacity_margin: float = 1.6):
        self.cfg = cfg
        self.frame_cfg = frame_cfg
        self.device = torch.device(device)
        self.p = {k: torch.from_numpy(np.ascontiguousarray(raw[k])).to(self.device) for k in NAMES}
        self.n = self.p["mean"].shape[1]
        self.nf = self.p["features"].shape[0]
        self.lam = torch.ones(self.nf, device=self.device)
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        n = self.n
        self.act = {"scale": torch.empty(3, n, device=self.device), "opacity": torch.empty(n, device=self.device),
                    "intensity": torch.empty(n, device=self.device)}
        self.g_act = {"scale": torch.empty(3, n, device=self.device), "opacity": torch.empty(n, device=self.device),
                      "intensity": torch.empty(n, device=self.device)}
        self.step_count = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.loss = torch.zeros(3, device=self.device)
        k = cfg.views_per_step
        self.groups = [list(range(i, min(i + k, len(views)))) for i in range(0, len(views), k)]
        self.views = list(views)
        self.targets = targets
        self.capacity_margin = capacity_margin
        self.iteration = 0
        self.gen = np.random.default_rng(cfg.seed)
        self.accum = torch.zeros(n, device=self.device)
        self.denom = torch.zeros(n, dtype=torch.int32, device=self.device)
        self.dens_ws = torch.empty(B.xg_densify_workspace_bytes() // 4 + 4, dtype=torch.int32, device=self.device)
        self.frames, self.images, self.grad_images, self.loss_ws, self.graphs = [], [], [], [], []
        self._raw = self._raw_struct()
        self._groups = self._adam_groups()
        self._build()

    # ---- plumbing ---------------------------------------------------------------------
    def _raw_struct(self) -> B.XgRawGaussians:
        return B.XgRawGaussians(self.p["log_scale"].data_ptr(), self.p["opacity_logit"].data_ptr(),
                                self.p["features"].data_ptr(), self.lam.data_ptr(), self.nf, 0, self.n)

    def _adam_groups(self) -> list:
        c = self.cfg
        lrs = {"mean": (c.lr_position * c.position_scale, c.lr_position_final * c.position_scale, c.decay_steps),
               "log_scale": (c.lr_scale, 0.0, 0), "quat": (c.lr_rotation, 0.0, 0),
               "opacity_logit": (c.lr_opacity, 0.0, 0), "features": (c.lr_feature, 0.0, 0)}
        return [B.XgAdamGroup(self.p[k].data_ptr(), self.g[k].data_ptr(), self.m[k].data_ptr(), self.v[k].data_ptr(),
                              self.p[k].numel(), lr, lr_f, ds, 0) for k, (lr, lr_f, ds) in lrs.items()]

    def _activated(self) -> tuple:
        return (self.p["mean"], self.act["scale"], self.p["quat"], self.act["opacity"], self.act["intensity"])

    def _param_set(self, d: dict) -> B.XgParamSet:
        return B.XgParamSet(d["mean"].data_ptr(), d["log_scale"].data_ptr(), d["quat"].data_ptr(),
                            d["opacity_logit"].data_ptr(), d["features"].data_ptr(), self.nf, 0, d["mean"].shape[1])

    def _build(self) -> None:
        s = _stream_handle()
        self.frames, self.images, self.grad_images, self.loss_ws = [], [], [], []
        B.xg_activate(self._raw, self.act["scale"].data_ptr(), self.act["opacity"].data_ptr(),
                      self.act["intensity"].data_ptr(), s)
        for idx in self.groups:
            vs = [self.views[i] for i in idx]
            cap = int(size_pairs(self.n, vs, self.frame_cfg, self._activated(), margin=self.capacity_margin))
            f = Frame(self.n, vs, self.frame_cfg, cap, self.device)
            H, W = f.H, f.W
            self.frames.append(f)
            self.images.append(torch.empty(len(vs), H, W, device=self.device))
            self.grad_images.append(torch.empty(len(vs), H, W, device=self.device))
            nb = B.xg_loss_workspace_bytes(len(vs), W, H)
            self.loss_ws.append(torch.empty(nb // 4 + 4, dtype=torch.float32, device=self.device))
        self.target_groups = [self.targets[idx[0]:idx[-1] + 1].contiguous() for idx in self.groups]
        self.graphs = [None] * len(self.groups)

    def _step_calls(self, gi: int) -> None:
        s = _stream_handle()
        f, img, gimg = self.frames[gi], self.images[gi], self.grad_images[gi]
        tgt, ws = self.target_groups[gi], self.loss_ws[gi]
        B.xg_activate(self._raw, self.act["scale"].data_ptr(), self.act["opacity"].data_ptr(),
                      self.act["intensity"].data_ptr(), s)
        f.project(*self._activated())
        f.bin_sort()
        f.render_fwd(img)
        B.xg_loss_l1_ssim(img.data_ptr(), tgt.data_ptr(), f.V, f.W, f.H, self.cfg.gamma, gimg.data_ptr(),
                          self.loss.data_ptr(), ws.data_ptr(), ws.numel() * 4, s)
        f.render_bwd(self._activated(), gimg, (self.g["mean"], self.g_act["scale"], self.g["quat"],
                                               self.g_act["opacity"], self.g_act["intensity"]))
        B.xg_activate_bwd(self._raw, self.g_act["scale"].data_ptr(), self.g_act["opacity"].data_ptr(),
                          self.g_act["intensity"].data_ptr(), self.g["log_scale"].data_ptr(),
                          self.g["opacity_logit"].data_ptr(), self.g["features"].data_ptr(), s)
        if self.cfg.densify:
            # |dL/du| per visible view, in normalised device units for a one-view mean loss
            B.xg_densify_stats(f.handle, float(f.V * f.W / 2), self.accum.data_ptr(), self.denom.data_ptr(), s)
        B.xg_adam_step(self._groups, self.step_count.data_ptr(), self.cfg.beta1, self.cfg.beta2, self.cfg.eps, s)

    def _capture_group(self, gi: int) -> None:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._step_calls(gi)
        self.graphs[gi] = g

    def capture(self) -> None:
        """Record one CUDA graph per view group that has none (recording runs nothing)."""
        for gi in range(len(self.groups)):
            if self.graphs[gi] is None:
                self._capture_group(gi)

    def check_capacity(self) -> bool:
        """True when every frame's pairs fitted (synchronises); frames that overflowed are
        rebuilt with more room and their graphs dropped."""
        ok = True
        for gi, f in enumerate(self.frames):
            st = f.status()
            if st.code == B.XG_ERR_CAPACITY:
                ok = False
                self.frames[gi] = Frame(self.n, f.views, self.frame_cfg, int(st.pairs * self.capacity_margin),
                                        self.device)
                self.graphs[gi] = None
            elif st.code != B.XG_OK:
                raise B.XgError(st.code, "training step")
        return ok

    def _resize(self, n: int) -> None:
        """Per-Gaussian work buffers for n Gaussians; frames and graphs are rebuilt."""
        self.n = n
        dev = self.device
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.act = {"scale": torch.empty(3, n, device=dev), "opacity": torch.empty(n, device=dev),
                    "intensity": torch.empty(n, device=dev)}
        self.g_act = {"scale": torch.empty(3, n, device=dev), "opacity": torch.empty(n, device=dev),
                      "intensity": torch.empty(n, device=dev)}
        self.accum = torch.zeros(n, device=dev)
        self.denom = torch.zeros(n, dtype=torch.int32, device=dev)
        self._raw = self._raw_struct()
        self._groups = self._adam_groups()
        self._build()

    def densify(self) -> int:
        """One densify-and-prune round (synchronises once to read the new count); returns N."""
        c, side = self.cfg, self.cfg.position_scale
        rules = B.XgDensityRules(c.grad_thresh, math.log(c.percent_dense * side),
                                 math.log(c.min_opacity / (1.0 - c.min_opacity)), math.log(c.max_size_fraction * side))
        s = _stream_handle()
        offsets = torch.empty(self.n + 1, dtype=torch.int32, device=self.device)
        B.xg_densify_plan(self._param_set(self.p), self.accum.data_ptr(), self.denom.data_ptr(), rules,
                          offsets.data_ptr(), self.dens_ws.data_ptr(), s)
        n_new = int(offsets[self.n].item()) & 0xFFFFFFFF
        if n_new == 0:
            raise RuntimeError("density control pruned every Gaussian")
        shapes = {"mean": (3,), "log_scale": (3,), "quat": (4,), "opacity_logit": (), "features": (self.nf,)}
        new = [{k: torch.empty(*shp, n_new, device=self.device) for k, shp in shapes.items()} for _ in range(3)]
        normals = torch.from_numpy(self.gen.standard_normal((2, 3, self.n)).astype(np.float32)).to(self.device)
        B.xg_densify_apply(self._param_set(self.p), self._param_set(self.m), self._param_set(self.v),
                           self.accum.data_ptr(), self.denom.data_ptr(), rules, offsets.data_ptr(), normals.data_ptr(),
                           self._param_set(new[0]), self._param_set(new[1]), self._param_set(new[2]), s)
        self.p, self.m, self.v = new
        self._resize(n_new)
        return n_new

    def reset_opacity(self) -> None:
        c = self.cfg
        B.xg_opacity_reset(self.p["opacity_logit"].data_ptr(), self.m["opacity_logit"].data_ptr(),
                           self.v["opacity_logit"].data_ptr(), self.n,
                           math.log(c.reset_opacity / (1.0 - c.reset_opacity)), _stream_handle())

    # ---- checkpoint / resume ------------------------------------------------------------
    def save(self, path: str) -> None:
        """Parameters, Adam moments and step, the iteration count, the density statistics
        and the random state: everything a resumed run continues from (synchronises)."""
        torch.save({"p": self.p, "m": self.m, "v": self.v, "step_count": self.step_count,
                    "iteration": self.iteration, "accum": self.accum, "denom": self.denom,
                    "rng": self.gen.bit_generator.state}, path)

    def load(self, path: str) -> None:
        """Restore a checkpoint written by save(); its N may differ from the current one."""
        ck = torch.load(path, map_location=self.device)
        self.p = {k: ck["p"][k].contiguous() for k in NAMES}
        self.m = {k: ck["m"][k].contiguous() for k in NAMES}
        self.v = {k: ck["v"][k].contiguous() for k in NAMES}
        self.step_count.copy_(ck["step_count"])
        self.iteration = int(ck["iteration"])
        self.gen.bit_generator.state = ck["rng"]
        self._resize(self.p["mean"].shape[1])
        self.accum.copy_(ck["accum"])
        self.denom.copy_(ck["denom"])

    # ---- public -------------------------------------------------------------------------
    def step(self, t: int) -> None:
        """One training step on view group t mod groups: replayed from its graph, or run as
        launches and then recorded (after a rebuild the next visit records it again)."""
        gi = t % len(self.groups)
        if self.graphs[gi] is None:
            self._step_calls(gi)
            self._capture_group(gi)
        else:
            self.graphs[gi].replay()

    def train(self, steps: int, check_every: int = 500) -> None:
        c = self.cfg
        for t in range(steps):
            self.step(t)
            self.iteration += 1
            it = self.iteration
            changed = False
            if c.densify and it < c.densify_until:
                if it >= c.densify_from and it % c.densify_interval == 0:
                    self.densify()
                    changed = True
                if it % c.opacity_reset_interval == 0:
                    self.reset_opacity()
            if check_every and it % check_every == 0 and not changed:
                self.check_capacity()  # frames that overflowed are rebuilt; their graphs re-recorded

    @torch.no_grad()
    def render(self, views) -> torch.Tensor:
        s = _stream_handle()
        B.xg_activate(self._raw, self.act["scale"].data_ptr(), self.act["opacity"].data_ptr(),
                      self.act["intensity"].data_ptr(), s)
        out = []
        for i in range(0, len(views), self.cfg.views_per_step):
            vs = views[i:i + self.cfg.views_per_step]
            cap = size_pairs(self.n, vs, self.frame_cfg, self._activated(), margin=1.1)
            f = Frame(self.n, vs, self.frame_cfg, cap, self.device)
            img = torch.empty(len(vs), f.H, f.W, device=self.device)
            f.project(*self._activated())
            f.bin_sort()
            f.render_fwd(img)
            out.append(img)
        return torch.cat(out)

    def psnr(self, views, targets: torch.Tensor) -> np.ndarray:
        img = self.render(views)
        out = torch.empty(len(views), device=self.device)
        B.xg_psnr(img.data_ptr(), targets.data_ptr(), len(views), img[0].numel(), out.data_ptr(), _stream_handle())
        return out.cpu().numpy()


def config3(n: int, W: int, seed_id: int = 3, span_rad: float = math.pi):
    """Scan of the paper's protocol (Sec. 4.1): 100 projections over 0-180 degrees (or
    another span), the even ones for training, the odd ones held out; cuboid-uniform
    initial Gaussians."""
    side = synth.scene_side_mm(W)
    views = synth.circular_views(100, W, W, span_rad=span_rad)
    ph = synth.ellipsoid_phantom(10, side, synth.rng(seed_id, 1))
    targets = synth.phantom_targets(ph, views)
    g = synth.gaussians(n, side, synth.rng(seed_id, 0))
    return side, views[0::2], targets[0::2], views[1::2], targets[1::2], g


def ct_report(trainer: "Trainer", side: float, W: int, n: int, seed_id: int = 3, span_rad: float = math.pi) -> dict:
    """The paper's downstream use (Table 2), on the synthetic phantom: FDK volumes (n^3, the
    scene cube) from 360 views rendered by the trained Gaussians, from 360 exact projections
    and from 50 exact projections (sparse view), each scored by 3-D PSNR against the
    phantom's density (in the units of the normalised projections)."""
    from .ct import fdk, psnr3d
    ph = synth.ellipsoid_phantom(10, side, synth.rng(seed_id, 1))
    scan = synth.circular_views(100, W, W, span_rad=span_rad)  # the training scan's normalisation
    norm = max(float(synth.phantom_line_integrals(ph, v).max()) for v in scan)
    vox = side / n
    truth = synth.phantom_density(ph, (n, n, n), vox) / norm
    full = synth.circular_views(360, W, W)
    rendered = trainer.render(full)
    fdk(rendered, full, (n, n, n), vox)  # warm-up
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    vol = fdk(rendered, full, (n, n, n), vox)
    t1.record()
    torch.cuda.synchronize()
    out = {"volume": [n, n, n], "voxel_mm": vox, "fdk_ms_360_views": t0.elapsed_time(t1),
           "psnr_rendered_360": psnr3d(vol.cpu().numpy(), truth)}
    for name, k in (("psnr_exact_360", 360), ("psnr_exact_50", 50)):
        vs = synth.circular_views(k, W, W)
        proj = np.stack([synth.phantom_line_integrals(ph, v) for v in vs]) / norm
        vol = fdk(torch.from_numpy(proj.astype(np.float32)).to(rendered.device), vs, (n, n, n), vox)
        out[name] = psnr3d(vol.cpu().numpy(), truth)
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--gaussians", type=int, default=200_000)
    ap.add_argument("--detector", type=int, default=512)
    ap.add_argument("--views-per-step", type=int, default=8)
    ap.add_argument("--tile", default="16x16:64:2")
    ap.add_argument("--init", choices=["uniform", "acui"], default="uniform")
    ap.add_argument("--acui-grid", type=int, default=256, help="voxels per axis M of Eq. 13")
    ap.add_argument("--acui-interval", type=float, default=8.0, help="sampling interval d of Eq. 13")
    ap.add_argument("--noise", type=float, default=0.0, help="projection noise level (0.03 in the paper)")
    ap.add_argument("--densify", action="store_true", help="adaptive density control (clone / split / prune)")
    ap.add_argument("--span", type=float, default=180.0, help="degrees covered by the 100 scan views (paper: 180)")
    ap.add_argument("--fdk", type=int, default=0, help="after training, reconstruct an N^3 volume by FDK from 360 "
                                                          "rendered views and report its 3-D PSNR")
    args = ap.parse_args()
    tw_th, b, p = args.tile.split(":")
    tw, th = (int(x) for x in tw_th.split("x"))
    fcfg = FrameConfig(tw, th, batch=int(b), pixels_per_thread=int(p))
    span = math.radians(args.span)
    side, tr_v, tr_t, te_v, te_t, g = config3(args.gaussians, args.detector, span_rad=span)
    cfg = TrainConfig(views_per_step=args.views_per_step, position_scale=side, decay_steps=args.steps,
                      densify=args.densify)
    B.lib(build_if_missing=True)
    if args.init == "acui":
        raw = acui_raw(side, args.acui_grid, args.acui_interval, cfg.n_features)
    else:
        raw = raw_from_activated(g, cfg.n_features, synth.rng(3, 2))
    if args.noise > 0:
        tr_t = synth.projection_noise(tr_t, args.noise, synth.rng(3, 3)).astype(np.float32)
    dev = torch.device("cuda")
    tr_t, te_t = torch.from_numpy(tr_t).to(dev), torch.from_numpy(te_t).to(dev)
    trainer = Trainer(raw, tr_v, tr_t, cfg, fcfg)
    n_start = trainer.n
    psnr0 = trainer.psnr(te_v, te_t)
    trainer.capture()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trainer.train(args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    loss = trainer.loss.cpu().numpy()
    psnr1 = trainer.psnr(te_v, te_t)
    ct = ct_report(trainer, side, args.detector, args.fdk, span_rad=span) if args.fdk else None
    print(json.dumps({"workload": "config3", "span_deg": args.span, "init": args.init, "noise": args.noise,
                      "densify": args.densify,
                      "gaussians_start": n_start, "gaussians": trainer.n, "detector": args.detector,
                      "train_views": len(tr_v), "test_views": len(te_v), "views_per_step": args.views_per_step,
                      "steps": args.steps, "wall_s": wall, "steps_per_s": args.steps / wall,
                      "last_loss": float(loss[0]), "last_l1": float(loss[1]), "last_ssim": float(loss[2]),
                      "heldout_psnr_before": float(psnr0.mean()), "heldout_psnr_after": float(psnr1.mean()),
                      "tile": args.tile, "ct": ct}), flush=True)


if __name__ == "__main__":
    main()
