"""Batched training steps: every view of a scan in one launch per stage, replayed from a
CUDA graph, plus the tile-shape / staging-batch autotuner.

``GraphedStep`` captures project -> bin + sort -> composite -> L1 loss -> backward for all
views of a frame once, then replays it; only tensor contents change between replays (the
Gaussian parameters and the targets are copied into its input buffers).  ``GraphedScan``
renders a scan too large for one pass (hundreds of views of a dense scene) in passes of a
few views through one workspace, every pass recorded in the same graph.  ``PlainSteps``
is the reference form: one frame per view and one launch sequence per view, no graph.
Both run the same kernels, so their images and gradients agree (gradients up to the order
of float atomics).
"""
from __future__ import annotations

import json
import os
import statistics
from dataclasses import asdict, dataclass

import torch

from . import binding as B
from .render import Frame, FrameConfig, loss_l1_into

_NAMES = ("mean", "scale", "quat", "opacity", "intensity")
CANDIDATE_TILES = ((8, 8), (16, 16), (32, 16), (16, 8), (16, 32))
CANDIDATE_BATCHES = (64, 128, 256, 512)
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def size_pairs(n: int, views, cfg: FrameConfig, gaussians: tuple, margin: float = 1.05) -> int:
    """Pair count of one binning pass (synchronises), with a margin, for sizing frames."""
    probe = Frame(n, views, cfg, pair_capacity=1 << 20)
    probe.project(*gaussians)
    probe.bin_sort()
    st = probe.status()
    if st.code not in (B.XG_OK, B.XG_ERR_CAPACITY):
        raise B.XgError(st.code, "xg_bin_sort")
    return int(st.pairs * margin) + 4096


class GraphedStep:
    """Forward + L1 loss + backward of all views, captured in one CUDA graph."""

    def __init__(self, n: int, views, cfg: FrameConfig, pair_capacity: int, device="cuda"):
        self.frame = Frame(n, views, cfg, pair_capacity, device)
        V, H, W = self.frame.V, self.frame.H, self.frame.W
        self.inputs = (torch.zeros(3, n, device=device), torch.ones(3, n, device=device),
                       torch.zeros(4, n, device=device), torch.zeros(n, device=device), torch.zeros(n, device=device))
        self.inputs[2][0] = 1.0
        self.target = torch.zeros(V, H, W, device=device)
        self.image = torch.empty(V, H, W, device=device)
        self.grad_image = torch.empty_like(self.image)
        self.loss = torch.empty(1, device=device)
        self.grads = tuple(torch.empty_like(t) for t in self.inputs)
        self.graph = None

    def _run(self) -> None:
        f = self.frame
        f.project(*self.inputs)
        f.bin_sort()
        f.render_fwd(self.image)
        loss_l1_into(self.image, self.target, self.grad_image, self.loss)
        f.render_bwd(self.inputs, self.grad_image, self.grads)

    def load(self, gaussians: tuple, target: torch.Tensor | None = None) -> None:
        for dst, src in zip(self.inputs, gaussians):
            dst.copy_(src, non_blocking=True)
        if target is not None:
            self.target.copy_(target, non_blocking=True)

    def capture(self) -> None:
        """Warm up on a side stream, then record the step (the frame must not overflow)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._run()
        torch.cuda.current_stream().wait_stream(side)
        st = self.frame.status()
        if st.code != B.XG_OK:
            raise B.XgError(st.code, "graph warm-up")
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._run()

    def replay(self) -> None:
        self.graph.replay()

    def capture_host(self, host_gaussians: tuple, host_target: torch.Tensor, slots: int = 2) -> None:
        """Record the step with its transfers: the Gaussians and the targets copied in from
        these pinned host tensors (the targets on a side stream, overlapped with the forward
        pass and joined before the loss) and the loss copied out to a pinned slot.  ``slots``
        graphs are recorded, identical but for their loss slot, so a loop can enqueue the
        next step before it reads the previous step's loss (``replay_host`` then
        ``loss_of``).  Each replay reads whatever the host tensors hold when its copies run."""
        self.host_losses = [torch.empty(1, dtype=torch.float32).pin_memory() for _ in range(slots)]
        self.host_loss = self.host_losses[0]
        self._host_in = (tuple(host_gaussians), host_target)  # keep the sources alive
        self._host_done = [torch.cuda.Event() for _ in range(slots)]
        copy = torch.cuda.Stream()
        f = self.frame
        self.graphs_host = []
        for k in range(slots):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                main = torch.cuda.current_stream()
                for dst, src in zip(self.inputs, host_gaussians):
                    dst.copy_(src, non_blocking=True)
                copy.wait_stream(main)
                with torch.cuda.stream(copy):
                    self.target.copy_(host_target, non_blocking=True)
                f.project(*self.inputs)
                f.bin_sort()
                f.render_fwd(self.image)
                main.wait_stream(copy)
                loss_l1_into(self.image, self.target, self.grad_image, self.loss)
                f.render_bwd(self.inputs, self.grad_image, self.grads)
                self.host_losses[k].copy_(self.loss, non_blocking=True)
            self.graphs_host.append(g)
        self.graph_host = self.graphs_host[0]

    def replay_host(self, slot: int = 0) -> None:
        """One step from the host inputs, its loss to slot ``slot`` (``host_losses[slot]``,
        valid once the stream reaches it: ``loss_of``)."""
        self.graphs_host[slot].replay()
        self._host_done[slot].record()

    def loss_of(self, slot: int = 0) -> float:
        """Wait for the last step replayed into ``slot`` and return its loss."""
        self._host_done[slot].synchronize()
        return float(self.host_losses[slot][0])


class GraphedScan:
    """Forward projections of every view of a scan, ``views_per_pass`` views at a time,
    all passes captured in one CUDA graph.

    Two frames alternate on two streams, so a pass's binning and sort (latency- and
    memory-bound) overlap the previous pass's compositing (issue-bound).  The device status
    word of each pass (pair count, capacity overflow, work counters) is copied into
    ``pass_status`` inside the graph, so one read after a replay covers them all.
    ``capture_host`` records a second graph that also copies each pass's projections to
    pinned host memory (``host_image``) on a side stream as soon as the pass is done, so
    the copies overlap the following passes.
    """

    def __init__(self, n: int, views, cfg: FrameConfig, pair_capacity: int, views_per_pass: int, device="cuda",
                 overlap: bool = True):
        self.frames = [Frame(n, views, cfg, pair_capacity, device, views_per_pass=views_per_pass)
                       for _ in range(2 if overlap else 1)]
        self.frame = self.frames[0]
        f = self.frame
        self.starts = list(range(0, f.n_scan, f.views_per_pass))
        self.inputs = (torch.zeros(3, n, device=device), torch.ones(3, n, device=device),
                       torch.zeros(4, n, device=device), torch.zeros(n, device=device), torch.zeros(n, device=device))
        self.inputs[2][0] = 1.0
        self.image = torch.empty(f.n_scan, f.H, f.W, device=device)
        self.pass_status = torch.zeros(len(self.starts), 7, dtype=torch.int64, device=device)
        self._streams = [None] + [torch.cuda.Stream() for _ in self.frames[1:]]
        self.graph = None
        self.graph_host = None
        self.host_image = None
        self._copy_stream = None

    def _run(self, to_host: bool = False, serial: bool = False) -> None:
        """Enqueue every pass; ``serial`` keeps them all on the current stream (for
        per-kernel timing without overlap)."""
        main = torch.cuda.current_stream()
        streams = [main] * len(self.frames) if serial else [main] + self._streams[1:]
        for s in streams[1:]:
            if s is not main:
                s.wait_stream(main)
        for i, first in enumerate(self.starts):
            k = i % len(self.frames)
            f, s = self.frames[k], streams[k]
            with torch.cuda.stream(s):
                V = f.select(first)
                f.project(*self.inputs)
                f.bin_sort()
                f.render_fwd(self.image[first:first + V])
                f.copy_status(self.pass_status[i])
                if to_host:
                    done = torch.cuda.Event()
                    done.record(s)
                    self._copy_stream.wait_event(done)
                    with torch.cuda.stream(self._copy_stream):
                        self.host_image[first:first + V].copy_(self.image[first:first + V], non_blocking=True)
        for f in self.frames:
            f.select(0)
        for s in streams[1:]:
            if s is not main:
                main.wait_stream(s)
        if to_host:
            main.wait_stream(self._copy_stream)

    def load(self, gaussians: tuple) -> None:
        for dst, src in zip(self.inputs, gaussians):
            dst.copy_(src, non_blocking=True)

    def statuses(self) -> list:
        """Per-pass (code, pairs, fwd_evaluated, fwd_contrib) of the latest run (synchronises)."""
        out = []
        for row in self.pass_status.cpu().numpy():
            st = B.XgDeviceStatus.from_buffer_copy(row.tobytes())
            out.append((st.code, st.pairs, st.fwd_evaluated, st.fwd_contrib))
        return out

    def max_pairs(self) -> int:
        """Largest pass of one uncaptured run (synchronises); for sizing the capacity."""
        self._run()
        return max(p for _, p, _, _ in self.statuses())

    def capture(self) -> None:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._run()
        torch.cuda.current_stream().wait_stream(side)
        bad = [c for c, _, _, _ in self.statuses() if c != B.XG_OK]
        if bad:
            raise B.XgError(bad[0], "graph warm-up")
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._run()

    def capture_host(self) -> None:
        """Record the scan with the per-pass copies to ``host_image`` (pinned)."""
        if self.host_image is None:
            self.host_image = torch.empty(self.image.shape, dtype=torch.float32).pin_memory()
            self._copy_stream = torch.cuda.Stream()
        self.graph_host = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph_host):
            self._copy_stream.wait_stream(torch.cuda.current_stream())
            self._run(to_host=True)

    def replay(self) -> None:
        self.graph.replay()

    def replay_host(self) -> None:
        """One scan whose projections land in ``host_image`` when the stream reaches its end."""
        self.graph_host.replay()


class PlainSteps:
    """The same step as one frame and one launch sequence per view (no graph)."""

    def __init__(self, n: int, views, cfg: FrameConfig, pair_capacity_per_view: int, device="cuda"):
        self.frames = [Frame(n, [v], cfg, pair_capacity_per_view, device) for v in views]
        H, W = self.frames[0].H, self.frames[0].W
        self.images = [torch.empty(1, H, W, device=device) for _ in views]
        self.grad_images = [torch.empty(1, H, W, device=device) for _ in views]
        self.loss = torch.empty(1, device=device)
        self.view_grads = [None] * len(views)

    def run(self, gaussians: tuple, target: torch.Tensor, grads: tuple) -> None:
        for g in grads:
            g.zero_()
        tmp = tuple(torch.empty_like(g) for g in grads)
        for v, f in enumerate(self.frames):
            f.project(*gaussians)
            f.bin_sort()
            f.render_fwd(self.images[v])
            loss_l1_into(self.images[v], target[v:v + 1], self.grad_images[v], self.loss,
                         scale=1.0 / target.numel())
            f.render_bwd(gaussians, self.grad_images[v], tmp)
            for g, t in zip(grads, tmp):
                g.add_(t)


@dataclass
class TuneResult:
    tile_w: int
    tile_h: int
    batch: int
    pixels_per_thread: int
    ms: float
    pair_capacity: int
    persistent: int = 0

    def config(self) -> FrameConfig:
        return FrameConfig(self.tile_w, self.tile_h, batch=self.batch, pixels_per_thread=self.pixels_per_thread,
                           persistent=self.persistent)


def build_scan(n: int, views, cfg: FrameConfig, views_per_pass: int, gaussians: tuple,
               margin: float = 1.05) -> GraphedScan:
    """A GraphedScan whose pair capacity fits the largest pass of these Gaussians (sized by
    uncaptured runs, which synchronise), loaded with them and captured."""
    cap = size_pairs(n, views[:views_per_pass], cfg, gaussians, margin=1.25)
    while True:
        scan = GraphedScan(n, views, cfg, cap, views_per_pass)
        scan.load(gaussians)
        need = scan.max_pairs()
        if need <= cap:
            break
        cap = int(need * margin) + 4096
        del scan
    scan.capture()
    return scan


def autotune_scan(n: int, views, gaussians: tuple, tiles=((16, 16), (32, 16)), passes=(8, 12, 16, 30),
                  shapes=((64, 2), (128, 2), (64, 1)), reps: int = 3) -> tuple:
    """Tile shape and views per pass, then staging batch and pixels per thread, with the
    fastest replay of the captured scan; returns (FrameConfig, views_per_pass, ms)."""
    def time_scan(cfg, vpp):
        scan = build_scan(n, views, cfg, vpp, gaussians)
        scan.replay()
        times = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            scan.replay()
            e.record()
            torch.cuda.synchronize()
            times.append(s.elapsed_time(e))
        del scan
        torch.cuda.empty_cache()
        return statistics.median(times)

    best = None
    b0, p0 = shapes[0]
    for tw, th in tiles:
        for vpp in passes:
            cfg = FrameConfig(tw, th, batch=b0, pixels_per_thread=p0)
            try:
                ms = time_scan(cfg, vpp)
            except (ValueError, B.XgError):
                continue  # more pairs per pass than one frame indexes
            if best is None or ms < best[2]:
                best = (cfg, vpp, ms)
    cfg0, vpp, _ = best
    for b, p in shapes[1:]:
        if cfg0.tile_h % (4 * p):
            continue
        cfg = FrameConfig(cfg0.tile_w, cfg0.tile_h, batch=b, pixels_per_thread=p)
        try:
            ms = time_scan(cfg, vpp)
        except (ValueError, B.XgError):
            continue
        if ms < best[2]:
            best = (cfg, vpp, ms)
    c = best[0]
    cfg = FrameConfig(c.tile_w, c.tile_h, batch=c.batch, pixels_per_thread=c.pixels_per_thread, persistent=1)
    try:
        ms = time_scan(cfg, vpp)
        if ms < best[2]:
            best = (cfg, vpp, ms)
    except (ValueError, B.XgError):
        pass
    return best


def _key(n: int, views) -> str:
    bucket = 1 << max(0, (n - 1).bit_length())
    v0 = views[0]
    return f"n<={bucket}|V={len(views)}|{v0.width}x{v0.height}"


def time_step(n: int, views, cfg: FrameConfig, cap: int, gaussians: tuple, target: torch.Tensor,
              reps: int = 5) -> float:
    """Median ms of the graphed fwd+bwd step in this configuration (ValueError if the
    configuration is invalid, e.g. its compositing block needs too much shared memory)."""
    step = GraphedStep(n, views, cfg, cap)
    step.load(gaussians, target)
    step.capture()
    times = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        step.replay()
        e.record()
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
    del step
    return statistics.median(times)


def autotune(n: int, views, gaussians: tuple, target: torch.Tensor, tiles=CANDIDATE_TILES,
             batches=CANDIDATE_BATCHES, ppts=(1, 2, 4), reps: int = 5, use_cache: bool = True) -> TuneResult:
    """Pick the tile shape, pixels per thread, staging batch and launch form (one block per
    tile or persistent blocks) with the fastest graphed step (cached on disk): first tile
    shape and pixels per thread at the smallest batch, then batch and launch form for the
    best of those.

    Every candidate computes the same image (tiles, batch and launch form are pure
    acceleration), so the choice never changes results."""
    key = _key(n, views)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            try:
                return TuneResult(**cache[key])
            except TypeError:
                pass
    best = None
    caps = {}
    for tw, th in tiles:
        caps[(tw, th)] = size_pairs(n, views, FrameConfig(tw, th), gaussians)
        for ppt in [p for p in ppts if th % (4 * p) == 0]:
            try:
                ms = time_step(n, views, FrameConfig(tw, th, batch=batches[0], pixels_per_thread=ppt),
                               caps[(tw, th)], gaussians, target, reps)
            except ValueError:
                continue
            if best is None or ms < best.ms:
                best = TuneResult(tw, th, batches[0], ppt, ms, caps[(tw, th)])
    b0 = best
    for b in batches:
        for pers in (0, 1):
            if b == b0.batch and pers == 0:
                continue
            cfg = FrameConfig(b0.tile_w, b0.tile_h, batch=b, pixels_per_thread=b0.pixels_per_thread, persistent=pers)
            try:
                ms = time_step(n, views, cfg, b0.pair_capacity, gaussians, target, reps)
            except ValueError:
                continue
            if ms < best.ms:
                best = TuneResult(b0.tile_w, b0.tile_h, b, b0.pixels_per_thread, ms, b0.pair_capacity, pers)
    cache[key] = asdict(best)
    if use_cache:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as fh:
            json.dump(cache, fh, indent=1)
    return best
