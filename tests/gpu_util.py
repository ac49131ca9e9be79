"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and pull every
intermediate array back to the host."""
from __future__ import annotations

import numpy as np
import torch

from paper_2403_04116_gb300 import binding as B
from paper_2403_04116_gb300.render import Frame, FrameConfig

NAMES = ("mean", "scale", "quat", "opacity", "intensity")


def to_device(g: dict) -> tuple:
    return tuple(torch.from_numpy(np.ascontiguousarray(g[k], dtype=np.float32)).cuda() for k in NAMES)


def run_forward(g: dict, views, tile=(16, 16), capacity=None, near_mm=0.2, batch=256, ppt=2) -> dict:
    """Project, bin, sort and render through the C ABI.  Without ``capacity`` the pair
    capacity is sized from a first binning pass (so the frame never overflows)."""
    dev = to_device(g)
    n = dev[4].shape[0]
    cap = capacity or max(1 << 16, 16 * n * len(views))
    cfg = FrameConfig(tile[0], tile[1], near_mm, batch=batch, pixels_per_thread=ppt)
    f = Frame(n, views, cfg, cap)
    f.project(*dev)
    proj = {"records": f.array("records").cpu().numpy(), "depth": f.array("depth").cpu().numpy(),
            "rect": f.array("rect").cpu().numpy().astype(np.int32), "count": f.array("count").cpu().numpy()}
    f.bin_sort()
    st = f.status()
    if capacity is None and st.code == B.XG_ERR_CAPACITY:
        f = Frame(n, views, cfg, int(st.pairs))
        f.project(*dev)
        f.bin_sort()
        st = f.status()
    image = torch.empty((f.V, f.H, f.W), dtype=torch.float32, device="cuda")
    ncon = torch.empty((f.V, f.H, f.W), dtype=torch.int32, device="cuda")
    f.render_fwd(image, ncon)
    torch.cuda.synchronize()
    M = int(st.pairs) if st.code == B.XG_OK else 0
    out = {**proj, "status": st, "M": M, "frame": f, "dev": dev,
           "value": f.array("value")[:M].cpu().numpy(),
           "range": f.array("range").cpu().numpy().view(np.uint32),
           "image": image.cpu().numpy(), "ncontrib": ncon.cpu().numpy(),
           "tfinal": f.array("tfinal").cpu().numpy().reshape(f.V, f.H, f.W),
           "last": f.array("last").cpu().numpy().reshape(f.V, f.H, f.W)}
    # key view * S + tile of every pair, from the ranges (which must tile [0, M) exactly),
    # and its depth key, looked up from its (view, Gaussian)
    out["key_tile"] = keys_from_ranges(out["range"], M)
    views_of = out["key_tile"].astype(np.int64) // f.range_stride
    out["key_depth"] = proj["depth"].view(np.uint32)[views_of * n + out["value"].astype(np.int64)]
    return out


def keys_from_ranges(rng: np.ndarray, M: int) -> np.ndarray:
    """The key (index into ``rng``) of each of the M pairs; every pair must lie in exactly
    one non-empty range."""
    key = np.full(M, 0xFFFFFFFF, np.uint32)
    hits = np.zeros(M, np.int64)
    for q in np.nonzero(rng[:, 1] > rng[:, 0])[0]:
        a, b = int(rng[q, 0]), int(rng[q, 1])
        assert b <= M, (q, a, b, M)
        key[a:b] = q
        hits[a:b] += 1
    assert (hits == 1).all(), "ranges overlap or leave pairs out"
    return key


def run_backward(fwd: dict, grad_image: np.ndarray) -> dict:
    f, dev = fwd["frame"], fwd["dev"]
    G = torch.from_numpy(np.ascontiguousarray(grad_image, dtype=np.float32)).cuda()
    grads = tuple(torch.empty_like(t) for t in dev)
    f.render_bwd(dev, G, grads)
    torch.cuda.synchronize()
    out = {k: t.cpu().numpy() for k, t in zip(NAMES, grads)}
    out["g2d"] = np.ascontiguousarray(f.array("grad2d").cpu().numpy()[:, :7].T)  # (7, V*n)
    return out


# ------------------------------------------------------------------------------------------
# gradient tolerance: strict (the stated bound) and with the FP32 term allowance
# ------------------------------------------------------------------------------------------
GRAD_RTOL, GRAD_ATOL = 1e-3, 1e-6
# FP32 allowance per unit of sum |per-pixel terms| behind a gradient (see test_gpu_parity)
GRAD_TERM_REL = 3e-5
GRAD_STATS: list = []  # one record per comparison, printed at the end of the session
PIXEL_STATS: list = []  # flagged-pixel counts of the image comparisons, printed likewise


def grad_compare(got, want, mag, what: str) -> dict:
    """Compare GPU gradients with the FP64 oracle's.  Strict: within 1e-3 relative with a
    1e-6 absolute floor.  Widened: plus GRAD_TERM_REL times the sum of |per-pixel terms|
    behind each gradient (``mag``).  Only entries with a term behind them are counted."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    mag = np.asarray(mag, np.float64)
    live = mag > 0
    err = np.abs(got - want)
    strict = GRAD_RTOL * np.abs(want) + GRAD_ATOL
    widened = strict + GRAD_TERM_REL * mag
    rec = {"what": what, "checked": int(live.sum()), "strict_ok": int((err <= strict)[live].sum()),
           "widened_ok": int((err <= widened)[live].sum()),
           "max_err_over_strict": float((err / strict)[live].max(initial=0.0)),
           "bad_widened": int((err > widened).sum()),
           # the smallest term allowance that would have passed every entry
           "term_rel_needed": float(((err - strict) / np.where(mag > 0, mag, np.inf))[live].max(initial=0.0))}
    rec["strict_frac"] = rec["strict_ok"] / max(1, rec["checked"])
    GRAD_STATS.append(rec)
    return rec


def merge_stats(recs: list, what: str) -> dict:
    out = {"what": what, "checked": sum(r["checked"] for r in recs), "strict_ok": sum(r["strict_ok"] for r in recs),
           "widened_ok": sum(r["widened_ok"] for r in recs), "bad_widened": sum(r["bad_widened"] for r in recs),
           "max_err_over_strict": max((r["max_err_over_strict"] for r in recs), default=0.0),
           "term_rel_needed": max((r.get("term_rel_needed", 0.0) for r in recs), default=0.0)}
    out["strict_frac"] = out["strict_ok"] / max(1, out["checked"])
    return out
