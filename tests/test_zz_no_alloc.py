"""xg_sort_pairs_noalloc, the allocation-free pair sort, against xg_bin_sort and against
a host stable sort.

Callers that may not allocate device memory (a plugin inside an application that owns
the GPU's memory pool, a real-time pipeline that forbids allocation after start-up) sort
their (tile, depth, Gaussian) pairs with xg_sort_pairs_noalloc, whose scratch lives in a
static device array inside the library.  These tests feed it the pairs xg_bin_sort emits
and require xg_bin_sort's sorted output bit for bit, on two different calls in a row (the
static array is shared by every call and keeps the previous call's contents); the frame's
pair keys are read off its ranges.  Both sorts run the same radix kernels, so every output
is also checked against NumPy's stable lexsort, on the frame's pairs and on random keys:
inputs four bytes off a 16-byte boundary (the direct-load path), tile_bits 0, 24 and 32
(four, seven and eight passes), and the largest accepted count.  A child process with
every bounded wait made to give up shows that a failure on the device is reported by
xg_sort_pairs_noalloc_status.

The file is named so that pytest collects it last.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2403_04116_gb300 import binding as B  # noqa: E402
from paper_2403_04116_gb300 import synth  # noqa: E402
from paper_2403_04116_gb300.render import Frame, FrameConfig  # noqa: E402
from tests.gpu_util import keys_from_ranges  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2403_04116_gb300 import build
    build.build()
    B.lib()


def _binned_frame(n, n_views, W, H, tile, cid):
    g = synth.gaussians(n, synth.scene_side_mm(W), synth.rng(cid, 0))
    views = synth.circular_views(n_views, W, H, first_rad=0.37 * cid)
    dev = tuple(torch.from_numpy(g[k]).cuda() for k in ("mean", "scale", "quat", "opacity", "intensity"))
    f = Frame(n, views, FrameConfig(*tile), pair_capacity=1 << 20)
    f.project(*dev)
    f.bin_sort()
    st = f.status()
    assert st.code == B.XG_OK
    return f, int(st.pairs)


def _emitted_pairs(f: Frame, M: int):
    """Every pair of the frame in (view, Gaussian index) order, each Gaussian's tiles
    row-major, keyed tile * V + view -- an unsorted input whose stable sort by (key, depth)
    is the frame's sorted pair list, which is ordered by (tile, view, depth, index)."""
    rect = f.array("rect").cpu().numpy().astype(np.int64)
    count = f.array("count").cpu().numpy().view(np.uint32)
    offset = np.concatenate([[0], np.cumsum(count.astype(np.int64))[:-1]])
    dbits = f.array("depth").cpu().numpy().view(np.uint32)
    kt, kd, val = (np.empty(M, np.uint32) for _ in range(3))
    for vg in np.nonzero(count)[0]:
        v, g = divmod(int(vg), f.n)
        x0, y0, x1, y1 = rect[vg]
        ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        tiles = ((ys.ravel() * f.tiles_x + xs.ravel()) * f.V + v).astype(np.uint32)
        o = int(offset[vg])
        kt[o:o + tiles.size] = tiles
        kd[o:o + tiles.size] = dbits[vg]
        val[o:o + tiles.size] = g
    return kt, kd, val


def _sort_noalloc(kt, kd, val, tile_bits, offset=0):
    """Sort through the C ABI.  With ``offset`` the inputs and outputs start ``offset``
    words into larger device buffers (4-byte, not 16-byte, aligned for offset 1)."""
    def to_dev(a):
        t = torch.zeros(a.size + offset, dtype=torch.int32, device="cuda")
        t[offset:] = torch.from_numpy(a.view(np.int32)).cuda()
        return t
    ins = [to_dev(a) for a in (kt, kd, val)]
    outs = [torch.full_like(t, -1) for t in ins]
    ptr = lambda t: t.data_ptr() + 4 * offset  # noqa: E731
    stream = torch.cuda.current_stream().cuda_stream
    B.xg_sort_pairs_noalloc(ptr(ins[0]), ptr(ins[1]), ptr(ins[2]), kt.size, tile_bits,
                            ptr(outs[0]), ptr(outs[1]), ptr(outs[2]), stream)
    assert B.xg_sort_pairs_noalloc_status(stream) == B.XG_OK
    torch.cuda.synchronize()
    return [o[offset:].cpu().numpy().view(np.uint32) for o in outs]


def _host_stable_sort(kt, kd, val):
    """NumPy's stable sort by (key_tile, key_depth): lexsort's last key is the primary one."""
    order = np.lexsort((kd, kt))
    return [kt[order], kd[order], val[order]]


@pytest.mark.parametrize("first,second", [((3000, 5, 100, 75, (8, 8), 10), (6000, 2, 128, 128, (16, 16), 31))])
def test_noalloc_sort_matches_bin_sort_twice(first, second):
    for case in (first, second):
        f, M = _binned_frame(*case)
        assert 0 < M <= B.XG_NOALLOC_MAX_PAIRS
        kt, kd, val = _emitted_pairs(f, M)
        keys = f.V * f.tiles_per_view
        tile_bits = int(np.ceil(np.log2(keys))) if keys > 1 else 0
        got = _sort_noalloc(kt, kd, val, tile_bits)
        key = keys_from_ranges(f.array("range").cpu().numpy().view(np.uint32), M).astype(np.int64)
        view, tile = key // f.range_stride, key % f.range_stride
        val_s = f.array("value")[:M].cpu().numpy().view(np.uint32)
        dbits = f.array("depth").cpu().numpy().view(np.uint32)
        kd_s = dbits[view * f.n + val_s]
        want = [(tile * f.V + view).astype(np.uint32), kd_s, val_s]
        for g_, w_, name in zip(got, want, ("key_tile", "key_depth", "value")):
            np.testing.assert_array_equal(g_, w_, err_msg=name)
        for g_, w_, name in zip(got, _host_stable_sort(kt, kd, val), ("key_tile", "key_depth", "value")):
            np.testing.assert_array_equal(g_, w_, err_msg=f"{name} against the host stable sort")


# (pairs, tile_bits, word offset of the buffers, distinct depth keys): ties in (tile, depth)
# are frequent, so the order of equal keys (the input order) is checked too
RANDOM_CASES = [(B.XG_NOALLOC_MAX_PAIRS, 23, 0, 1 << 20), (5000, 0, 1, 50), (70_000, 24, 1, 3000),
                (300_000, 32, 0, 1 << 32), (B.XG_NOALLOC_MAX_PAIRS, 8, 1, 1000)]


def test_noalloc_sort_random_keys_against_host_stable_sort():
    gen = np.random.default_rng(12)
    for count, tile_bits, offset, depths in RANDOM_CASES:  # one call after another
        kt = gen.integers(0, 1 << tile_bits, size=count, dtype=np.uint64).astype(np.uint32)
        kd = gen.integers(0, depths, size=count, dtype=np.uint64).astype(np.uint32)
        if depths == 1 << 32:
            kd[::3] = kd[1::3][: kd[::3].size]  # repeated depth keys among full-range ones
        val = gen.permutation(count).astype(np.uint32)
        got = _sort_noalloc(kt, kd, val, tile_bits, offset)
        for g_, w_, name in zip(got, _host_stable_sort(kt, kd, val), ("key_tile", "key_depth", "value")):
            np.testing.assert_array_equal(g_, w_, err_msg=f"{name}: {count} pairs, tile_bits {tile_bits}, "
                                                          f"offset {offset}")


CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2403_04116_gb300 import binding as B
n = B.XG_NOALLOC_MAX_PAIRS
gen = np.random.default_rng(3)
ins = [torch.from_numpy(gen.integers(0, 1 << 16, size=n, dtype=np.int64).astype(np.int32)).cuda() for _ in range(3)]
outs = [torch.empty_like(t) for t in ins]
s = torch.cuda.current_stream().cuda_stream
B.xg_sort_pairs_noalloc(*(t.data_ptr() for t in ins), n, 16, *(t.data_ptr() for t in outs), s)
code = B.xg_sort_pairs_noalloc_status(s)
after = float(torch.ones(1000, device="cuda").sum().item())  # the context still works
print("code", code, "after", after)
"""


def _child(env_extra):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(root))], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    words = r.stdout.split()
    return {words[i]: float(words[i + 1]) for i in range(0, len(words) - 1, 2)}


def test_noalloc_sort_reports_device_failures():
    """XG_SPIN_LIMIT=0 (read once per process) makes every first bounded wait of the radix
    scatter give up, as an expired wait would: the status query must say XG_ERR_CHECK,
    and the context must stay usable.  A clean child is the control."""
    ok = _child({})
    assert ok["code"] == B.XG_OK and ok["after"] == 1000.0
    bad = _child({"XG_SPIN_LIMIT": "0"})
    assert bad["code"] == B.XG_ERR_CHECK and bad["after"] == 1000.0


def test_noalloc_sort_rejects_too_many_pairs():
    with pytest.raises(B.XgError) as e:
        B.xg_sort_pairs_noalloc(0, 0, 0, B.XG_NOALLOC_MAX_PAIRS + 1, 8, 0, 0, 0, 0)
    assert e.value.code == B.XG_ERR_INVALID_ARG
