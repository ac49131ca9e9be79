"""xg_sort_pairs_noalloc, the allocation-free pair sort, against xg_bin_sort.

Callers that may not allocate device memory (a plugin inside an application that owns
the GPU's memory pool, a real-time pipeline that forbids allocation after start-up) sort
their (tile, depth, Gaussian) pairs with xg_sort_pairs_noalloc, whose scratch lives in a
static device array inside the library.  These tests feed it the pairs xg_bin_sort emits
and require xg_bin_sort's sorted output bit for bit, on two different calls in a row (the
static array is shared by every call and keeps the previous call's contents).  The
frame's pair keys are read off its ranges.

The file is named so that pytest collects it last.
"""
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


def _sort_noalloc(kt, kd, val, tile_bits):
    to_dev = lambda a: torch.from_numpy(a.view(np.int32)).cuda()  # noqa: E731
    ins = [to_dev(a) for a in (kt, kd, val)]
    outs = [torch.empty_like(t) for t in ins]
    B.xg_sort_pairs_noalloc(ins[0].data_ptr(), ins[1].data_ptr(), ins[2].data_ptr(), kt.size, tile_bits,
                            outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return [o.cpu().numpy().view(np.uint32) for o in outs]


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


def test_noalloc_sort_rejects_too_many_pairs():
    with pytest.raises(B.XgError) as e:
        B.xg_sort_pairs_noalloc(0, 0, 0, B.XG_NOALLOC_MAX_PAIRS + 1, 8, 0, 0, 0, 0)
    assert e.value.code == B.XG_ERR_INVALID_ARG
