"""ACUI grid initialisation on the device (Eq. 13) against the FP64 oracle: every point
bit-exact (the oracle's FP64 value rounded once to FP32), and the error paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import acui64 as A  # noqa: E402
from paper_2403_04116_gb300 import binding as B  # noqa: E402
from paper_2403_04116_gb300.render import _stream_handle  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib(build_if_missing=True)


@pytest.mark.parametrize("S,M,d", [((200.0, 200.0, 200.0), (256, 256, 256), 8), ((341.3, 170.7, 85.3), (512, 300, 97), 8),
                                   ((1.0, 2.0, 3.0), (100, 10, 1), 3.5), ((50.0, 60.0, 70.0), (1024, 1024, 1024), 16)])
def test_points_bit_exact(S, M, d):
    n = B.xg_acui_count(S, M, d)
    assert n == A.acui_count(S, M, d)
    out = torch.full((3, n), float("nan"), device="cuda")
    B.xg_acui_points(S, M, d, out.data_ptr(), n, _stream_handle())
    want = A.acui_points64(S, M, d).astype(np.float32)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_capacity_and_argument_errors():
    out = torch.empty(3, 10, device="cuda")
    with pytest.raises(B.XgError) as e:
        B.xg_acui_points((1.0,) * 3, (8, 8, 8), 2, out.data_ptr(), 10, _stream_handle())
    assert e.value.code == B.XG_ERR_CAPACITY
    with pytest.raises(B.XgError) as e:
        B.xg_acui_points((1.0,) * 3, (8, 8, 8), -1.0, out.data_ptr(), 10, _stream_handle())
    assert e.value.code == B.XG_ERR_INVALID_ARG


def test_training_from_the_acui_grid_improves_heldout_psnr():
    import math
    from paper_2403_04116_gb300.render import FrameConfig
    from paper_2403_04116_gb300.train import TrainConfig, Trainer, acui_raw, config3
    side, tr_v, tr_t, te_v, te_t, _ = config3(1000, 128, seed_id=61)
    cfg = TrainConfig(views_per_step=8, position_scale=side, decay_steps=300)
    raw = acui_raw(side, 64, 2.0, cfg.n_features)  # floor(64 / 4) + 1 = 17: 35^3 Gaussians
    assert raw["mean"].shape == (3, 35 ** 3)
    tr = Trainer(raw, tr_v, torch.from_numpy(tr_t).cuda(), cfg, FrameConfig(16, 16))
    te = torch.from_numpy(te_t).cuda()
    before = tr.psnr(te_v, te).mean()
    tr.capture()
    tr.train(300, check_every=100)
    torch.cuda.synchronize()
    after = tr.psnr(te_v, te).mean()
    assert math.isfinite(after) and after > before + 1.0, (before, after)
