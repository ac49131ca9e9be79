"""The compositing kernels' decision exponential on the device, scalar and two-lane packed,
bit-identical to the FP32 replica's (an independent C implementation of the same published
method) on 16 M inputs: uniform over [-80, 0] and every float within a few ulps of the
range-reduction boundaries x log2 e = k - 1/2, where both sides must take k as the integer
nearest the exact product x log2 e (one fused multiply-add), not as the rounding of a
separately rounded product."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2403_04116_gb300 import binding as B  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2403_04116_gb300 import build
    build.build()
    oracle.lib()


def _inputs() -> np.ndarray:
    gen = np.random.default_rng(7)
    uniform = gen.uniform(-80.0, 0.0, 1 << 23).astype(np.float32)
    near = []
    for k in range(-114, 1):
        c = np.float32((k - 0.5) / np.log2(np.e)).view(np.uint32).astype(np.int64)
        near.append(np.arange(c - 32768, c + 32769).astype(np.uint32).view(np.float32))
    x = np.concatenate([uniform] + near + [np.float32([0.0, -80.0, -100.0, -1e-30, 1e-30])])
    return x if x.size % 2 else x[:-1]  # an odd count: the last pair has one lane


def test_decision_exp_bit_identical_to_the_replica():
    x = _inputs()
    assert x.size % 2 == 1 and x.size > (1 << 23)
    d = torch.from_numpy(x).cuda()
    ys, yp = torch.empty_like(d), torch.empty_like(d)
    B.xg_exp_check(d.data_ptr(), ys.data_ptr(), yp.data_ptr(), d.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    want = oracle.replica_exp(x).view(np.uint32)
    got_s = ys.cpu().numpy().view(np.uint32)
    got_p = yp.cpu().numpy().view(np.uint32)
    assert np.count_nonzero(got_s != want) == 0
    assert np.count_nonzero(got_p != want) == 0


def test_exp_check_rejects_bad_arguments():
    with pytest.raises(B.XgError) as e:
        B.xg_exp_check(0, 0, 0, 10, 0)
    assert e.value.code == B.XG_ERR_INVALID_ARG
