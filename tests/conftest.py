import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); run with -m gpu")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.lib()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """Gradient comparisons of the GPU tests: how many entries meet the stated tolerance
    (1e-3 relative, 1e-6 absolute) on their own, and how many need the FP32 term allowance."""
    try:
        from tests.gpu_util import GRAD_STATS, PIXEL_STATS
    except Exception:
        return
    tr = terminalreporter
    if PIXEL_STATS:
        tr.write_sep("-", "pixels the oracle flags as ambiguous (a decision within rounding of its threshold)")
        for r in PIXEL_STATS:
            tr.write_line(f"{r['what']}: {r['pixels']} pixels, {r['flagged']} flagged "
                          f"({r['flagged'] / max(1, r['pixels']):.2e}), {r['over_tol']} of them beyond 1e-4")
    if not GRAD_STATS:
        return
    tr.write_sep("-", "gradient tolerance: strict (1e-3 rel, 1e-6 abs) vs with the FP32 term allowance")
    for r in GRAD_STATS:
        tr.write_line(f"{r['what']}: {r['checked']} checked, strict {r['strict_ok']} "
                      f"({100 * r['strict_frac']:.3f} %), with allowance {r['widened_ok']}, "
                      f"max err / strict tol {r['max_err_over_strict']:.3g}, "
                      f"allowance needed {r.get('term_rel_needed', float('nan')):.2g}")
