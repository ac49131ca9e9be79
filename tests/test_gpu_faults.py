"""Failure detection without a GPU fault.  XG_SPIN_LIMIT=0 (read once per process) makes
every first wait of the radix scatter give up at once, as an expired wait would: the
kernels must record XG_ERR_CHECK in the status word, return without a hang or a stray
access (the copy in flight is drained with the full limit), and leave the stream usable.
Run in child processes, each with its own CUDA context."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2403_04116_gb300 import binding as B, synth
from paper_2403_04116_gb300.render import Frame, FrameConfig
W = 256
g = synth.gaussians(50000, synth.scene_side_mm(W), synth.rng(1, 0))
views = synth.circular_views(8, W, W)
dev = tuple(torch.from_numpy(g[k]).cuda() for k in ("mean", "scale", "quat", "opacity", "intensity"))
f = Frame(50000, views, FrameConfig(16, 16), 1 << 22)
f.project(*dev)
f.bin_sort()
st = f.status()
img = torch.full((8, W, W), -1.0, device="cuda")
f.render_fwd(img)
torch.cuda.synchronize()
after = float(torch.ones(1000, device="cuda").sum().item())  # the context still works
print("code", st.code, "pairs", st.pairs, "image_max", float(img.max()), "after", after)
"""


def _run(env_extra):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    words = r.stdout.split()
    return {words[i]: float(words[i + 1]) for i in range(0, len(words) - 1, 2)}


def test_expired_waits_are_reported_and_the_context_stays_usable():
    ok = _run({})
    assert ok["code"] == 0 and ok["pairs"] > 0 and ok["after"] == 1000.0
    bad = _run({"XG_SPIN_LIMIT": "0"})
    assert bad["code"] == 5  # XG_ERR_CHECK
    assert bad["pairs"] == 0 and bad["image_max"] == 0.0  # later stages were no-ops writing zeros
    assert bad["after"] == 1000.0
