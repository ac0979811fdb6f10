"""Failure detection on the GPU without a fault: every wait of the tensor-core kernels is
bounded, and a wait that runs out makes the kernel drain its copies, free its tensor memory
and return, with an error word that the host turns into LNR_E_TIMEOUT.

LNR_TEST_STALL_ONCE=1 makes the first tensor-core conv launch of the process wait on a
barrier that nothing arrives on, with a ~1 ms limit on every wait of that launch.  The
render must fail with LNR_E_TIMEOUT, and the same context must then render the frame
correctly (BF16 bars against the oracle's FP64 U-Net).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import synth, oracle
import paper_2502_11618_gb300 as lnr
s = synth.room_scene(n_points=60_000, seed=0)
ch = (16, 32, 64)
w = synth.unet_weights(ch, seed=1)
W, H = 128, 96
intr = synth.intrinsics_for(W, H)
view = synth.random_poses(s, 1, seed=2)[0]
r = lnr.Renderer(0)
r.load_cloud(s.xyz, s.rgb, s.scan_id); r.build_grid(0.5); r.set_unet(ch, w, "bf16")
try:
    r.render(view, intr, W, H, 3, 1.0)
    print("no timeout"); sys.exit(2)
except lnr.LnrError as e:
    assert e.status == -5, e
    print("timeout reported:", e)
g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.5)
ref = oracle.render(g, view, intr, W, H, 3, 1.0, w, ch)["y"]
for _ in range(2):                       # eager, then the captured graph
    y = r.render(view, intr, W, H, 3, 1.0)
    d = y.astype(np.float64) - ref
    assert np.abs(d).max() <= 2e-2 and 10 * np.log10(1 / np.mean(d * d)) >= 45.0
print("recovered")
r.close()
"""


def test_bounded_wait_runs_out_and_the_context_recovers():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    from paper_2502_11618_gb300 import build
    build.build()
    env = dict(os.environ, LNR_TEST_STALL_ONCE="1")
    r = subprocess.run([sys.executable, "-c", _SCRIPT.format(root=root)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "timeout reported" in r.stdout and "recovered" in r.stdout
