"""Synthetic training-pair input (Sec. 3, "Training Data Generation") through the C ABI:
the filtered and unfiltered variants must equal the oracle's composition of its own
(bit-exact) depth, kept mask and colours with the same ground-truth image."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2502_11618_gb300 as lnr
    from paper_2502_11618_gb300 import build
    build.build()
    s = synth.room_scene()
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.5)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.5)
    yield lnr, s, g, r
    r.close()


@pytest.mark.parametrize("unfiltered", [False, True])
@pytest.mark.parametrize("W,H,nl,fs", [(256, 256, 3, 1.0), (200, 136, 2, 0.5)])
def test_training_input_matches_oracle(setup, unfiltered, W, H, nl, fs):
    lnr, s, g, r = setup
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 2, seed=8)[1]
    gt = np.random.default_rng(3).random((H, W, 3), dtype=np.float32)
    ref = oracle.render(g, view, intr, W, H, nl, fs)
    exp = oracle.training_input(ref["D"], ref["U0"], ref["rgb"], gt, intr.zfar, unfiltered)
    got = r.training_input(view, intr, W, H, nl, fs, gt, unfiltered)
    assert np.array_equal(got, exp)
    kept = np.isfinite(ref["U0"])
    assert np.array_equal(got[..., 4] == 1, (kept | np.isfinite(ref["D"])) if unfiltered else kept)


def test_training_input_errors(setup):
    lnr, s, g, r = setup
    intr = synth.intrinsics_for(64, 64)
    view = synth.random_poses(s, 1)[0]
    with pytest.raises(ValueError):
        r.training_input(view, intr, 64, 64, 2, 1.0, np.zeros((32, 64, 3), np.float32))
    with pytest.raises(lnr.LnrError) as e:
        r.training_input(view, intr, 64, 64, 2, -1.0, np.zeros((64, 64, 3), np.float32))  # negative fs
    assert e.value.status == -1
