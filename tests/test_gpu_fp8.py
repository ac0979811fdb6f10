"""FP8 (E4M3) tensor-core U-Net against the CPU oracle's FP64 U-Net.

Bar: PSNR >= 38 dB per view, outputs in [0, 1].  Scales are calibrated on one view and the
bar is checked on other views.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FP8_PSNR = 38.0


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


@pytest.fixture(scope="module")
def setup():
    import paper_2502_11618_gb300 as lnr
    from paper_2502_11618_gb300 import build
    build.build()
    s = synth.multiroom_scene(n_points=800_000)
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    ch = (32, 64, 128, 256)
    w = synth.unet_weights(ch, seed=1)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.25)
    r.set_unet(ch, w, "bf16")
    yield lnr, s, g, ch, w, r
    r.close()


def test_fp8_needs_calibration(setup):
    lnr, s, g, ch, w, r = setup
    with pytest.raises(lnr.LnrError) as e:
        r.set_precision("fp8")
    assert e.value.status == -2


def test_fp8_psnr_against_fp64(setup):
    lnr, s, g, ch, w, r = setup
    W, H = 960, 544
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 4, seed=21)
    r.calibrate(views[0], intr, W, H, 4, 1.0)
    r.set_precision("fp8")
    for v in views[1:]:
        ref = oracle.render(g, v, intr, W, H, 4, 1.0, w, ch)
        y = r.render(v, intr, W, H, 4, 1.0)
        assert 0.0 <= y.min() and y.max() <= 1.0
        assert psnr(y, ref["y"]) >= FP8_PSNR, psnr(y, ref["y"])
    yb = r.render_batch(views[1:3], intr, W, H, 4, 1.0)
    assert np.array_equal(yb[0], r.render(views[1], intr, W, H, 4, 1.0))
    r.autotune(W, H, 2)
    y = r.render(views[1], intr, W, H, 4, 1.0)
    ref = oracle.render(g, views[1], intr, W, H, 4, 1.0, w, ch)
    assert psnr(y, ref["y"]) >= FP8_PSNR
    r.set_precision("bf16")
