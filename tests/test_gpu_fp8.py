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



# One FP8 render of a ragged 264 x 136 frame by the untuned halo kernel, written to argv[1].
_FP8_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import synth
import paper_2502_11618_gb300 as lnr
s = synth.multiroom_scene(n_points=300_000)
ch = (32, 64, 128, 256)
w = synth.unet_weights(ch, seed=4)
r = lnr.Renderer(0); r.load_cloud(s.xyz, s.rgb, s.scan_id); r.build_grid(0.25); r.set_unet(ch, w, "bf16")
W, H = 264, 136
intr = synth.intrinsics_for(W, H)
views = synth.random_poses(s, 3, seed=9)
r.calibrate(views[0], intr, W, H, 4, 1.0)
r.set_precision("fp8")
np.save(sys.argv[1], np.stack([r.render(v, intr, W, H, 4, 1.0) for v in views[1:]]))
"""

_FP8_VARIANTS = {
    "4_epilogue_warps": dict(LNR_CONV_EPI="4"),
    "12_epilogue_warps": dict(LNR_CONV_EPI="12"),
    "12_epilogue_warps_direct_stores": dict(LNR_CONV_EPI="12", LNR_CONV_TMA_STORE="0"),
    "one_staging_buffer": dict(LNR_CONV_TMA_STORE="1"),
}


def _fp8_render(env_extra, tmp_path, tag):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / f"{tag}.npy")
    env = dict(os.environ, **env_extra)
    for k in ("LNR_CONV_EPI", "LNR_CONV_TMA_STORE", "LNR_CONV_KERNEL"):
        if k not in env_extra:
            env.pop(k, None)
    r = subprocess.run([sys.executable, "-c", _FP8_SCRIPT.format(root=root), out], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


@pytest.fixture(scope="module")
def fp8_default(setup, tmp_path_factory):
    return _fp8_render({}, tmp_path_factory.mktemp("fp8"), "default")


@pytest.mark.parametrize("variant", list(_FP8_VARIANTS))
def test_fp8_each_halo_variant(fp8_default, variant, tmp_path):
    """Forcing the untuned FP8 halo kernel to 4 or 12 epilogue warps, direct or
    single-buffered stores changes only how accumulators leave TMEM, not the arithmetic: every variant's frames equal the default
    configuration's bit for bit, on a ragged frame size, and stay in [0, 1]."""
    y = _fp8_render(_FP8_VARIANTS[variant], tmp_path, variant)
    assert 0.0 <= y.min() and y.max() <= 1.0
    assert np.array_equal(y, fp8_default)
