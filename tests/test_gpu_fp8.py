"""FP8 (E4M3) tensor-core U-Net against the CPU oracle's FP64 U-Net.

Bar: PSNR >= 38 dB per view, outputs in [0, 1].  Scales are calibrated on other views than
the ones checked.  Sizes: the benchmark's 16 poses of the 20M-point scan at 1920x1080 (the
precision workload; the FP64 U-Net runs on three aligned 256x256 crops per view, which keeps
the oracle to seconds), a 960x544 frame of a smaller scan, and a ragged 264x136 frame with
other weights, once the weakest case on record.
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



def test_fp8_small_ragged_frame_meets_the_bar():
    """264x136 (a ragged tail at every level), seed-4 weights, calibrated on one view."""
    import paper_2502_11618_gb300 as lnr
    s = synth.multiroom_scene(n_points=300_000)
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    ch = (32, 64, 128, 256)
    w = synth.unet_weights(ch, seed=4)
    r = lnr.Renderer(0)
    try:
        r.load_cloud(s.xyz, s.rgb, s.scan_id)
        r.build_grid(0.25)
        r.set_unet(ch, w, "bf16")
        W, H = 264, 136
        intr = synth.intrinsics_for(W, H)
        views = synth.random_poses(s, 3, seed=9)
        r.calibrate(views[0], intr, W, H, 4, 1.0)
        r.set_precision("fp8")
        for v in views[1:]:
            ref = oracle.render(g, v, intr, W, H, 4, 1.0, w, ch)["y"]
            y = r.render(v, intr, W, H, 4, 1.0)
            assert 0.0 <= y.min() and y.max() <= 1.0
            assert psnr(y, ref) >= FP8_PSNR, psnr(y, ref)
    finally:
        r.close()


def test_fp8_1080p_16_views_of_the_20M_scan():
    """The precision workload: multiroom_20M, the 16 benchmark poses at 1920x1080, in
    batches of 8; scales calibrated on 4 other poses.  Per view the PSNR over three aligned
    crops (two corners, one interior window) against the oracle's FP64 U-Net on the
    bit-exact U-Net input must reach the bar; the minimum over the views is printed."""
    import paper_2502_11618_gb300 as lnr
    from synth.workloads import MULTIROOM_20M, make_scene
    W, H, NLEV, CROP, MARGIN = 1920, 1080, 5, 256, 64
    ch = (32, 64, 128, 256)
    s = make_scene(MULTIROOM_20M, device="cuda")
    w = synth.unet_weights(ch, seed=1)
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 16, seed=2)
    fs = [0.5, 1.0] * 8
    r = lnr.Renderer(0)
    worst = []
    try:
        r.load_cloud(s.xyz, s.rgb, s.scan_id)
        r.build_grid(0.25)
        r.set_unet(ch, w, "bf16")
        r.calibrate(synth.random_poses(s, 4, seed=77), intr, W, H, NLEV, 1.0)
        r.set_precision("fp8")
        ys = np.concatenate([r.render_batch(views[k:k + 8], intr, W, H, NLEV, fs[k:k + 8]) for k in (0, 8)])
        for i, v in enumerate(views):
            x = r.render_stage(v, intr, W, H, NLEV, fs[i], lnr.STAGE_UNET_IN)
            got, exp = [], []
            for x0, y0 in [(0, 0), (W - CROP, H - CROP), (832, 416)]:
                ref = oracle.unet(np.ascontiguousarray(x[y0:y0 + CROP, x0:x0 + CROP]), ch, w)
                xa = 0 if x0 == 0 else MARGIN
                ya = 0 if y0 == 0 else MARGIN
                xb = CROP if x0 + CROP == W else CROP - MARGIN
                yb = CROP if y0 + CROP == H else CROP - MARGIN
                got.append(ys[i][y0 + ya:y0 + yb, x0 + xa:x0 + xb].ravel())
                exp.append(ref[ya:yb, xa:xb].ravel())
            assert 0.0 <= ys[i].min() and ys[i].max() <= 1.0
            worst.append(psnr(np.concatenate(got), np.concatenate(exp)))
    finally:
        r.close()
    print("FP8 crop PSNR per view:", [round(p, 2) for p in worst], "min", round(min(worst), 2))
    assert min(worst) >= FP8_PSNR, worst


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
    for k in ("LNR_CONV_EPI", "LNR_CONV_TMA_STORE", "LNR_CONV_KERNEL", "LNR_CONV_TMEM1"):
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
