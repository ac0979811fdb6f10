"""Soft z-buffer (Sec. 3, "Point Cloud Projection": colours of points that arrive at similar
depths are averaged) on the GPU against the CPU oracle.

The soft colours are integer sums of the contributing points' colours, so the GPU result
is bit-exact whatever the order of its atomics: RGB, D and A before the filter, the kept
depth and the U-Net input must equal the oracle's; the BF16 U-Net output stays within the
BF16 bars of the oracle's FP64 U-Net.  Served and batched renders equal the same requests
rendered alone, and switching back to the hard z-buffer restores its results.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

REL = 0.01
CH = (16, 32, 64)


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


@pytest.fixture(scope="module")
def scene():
    import paper_2502_11618_gb300 as lnr
    from paper_2502_11618_gb300 import build
    build.build()
    s = synth.multiroom_scene(n_points=1_500_000)
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    w = synth.unet_weights(CH, seed=1)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.25)
    r.set_unet(CH, w, "bf16")
    yield lnr, s, g, w, r
    r.close()


@pytest.mark.parametrize("pose", range(3))
def test_soft_stages_bit_exact(scene, pose):
    lnr, s, g, w, r = scene
    W, H, nl, fs = 320, 240, 3, 1.0
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 3, seed=5)[pose]
    r.set_soft_zbuffer(REL)
    try:
        ref = oracle.render(g, view, intr, W, H, nl, fs, soft=REL)
        hard = oracle.render(g, view, intr, W, H, nl, fs)
        rgb, D, A = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_RGBDA_RAW)
        assert np.array_equal(D, ref["D"]) and np.array_equal(A, ref["A"])
        assert np.array_equal(rgb, ref["rgb"])
        assert not np.array_equal(ref["rgb"], hard["rgb"])     # the rule changes colours here
        assert np.array_equal(r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_FILTERED), ref["U0"])
        assert np.array_equal(r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_UNET_IN), ref["x"])
    finally:
        r.set_soft_zbuffer(0.0)


def test_soft_unet_bf16_bars_and_batch(scene):
    lnr, s, g, w, r = scene
    W, H, nl = 256, 192, 3
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 3, seed=6)
    r.set_soft_zbuffer(REL)
    try:
        ys = r.render_batch(views, intr, W, H, nl, [1.0, 0.5, 1.0])
        ref = oracle.render(g, views[0], intr, W, H, nl, 1.0, w, CH, soft=REL)
        assert 0.0 <= ys[0].min() and ys[0].max() <= 1.0
        assert np.abs(ys[0] - ref["y"]).max() <= 2e-2
        assert psnr(ys[0], ref["y"]) >= 45.0
        for i, f in enumerate([1.0, 0.5, 1.0]):
            assert np.array_equal(ys[i], r.render(views[i], intr, W, H, nl, f))
    finally:
        r.set_soft_zbuffer(0.0)
    # back to the hard rule: its results again
    hard = oracle.render(g, views[0], intr, W, H, nl, 1.0)
    rgb, D, A = r.render_stage(views[0], intr, W, H, nl, 1.0, lnr.STAGE_RGBDA_RAW)
    assert np.array_equal(rgb, hard["rgb"])


def test_soft_served_equals_alone(scene):
    lnr, s, g, w, r = scene
    W, H, nl = 192, 128, 3
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 6, seed=7)
    r.set_soft_zbuffer(REL)
    try:
        alone = [r.render(v, intr, W, H, nl, 1.0) for v in views]
        r.serve_start(max_batch=4, slots=2)
        try:
            with pytest.raises(lnr.LnrError) as e:
                r.set_soft_zbuffer(0.02)                      # not while serving
            assert e.value.status == -2
            tickets = [r.submit(v, intr, W, H, nl, 1.0) for v in views]
            for t, a in zip(tickets, alone):
                img = np.empty((H, W, 3), np.float32)
                while r.poll(t, img)[0] is None:
                    pass
                assert np.array_equal(img, a)
        finally:
            r.serve_stop()
    finally:
        r.set_soft_zbuffer(0.0)


def test_soft_threshold_errors(scene):
    lnr, s, g, w, r = scene
    for bad in (-0.01, float("nan"), 2e6):
        with pytest.raises(lnr.LnrError) as e:
            r.set_soft_zbuffer(bad)
        assert e.value.status == -1
