"""Parity at the benchmark's full sizes (launch configuration of bench.py).

multiroom_20M at 1920x1080, batches of 8 views: culling, z-buffer keys and the filtered
depth bit-exact for whole frames; the U-Net output on sampled crops, against the oracle's
FP64 U-Net run on the same (bit-exact) U-Net input: a crop aligned to the pooling grid
whose outputs lie further than the receptive field from its cut edges equals the full-frame
computation there.  multiroom_100M (8 views per batch; the serving mix of 1280x720,
1920x1080 and 2560x1440): keys bit-exact on a view, and served results equal to the same
requests rendered alone.
"""
import numpy as np
import pytest

import oracle
import synth
from synth.workloads import MULTIROOM_20M, MULTIROOM_100M, make_scene

pytestmark = pytest.mark.gpu

CH = (32, 64, 128, 256)
W, H, NLEV, CELL = 1920, 1080, 5, 0.25
MARGIN = 64      # > receptive-field radius of the 4-level net (about 58 pixels)
CROP = 256       # multiple of 2^(levels-1)


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


@pytest.fixture(scope="module")
def big():
    import paper_2502_11618_gb300 as lnr
    from paper_2502_11618_gb300 import build
    build.build()
    s = make_scene(MULTIROOM_20M, device="cuda")
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, CELL)
    w = synth.unet_weights(CH, seed=1)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(CELL)
    r.set_unet(CH, w, "bf16")
    yield lnr, s, g, w, r
    r.close()


def _crops():
    # (x0, y0) of 256x256 windows: two image corners and an interior window
    return [(0, 0), (W - CROP, H - CROP), (832, 416)]


def _check_crops(x_full, y_full, w, tol_abs, tol_psnr):
    for x0, y0 in _crops():
        x = np.ascontiguousarray(x_full[y0:y0 + CROP, x0:x0 + CROP])
        ref = oracle.unet(x, CH, w)
        # compare where the window's cut edges (not image borders) are farther than MARGIN
        xa = 0 if x0 == 0 else MARGIN
        ya = 0 if y0 == 0 else MARGIN
        xb = CROP if x0 + CROP == W else CROP - MARGIN
        yb = CROP if y0 + CROP == H else CROP - MARGIN
        got = y_full[y0 + ya:y0 + yb, x0 + xa:x0 + xb]
        exp = ref[ya:yb, xa:xb]
        assert np.abs(got - exp).max() <= tol_abs, (x0, y0, np.abs(got - exp).max())
        if tol_psnr:
            assert psnr(got, exp) >= tol_psnr


def test_20M_1080p_batch_of_8(big):
    lnr, s, g, w, r = big
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 8, seed=2)
    fs = [0.5, 1.0] * 4
    r.autotune(W, H, 8)
    ys = r.render_batch(views, intr, W, H, NLEV, fs)        # the benchmark's launch configuration
    for i in (0, 5):
        ref = oracle.render(g, views[i], intr, W, H, NLEV, fs[i])
        ncell, npts = r.render_stage(views[i], intr, W, H, NLEV, fs[i], lnr.STAGE_CULL)
        assert npts == ref["n_vis_points"]
        keys = r.render_stage(views[i], intr, W, H, NLEV, fs[i], lnr.STAGE_KEYS)
        assert np.array_equal(keys, ref["keys"])
        U0 = r.render_stage(views[i], intr, W, H, NLEV, fs[i], lnr.STAGE_FILTERED)
        assert np.array_equal(U0, ref["U0"])
        x = r.render_stage(views[i], intr, W, H, NLEV, fs[i], lnr.STAGE_UNET_IN)
        assert np.array_equal(x, ref["x"])
        assert 0.0 <= ys[i].min() and ys[i].max() <= 1.0
        _check_crops(x, ys[i], w, 2e-2, 45.0)


def test_20M_1080p_fp32_plain_crops(big):
    lnr, s, g, w, r = big
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 1, seed=31)[0]
    r.set_precision("fp32")
    try:
        y = r.render(view, intr, W, H, NLEV, 1.0)
        x = r.render_stage(view, intr, W, H, NLEV, 1.0, lnr.STAGE_UNET_IN)
        _check_crops(x, y, w, 1e-4, None)
    finally:
        r.set_precision("bf16")


@pytest.fixture(scope="module")
def huge():
    import paper_2502_11618_gb300 as lnr
    s = make_scene(MULTIROOM_100M, device="cuda")
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(CELL)
    r.set_unet(CH, synth.unet_weights(CH, seed=1), "bf16")
    yield lnr, s, r
    r.close()


def test_100M_keys_and_batch(huge):
    lnr, s, r = huge
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, CELL)
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 8, seed=2)
    ref = oracle.render(g, views[3], intr, W, H, NLEV, 1.0)
    keys = r.render_stage(views[3], intr, W, H, NLEV, 1.0, lnr.STAGE_KEYS)
    assert np.array_equal(keys, ref["keys"])
    U0 = r.render_stage(views[3], intr, W, H, NLEV, 1.0, lnr.STAGE_FILTERED)
    assert np.array_equal(U0, ref["U0"])
    ys = r.render_batch(views, intr, W, H, NLEV, 1.0)
    assert np.array_equal(ys[3], r.render(views[3], intr, W, H, NLEV, 1.0))


def test_100M_serving_mix_equals_alone(huge):
    lnr, s, r = huge
    reqs = synth.request_stream(s, 12, lam=None, seed=3)
    alone = [r.render(q.view, synth.intrinsics_for(q.W, q.H), q.W, q.H, q.n_levels, q.fs) for q in reqs]
    r.serve_start(max_batch=4, slots=3)
    try:
        tickets = [r.submit(q.view, synth.intrinsics_for(q.W, q.H), q.W, q.H, q.n_levels, q.fs) for q in reqs]
        for t, q, a in zip(tickets, reqs, alone):
            img = np.empty((q.H, q.W, 3), np.float32)
            while r.poll(t, img)[0] is None:
                pass
            assert np.array_equal(img, a)
    finally:
        r.serve_stop()
