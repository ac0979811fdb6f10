"""GPU parity of the render path through the C ABI against the CPU oracle.

Culling, splat, resolve and filter are integer / compare work with a fixed FP32
operation sequence: they must match the oracle bit for bit.  The FP32 U-Net must stay
within 1e-4 (max abs) of the oracle's FP64 U-Net, outputs in [0, 1].
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module")
def lnr():
    import paper_2502_11618_gb300 as p
    from paper_2502_11618_gb300 import build
    build.build()
    return p


@pytest.fixture(scope="module")
def room():
    s = synth.room_scene()
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.5)
    return s, g


@pytest.fixture(scope="module")
def room_renderer(lnr, room):
    s, _ = room
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.5)
    r.set_unet((16, 32, 64), synth.unet_weights((16, 32, 64), seed=1), "fp32")
    yield r
    r.close()


def _nonempty_visible(g, vis):
    counts = np.diff(g.cell_start.astype(np.int64))
    return int(((vis == 1) & (counts > 0)).sum())


def test_grid_matches_oracle(lnr, room, room_renderer):
    s, g = room
    g0, dims = room_renderer.grid_info()
    assert np.array_equal(g0, g.g0) and np.array_equal(dims, g.dims)


@pytest.mark.parametrize("pose", range(4))
def test_stages_bit_exact_room(lnr, room, room_renderer, pose):
    s, g = room
    W, H, nl, fs = 256, 256, 3, 1.0
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 4, seed=2)[pose]
    ref = oracle.render(g, view, intr, W, H, nl, fs)
    r = room_renderer
    ncell, npts = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_CULL)
    assert ncell == _nonempty_visible(g, ref["visible"])
    assert npts == ref["n_vis_points"]
    keys = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_KEYS)
    assert np.array_equal(keys, ref["keys"])
    rgb, D, A = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_RGBDA_RAW)
    assert np.array_equal(D, ref["D"]) and np.array_equal(A, ref["A"])
    assert np.array_equal(rgb, ref["rgb"])
    U0 = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_FILTERED)
    assert np.array_equal(U0, ref["U0"])
    x = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_UNET_IN)
    assert np.array_equal(x, ref["x"])


@pytest.mark.parametrize("W,H,nl,fs", [(199, 131, 5, 0.5), (64, 64, 0, 1.0), (256, 200, 6, 0.0),
                                       (250, 170, 1, float("inf")), (33, 17, 4, 2.0)])
def test_filter_ragged_sizes_and_strengths(lnr, room, room_renderer, W, H, nl, fs):
    s, g = room
    intr = synth.intrinsics_for(W, H)
    for view in synth.random_poses(s, 2, seed=5):
        ref = oracle.render(g, view, intr, W, H, nl, fs)
        keys = room_renderer.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_KEYS)
        assert np.array_equal(keys, ref["keys"])
        U0 = room_renderer.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_FILTERED)
        assert np.array_equal(U0, ref["U0"])


def test_unet_fp32_room(lnr, room, room_renderer):
    s, g = room
    W, H, nl, fs = 256, 256, 3, 1.0
    intr = synth.intrinsics_for(W, H)
    w = synth.unet_weights((16, 32, 64), seed=1)
    for view in synth.random_poses(s, 2, seed=2):
        ref = oracle.render(g, view, intr, W, H, nl, fs, w, (16, 32, 64))
        y = room_renderer.render(view, intr, W, H, nl, fs)
        assert y.min() >= 0.0 and y.max() <= 1.0
        assert np.abs(y - ref["y"]).max() <= FP32_TOL


def test_batch_equals_single(lnr, room, room_renderer):
    s, g = room
    W, H, nl = 128, 96, 3
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 3, seed=8)
    fs = [0.5, 1.0, 1.5]
    yb = room_renderer.render_batch(views, intr, W, H, nl, fs)
    for i, v in enumerate(views):
        y1 = room_renderer.render(v, intr, W, H, nl, fs[i])
        assert np.array_equal(yb[i], y1)


def test_batch_beyond_one_splat_launch(lnr, room, room_renderer):
    """A batch of more views than one splat launch covers (64): views on either side of
    the boundary equal the same views rendered alone, bit for bit."""
    s, g = room
    W, H, nl = 64, 48, 2
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 67, seed=21)
    fs = [0.5 + (i % 3) * 0.5 for i in range(67)]
    yb = room_renderer.render_batch(views, intr, W, H, nl, fs)
    for i in (0, 1, 63, 64, 65, 66):
        assert np.array_equal(yb[i], room_renderer.render(views[i], intr, W, H, nl, fs[i])), i


def test_timing_reports_visible_points_and_launches(lnr, room, room_renderer):
    """lnr_get_timing after a timed batch: stage times that add up to the frame's, the
    batch's visible points (the oracle's splat count summed over the views) and the frame's
    kernel launches -- cull 3, splat 1, resolve 1, one upsample per pyramid level, then the
    FP32 U-Net's 2 (2L - 1) convs and its head for L = 3 levels."""
    s, g = room
    W, H, nl = 128, 96, 3
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 3, seed=8)
    fs = [0.5, 1.0, 1.5]
    r = room_renderer
    r.render_batch(views, intr, W, H, nl, fs)
    r.set_timing(True)
    try:
        r.render_batch(views, intr, W, H, nl, fs)
        t = r.get_timing()
    finally:
        r.set_timing(False)
    nvis = 0
    for v in views:
        vp = oracle.view_params(g, v.R, v.C)
        vis, _ = oracle.cull(g, vp, intr, W, H)
        nvis += oracle.splat(g, vp, intr, W, H, vis)[1]
    assert t["visible_points"] == nvis > 0
    assert t["kernels"] == 3 + 1 + 1 + nl + 2 * (2 * 3 - 1) + 1
    stages = [t[k] for k in ("cull", "splat", "resolve_pyramid", "upsample_pack", "unet")]
    assert all(x > 0 for x in stages)
    assert abs(sum(stages) - t["frame"]) <= 0.01


def test_device_output_and_torch_stream(lnr, room, room_renderer):
    import torch
    s, g = room
    W, H, nl, fs = 128, 128, 3, 1.0
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 1, seed=2)[0]
    out = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    room_renderer.render(view, intr, W, H, nl, fs, out=out)
    torch.cuda.synchronize()
    y = room_renderer.render(view, intr, W, H, nl, fs)
    assert np.array_equal(out.cpu().numpy(), y)


def test_unet_with_batch_norm_and_four_levels(lnr, room):
    s, g = room
    ch = (16, 32, 48, 64)
    w = synth.unet_weights(ch, seed=6, has_bn=True)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.5)
    r.set_unet(ch, w, "fp32", has_bn=True)
    W, H = 160, 120
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 1, seed=2)[0]
    ref = oracle.render(g, view, intr, W, H, 2, 1.0, w, ch, has_bn=True)
    y = r.render(view, intr, W, H, 2, 1.0)
    r.close()
    assert np.abs(y - ref["y"]).max() <= FP32_TOL


def test_edge_cases(lnr):
    # a single point; an empty view (camera facing away); exact duplicates (depth ties)
    xyz = np.array([[0.1, 0.2, 3.0]] * 5 + [[0.3, 0.1, 3.0]], np.float64)
    rgb = np.arange(18, dtype=np.uint8).reshape(6, 3)
    r = lnr.Renderer(0)
    r.load_cloud(xyz, rgb)
    r.build_grid(0.25)
    g = oracle.build_grid(xyz, rgb, None, 0.25)
    W, H = 32, 24
    intr = synth.intrinsics_for(W, H)
    for R in (np.eye(3), np.diag([-1.0, 1.0, -1.0])):
        view = synth.View(R, np.zeros(3))
        ref = oracle.render(g, view, intr, W, H, 2, 1.0)
        keys = r.render_stage(view, intr, W, H, 2, 1.0, lnr.STAGE_KEYS)
        assert np.array_equal(keys, ref["keys"])
        rgbx, D, A = r.render_stage(view, intr, W, H, 2, 1.0, lnr.STAGE_RGBDA_RAW)
        assert np.array_equal(rgbx, ref["rgb"])
    r.close()


def test_errors_are_reported(lnr, room):
    s, _ = room
    r = lnr.Renderer(0)
    intr = synth.intrinsics_for(64, 64)
    view = synth.random_poses(s, 1)[0]
    with pytest.raises(lnr.LnrError) as e:
        r.render(view, intr, 64, 64, 3, 1.0)
    assert e.value.status == -2                          # before build_grid
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.5)
    with pytest.raises(lnr.LnrError) as e:
        r.render(view, intr, 64, 64, 3, 1.0)
    assert e.value.status == -2                          # before set_unet
    r.set_unet((16, 32, 64), synth.unet_weights((16, 32, 64)), "fp32")
    bad = [dict(W=66, H=64), dict(nl=7), dict(fs=-1.0), dict(fs=float("nan"))]
    for b in bad:
        with pytest.raises(lnr.LnrError) as e:
            r.render(view, intr, b.get("W", 64), b.get("H", 64), b.get("nl", 3), b.get("fs", 1.0))
        assert e.value.status == -1
    nan_view = synth.View(view.R, np.array([np.nan, 0.0, 0.0]))
    with pytest.raises(lnr.LnrError):
        r.render(nan_view, intr, 64, 64, 3, 1.0)
    with pytest.raises(lnr.LnrError):
        r.set_unet((16, 32, 64), np.zeros(10, np.float32), "fp32")
    r.close()


def test_multiroom_geo_offset_bit_exact(lnr):
    s = synth.multiroom_scene(n_points=1_000_000)
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.25)
    W, H, nl = 480, 270, 5
    intr = synth.intrinsics_for(W, H)
    for view in synth.random_poses(s, 3):
        ref = oracle.render(g, view, intr, W, H, nl, 0.5)
        keys = r.render_stage(view, intr, W, H, nl, 0.5, lnr.STAGE_KEYS)
        assert np.array_equal(keys, ref["keys"])
        U0 = r.render_stage(view, intr, W, H, nl, 0.5, lnr.STAGE_FILTERED)
        assert np.array_equal(U0, ref["U0"])
    r.close()


def test_atomic_probe_measures_the_splat_update(lnr):
    """The z-buffer update's throughput probe runs coherent and hashed key patterns and
    rejects empty or oversized buffers."""
    r = lnr.Renderer(0)
    try:
        for coherent in (True, False):
            rate = r.probe_atomic_rate(1 << 20, 1 << 23, coherent)
            assert 1e8 < rate < 1e13, rate
        with pytest.raises(lnr.LnrError):
            r.probe_atomic_rate(0, 1 << 10)
        with pytest.raises(lnr.LnrError):
            r.probe_atomic_rate((1 << 32) + 1, 1 << 10)
    finally:
        r.close()
