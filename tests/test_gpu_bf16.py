"""BF16 tensor-core U-Net (tcgen05 + TMA) against the CPU oracle's FP64 U-Net.

Bars: max abs error <= 2e-2 and PSNR >= 45 dB per view, outputs in [0, 1].  The
upstream stages are shared with the FP32 path and stay bit-exact (checked there).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

BF16_MAXABS = 2e-2
BF16_PSNR = 45.0


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


@pytest.fixture(scope="module")
def lnr():
    import paper_2502_11618_gb300 as p
    from paper_2502_11618_gb300 import build
    build.build()
    return p


@pytest.fixture(scope="module")
def room():
    s = synth.room_scene()
    return s, oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.5)


def _renderer(lnr, s, cell, ch, w, prec):
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(cell)
    r.set_unet(ch, w, prec)
    return r


def test_bf16_room_three_levels(lnr, room):
    s, g = room
    ch = (16, 32, 64)
    w = synth.unet_weights(ch, seed=1)
    r = _renderer(lnr, s, 0.5, ch, w, "bf16")
    W, H = 256, 256
    intr = synth.intrinsics_for(W, H)
    for view in synth.random_poses(s, 3, seed=2):
        ref = oracle.render(g, view, intr, W, H, 3, 1.0, w, ch)
        y = r.render(view, intr, W, H, 3, 1.0)
        err = np.abs(y - ref["y"]).max()
        assert 0.0 <= y.min() and y.max() <= 1.0
        assert err <= BF16_MAXABS, err
        assert psnr(y, ref["y"]) >= BF16_PSNR
    r.close()


def test_bf16_multiroom_four_levels_ragged(lnr):
    s = synth.multiroom_scene(n_points=1_000_000)
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    ch = (32, 64, 128, 256)
    w = synth.unet_weights(ch, seed=1)
    r = _renderer(lnr, s, 0.25, ch, w, "bf16")
    W, H = 328, 200            # several tiles and a ragged tail at every level
    intr = synth.intrinsics_for(W, H)
    for view in synth.random_poses(s, 2, seed=2):
        ref = oracle.render(g, view, intr, W, H, 4, 0.5, w, ch)
        y = r.render(view, intr, W, H, 4, 0.5)
        assert np.abs(y - ref["y"]).max() <= BF16_MAXABS
        assert psnr(y, ref["y"]) >= BF16_PSNR
    r.close()


def test_bf16_batch_equals_single_and_precision_switch(lnr, room):
    s, g = room
    ch = (16, 32, 64)
    w = synth.unet_weights(ch, seed=1)
    r = _renderer(lnr, s, 0.5, ch, w, "bf16")
    W, H = 128, 96
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 3, seed=4)
    yb = r.render_batch(views, intr, W, H, 3, [1.0, 0.5, 1.5])
    for i, v in enumerate(views):
        assert np.array_equal(yb[i], r.render(v, intr, W, H, 3, [1.0, 0.5, 1.5][i]))
    r.set_precision("fp32")
    y32 = r.render(views[0], intr, W, H, 3, 1.0)
    ref = oracle.render(g, views[0], intr, W, H, 3, 1.0, w, ch)
    assert np.abs(y32 - ref["y"]).max() <= 1e-4
    r.close()


_KERNEL_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import synth, oracle
import paper_2502_11618_gb300 as lnr
s = synth.multiroom_scene(n_points=300_000)
g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
ch = (32, 64, 128, 256)
w = synth.unet_weights(ch, seed=3)
r = lnr.Renderer(0); r.load_cloud(s.xyz, s.rgb, s.scan_id); r.build_grid(0.25); r.set_unet(ch, w, "bf16")
W, H = 264, 136
intr = synth.intrinsics_for(W, H)
worst = 0.0
for v in synth.random_poses(s, 2, seed=7):
    ref = oracle.render(g, v, intr, W, H, 4, 1.0, w, ch)
    y = r.render(v, intr, W, H, 4, 1.0)
    mse = float(np.mean((y - ref["y"]) ** 2))
    worst = max(worst, float(np.abs(y - ref["y"]).max()))
    assert 10 * np.log10(1 / mse) >= 45.0
print("maxabs", worst)
assert worst <= 2e-2
"""


_VARIANTS = {
    "generic": dict(LNR_CONV_KERNEL="generic"),
    "halo": dict(LNR_CONV_KERNEL="halo"),
    "halo_direct_stores": dict(LNR_CONV_KERNEL="halo", LNR_CONV_TMA_STORE="0"),
    "halo_one_staging_buffer": dict(LNR_CONV_KERNEL="halo", LNR_CONV_TMA_STORE="1"),
    "halo_4_epilogue_warps": dict(LNR_CONV_KERNEL="halo", LNR_CONV_EPI="4"),
    "halo_single_buffered_accumulators": dict(LNR_CONV_KERNEL="halo", LNR_CONV_TMEM1="1"),
    "fused_level0_encoder_2_rows": dict(LNR_CONV_FUSE0="2"),
    "fused_level0_encoder_4_rows": dict(LNR_CONV_FUSE0="4"),
    "halo_12_epilogue_warps": dict(LNR_CONV_KERNEL="halo", LNR_CONV_EPI="12"),
    "halo_12_epilogue_warps_direct_stores": dict(LNR_CONV_KERNEL="halo", LNR_CONV_EPI="12", LNR_CONV_TMA_STORE="0"),
}


@pytest.mark.parametrize("kernel", list(_VARIANTS))
def test_bf16_each_conv_kernel(lnr, kernel):
    """Every tensor-core conv variant (forced for every layer it applies to) meets the BF16
    bars: the generic kernel; the halo kernel with staged TMA stores (two or one buffers),
    with direct stores, with 4 or 12 epilogue warps, with tiles of twice the pixels whose
    accumulators fill TMEM once (single-buffered), and the fused level-0 encoder (2 or 4
    rows per tile)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **_VARIANTS[kernel])
    r = subprocess.run([sys.executable, "-c", _KERNEL_SCRIPT.format(root=root)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr


def test_bf16_autotuned_kernels_meet_the_bars(lnr):
    """After the autotuner picks a kernel per layer, the BF16 bars still hold."""
    s = synth.multiroom_scene(n_points=500_000)
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    ch = (32, 64, 128, 256)
    w = synth.unet_weights(ch, seed=2)
    r = _renderer(lnr, s, 0.25, ch, w, "bf16")
    W, H = 392, 216
    r.autotune(W, H, 2)
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(s, 2, seed=5)
    ys = r.render_batch(views, intr, W, H, 4, 1.0)
    for v, y in zip(views, ys):
        ref = oracle.render(g, v, intr, W, H, 4, 1.0, w, ch)
        assert np.abs(y - ref["y"]).max() <= BF16_MAXABS
        assert psnr(y, ref["y"]) >= BF16_PSNR
    with pytest.raises(lnr.LnrError):
        r.autotune(390, 216, 2)
    r.close()


_FUSE_SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import synth
import paper_2502_11618_gb300 as lnr
s = synth.multiroom_scene(n_points=300_000)
ch = (32, 64, 128, 256)
r = lnr.Renderer(0); r.load_cloud(s.xyz, s.rgb, s.scan_id); r.build_grid(0.25)
r.set_unet(ch, synth.unet_weights(ch, seed=3), "bf16")
W, H = 392, 216
views = synth.random_poses(s, 3, seed=8)
np.save(sys.argv[1], r.render_batch(views, synth.intrinsics_for(W, H), W, H, 4, 1.0))
"""


def test_fused_level0_encoder_equals_the_two_convs(lnr, tmp_path):
    """The fused level-0 encoder computes the same BF16 roundings in the same order as the
    two convolutions run apart (one K chunk, the same tap order per row): the frames are
    bit-identical, for 2 and 4 rows per tile, on a frame with ragged tiles."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = {}
    for tag, extra in (("apart", {}), ("fused2", {"LNR_CONV_FUSE0": "2"}), ("fused4", {"LNR_CONV_FUSE0": "4"})):
        env = {k: v for k, v in os.environ.items() if not k.startswith("LNR_CONV")}
        env.update(extra)
        path = str(tmp_path / f"{tag}.npy")
        r = subprocess.run([sys.executable, "-c", _FUSE_SCRIPT.format(root=root), path], env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stdout + r.stderr
        outs[tag] = np.load(path)
    assert np.array_equal(outs["fused2"], outs["apart"])
    assert np.array_equal(outs["fused4"], outs["apart"])
