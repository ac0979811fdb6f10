"""Cloud shards through the C ABI: two contexts each holding half of a cloud's cells (one
common grid frame, key positions offset into the whole cloud's order) reproduce a context
holding the whole cloud, bit for bit: the element-wise minimum of their keys, the sum of
their own-point colours, and the finished frame (filter + BF16 U-Net)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
CH = (16, 32, 64)


def shard_points(g_whole, world, rank):
    cs = g_whole.cell_start.astype(np.int64)
    n = int(cs[-1])
    lo = int(np.searchsorted(cs, n * rank // world, side="left"))
    hi = int(np.searchsorted(cs, n * (rank + 1) // world, side="left")) if rank + 1 < world else len(cs) - 1
    return np.sort(g_whole.order[cs[lo]:cs[hi]]), int(cs[lo])


@pytest.fixture(scope="module")
def setup():
    import torch
    import paper_2502_11618_gb300 as lnr
    from paper_2502_11618_gb300 import build
    build.build()
    s = synth.multiroom_scene(n_points=1_200_000)
    w = synth.unet_weights(CH, seed=1)
    whole = lnr.Renderer(0)
    whole.load_cloud(s.xyz, s.rgb, s.scan_id)
    whole.build_grid(0.25)
    whole.set_unet(CH, w, "bf16")
    g0, dims = whole.grid_info()
    gw = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    assert np.array_equal(gw.g0, g0) and np.array_equal(gw.dims, dims)
    shards = []
    for rank in range(2):
        idx, base = shard_points(gw, 2, rank)
        r = lnr.Renderer(0)
        r.load_cloud(s.xyz[idx], s.rgb[idx], s.scan_id[idx])
        r.build_grid_frame(0.25, g0, dims)
        r.set_shard(base)
        r.set_unet(CH, w, "bf16")
        shards.append(r)
    yield lnr, torch, s, whole, shards
    for r in shards + [whole]:
        r.close()


@pytest.mark.parametrize("pose", range(2))
def test_two_shards_reproduce_the_whole_cloud(setup, pose):
    lnr, torch, s, whole, shards = setup
    W, H, nl, fs = 320, 240, 3, 1.0
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 2, seed=13)[pose]
    keys = [r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_KEYS) for r in shards]
    merged = np.minimum(keys[0], keys[1])                    # the u64 min-exchange
    ref_keys = whole.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_KEYS)
    assert np.array_equal(merged, ref_keys)
    assert (keys[0] != EMPTY).any() and (keys[1] != EMPTY).any()
    kd = torch.from_numpy(merged.reshape(-1).view(np.int64).copy()).cuda()
    cols = []
    for r in shards:
        c = torch.zeros(W * H, dtype=torch.int32, device="cuda")
        r.shard_resolve(view, intr, W, H, kd, c)
        cols.append(c)
    assert not bool(((cols[0] != 0) & (cols[1] != 0)).any())   # each front point has one owner
    rgba = cols[0] + cols[1]                                    # the colour exchange
    rgb, D, A = whole.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_RGBDA_RAW)
    ref = (rgb[..., 0].astype(np.int64) | (rgb[..., 1].astype(np.int64) << 8) |
           (rgb[..., 2].astype(np.int64) << 16) | (A.astype(np.int64) << 24)).reshape(-1)
    assert np.array_equal(rgba.cpu().numpy().astype(np.int64), ref)
    y = shards[0].shard_finish(view, intr, W, H, nl, fs, kd, rgba)
    assert np.array_equal(y, whole.render(view, intr, W, H, nl, fs))


def test_shard_arguments(setup):
    lnr, torch, s, whole, shards = setup
    with pytest.raises(lnr.LnrError) as e:
        shards[0].set_shard(0xFFFFFFF0)                       # positions would pass 2^32
    assert e.value.status == -1
    with pytest.raises(lnr.LnrError) as e:
        shards[0].build_grid_frame(0.25, [0.0, 0.0, 0.0], [0, 4, 4])
    assert e.value.status == -1
