"""Cloud shards with one u64 min-exchange of z-buffer keys, on 2 gloo ranks (CPU, oracle).

A cloud too large for one GPU is split by cells of one common grid frame: each rank
splats only its shard's points, with key positions in the whole cloud's sorted order; an
all-reduce MIN over the ranks' keys gives the whole cloud's z-buffer bit for bit, and an
all-reduce SUM of each rank's colours of its own front points gives the whole cloud's
colours.  The keys are positive int64 (float bits of z > 0 in the high word), so a signed
MIN is the unsigned one.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def shard_points(g_whole, xyz, world, rank):
    """Input indices of rank's shard (cells [lo, hi) of the whole grid, split by point
    count) and its base: the number of the whole cloud's points in the cells before lo."""
    cs = g_whole.cell_start.astype(np.int64)
    n = int(cs[-1])
    lo = int(np.searchsorted(cs, n * rank // world, side="left"))
    hi = int(np.searchsorted(cs, n * (rank + 1) // world, side="left")) if rank + 1 < world else len(cs) - 1
    idx = np.sort(g_whole.order[cs[lo]:cs[hi]])        # input order: the stable sort keeps it
    return idx, int(cs[lo])


def own_colours(keys, rgbs, base):
    """A shard's colours for the whole cloud's keys: its own front points only."""
    out = np.zeros(keys.shape, np.int64)
    full = keys != EMPTY
    pos = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64) - base
    own = full & (pos >= 0) & (pos < len(rgbs))
    out[own] = (rgbs[pos[own]].astype(np.int64) & 0xFFFFFF) | (1 << 24)
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    s = synth.room_scene(n_points=60_000, seed=5)
    W, H = 96, 80
    intr = synth.intrinsics_for(W, H)
    view = synth.random_poses(s, 1, seed=9)[0]
    whole = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.5)
    idx, base = shard_points(whole, s.xyz, world, rank)
    g = oracle.build_grid(s.xyz[idx], s.rgb[idx], s.scan_id[idx], 0.5, frame=(whole.g0, whole.dims))
    keys, _ = oracle.splat(g, oracle.view_params(g, view.R, view.C), intr, W, H)
    full = keys != EMPTY
    keys = keys.copy()
    keys[full] = (keys[full] & ~np.uint64(0xFFFFFFFF)) | ((keys[full] & np.uint64(0xFFFFFFFF)) + np.uint64(base))
    t = torch.from_numpy(keys.view(np.int64).copy())
    t[torch.from_numpy(~full)] = torch.iinfo(torch.int64).max   # empty: larger than every key
    dist.all_reduce(t, op=dist.ReduceOp.MIN)                    # the one key exchange
    merged = t.numpy().view(np.uint64).copy()
    merged[t.numpy() == np.iinfo(np.int64).max] = EMPTY
    col = torch.from_numpy(own_colours(merged, g.rgbs, base))
    dist.all_reduce(col, op=dist.ReduceOp.SUM)                  # each pixel's owner contributes
    ref_keys, _ = oracle.splat(whole, oracle.view_params(whole, view.R, view.C), intr, W, H)
    rgb, D, A = oracle.resolve(ref_keys, whole.rgbs, W, H)
    ref_col = (rgb[..., 0].astype(np.int64) | (rgb[..., 1].astype(np.int64) << 8) |
               (rgb[..., 2].astype(np.int64) << 16) | (A.astype(np.int64) << 24)).reshape(-1)
    q.put((rank, len(idx), bool(np.array_equal(merged, ref_keys)), bool(np.array_equal(col.numpy(), ref_col)),
           int(full.sum()), int((ref_keys != EMPTY).sum())))
    dist.destroy_process_group()


def test_two_shards_min_exchange_equals_whole_cloud():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, npts, keys_ok, col_ok, filled, filled_whole in res:
        assert npts > 10_000                       # both shards hold part of the cloud
        assert keys_ok and col_ok, rank
        assert 0 < filled < filled_whole           # neither shard alone covers the image
