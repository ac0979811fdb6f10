"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: float64 pinhole
projection from world coordinates, brute-force z-buffers, numpy stable sorts, exact
georeferencing invariance, brute-force block minima, hand-computed filter cases and
torch.nn.functional in float64.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers ----

def _tiny_cloud(n, rng, center_z=5.0, spread=2.0, lattice=4096.0):
    xyz = np.stack([rng.uniform(-spread, spread, n), rng.uniform(-spread, spread, n),
                    rng.uniform(center_z - spread, center_z + spread, n)], axis=1)
    xyz = np.round(xyz * lattice) / lattice
    rgb = rng.integers(0, 256, size=(n, 3)).astype(np.uint8)
    scan = rng.integers(0, 4, size=n).astype(np.uint8)
    return xyz, rgb, scan


def _pinhole64(xyz, R, Cw, intr):
    pc = (xyz - Cw) @ R.T
    x, y, z = pc[:, 0], pc[:, 1], pc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = intr.fx * x / z + intr.cx
        v = intr.fy * y / z + intr.cy
    return u, v, z


def _stable_pos(xyz, g):
    """Sorted position of every input point by an independent numpy stable sort."""
    ijk = np.floor((xyz - g.g0) / g.cell)
    ijk = np.clip(ijk, 0, g.dims - 1).astype(np.int64)
    cid = (ijk[:, 2] * g.dims[1] + ijk[:, 1]) * g.dims[0] + ijk[:, 0]
    order = np.argsort(cid, kind="stable")
    pos = np.empty_like(order)
    pos[order] = np.arange(len(order))
    return cid, order, pos


# ------------------------------------------------------------------- grid ----

def test_grid_is_stable_counting_sort():
    rng = np.random.default_rng(11)
    xyz, rgb, scan = _tiny_cloud(5000, rng)
    xyz[100:200] = xyz[50]            # duplicates in one cell
    g = oracle.build_grid(xyz, rgb, scan, 0.25)
    cid, order, pos = _stable_pos(xyz, g)
    assert np.array_equal(g.order, order.astype(np.uint32))
    counts = np.bincount(cid, minlength=g.n_cells)
    assert np.array_equal(np.diff(g.cell_start.astype(np.int64)), counts)
    # offsets: one FP32 rounding of the exact FP64 offset to the cell origin
    ijk = np.clip(np.floor((xyz - g.g0) / g.cell), 0, g.dims - 1)
    off64 = xyz - (g.g0 + ijk * g.cell)
    off = np.stack([g.ox, g.oy, g.oz], 1)[pos]
    assert np.array_equal(off, off64.astype(np.float32))
    assert np.all(off >= 0) and np.all(off <= g.cell)
    packed = g.rgbs[pos]
    assert np.array_equal(packed & 0xFF, rgb[:, 0])
    assert np.array_equal((packed >> 8) & 0xFF, rgb[:, 1])
    assert np.array_equal((packed >> 16) & 0xFF, rgb[:, 2])
    assert np.array_equal(packed >> 24, scan)


def test_grid_dims_cover_the_cloud():
    rng = np.random.default_rng(12)
    xyz, rgb, scan = _tiny_cloud(1000, rng)
    g = oracle.build_grid(xyz, rgb, scan, 0.5)
    assert np.all(g.g0 <= xyz.min(0)) and np.all(g.g0 + g.dims * 0.5 > xyz.max(0))
    assert np.all(g.g0 / 0.5 == np.floor(g.g0 / 0.5))


# ------------------------------------------------------------- projection ----

def test_single_points_land_on_pinhole_pixels():
    """Points on known camera rays land on the pixel the FP64 pinhole model predicts."""
    W, H = 64, 48
    intr = synth.intrinsics_for(W, H)
    R = np.eye(3)
    Cw = np.array([0.25, -0.5, 0.0])
    zs = np.array([1.0, 2.5, 7.0, 30.0])
    pts = []
    for z in zs:
        pts.append((0.0, 0.0, z))                          # optical axis -> (cx, cy)
        for k in (-3, -1, 2, 5):                           # columns at tan(angle) * z
            pts.append(((k + 0.5) / intr.fx * z, 0.0, z))
    xyz = np.array(pts) + Cw
    xyz = np.round(xyz * 4096.0) / 4096.0
    for i, p in enumerate(xyz):                            # one point per cloud: no occlusion
        g = oracle.build_grid(p[None], np.zeros((1, 3), np.uint8), None, 0.5)
        keys, n = oracle.splat(g, oracle.view_params(g, R, Cw), intr, W, H)
        u, v, z = _pinhole64(p[None], R, Cw, intr)
        hit = np.nonzero(keys != np.uint64(~np.uint64(0)))[0]
        assert len(hit) == 1
        assert hit[0] == int(math.floor(v[0])) * W + int(math.floor(u[0]))
        zbits = np.uint32(keys[hit[0]] >> np.uint64(32)).view(np.float32)
        assert abs(float(zbits) - z[0]) <= 1e-6 * z[0]


def test_random_points_match_fp64_pinhole_with_geo_offset():
    """Cell-offset FP32 projection equals the FP64 pinhole pixel away from pixel edges."""
    rng = np.random.default_rng(5)
    W, H = 160, 120
    intr = synth.intrinsics_for(W, H)
    xyz, rgb, scan = _tiny_cloud(3000, rng, center_z=6.0, spread=3.0)
    T = np.array(synth.GEO_OFFSET)
    xyz = xyz + T
    R = synth.camera.look(math.pi / 2 - 0.1, -0.05)
    Cw = T + np.array([0.3, -8.0, 6.1])
    g = oracle.build_grid(xyz, rgb, scan, 0.25)
    keys, _ = oracle.splat(g, oracle.view_params(g, R, Cw), intr, W, H)
    u, v, z = _pinhole64(xyz, R, Cw, intr)
    _, _, pos = _stable_pos(xyz, g)
    inside = (z > intr.znear) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    safe = inside & (np.abs(u - np.round(u)) > 1e-3) & (np.abs(v - np.round(v)) > 1e-3)
    pix = np.floor(v).astype(np.int64) * W + np.floor(u).astype(np.int64)
    n_checked = 0
    for i in np.nonzero(safe)[0]:
        same = np.nonzero(inside & (pix == pix[i]))[0]
        if len(same) != 1:
            continue
        n_checked += 1
        assert int(keys[pix[i]]) & 0xFFFFFFFF == pos[i]
    assert n_checked > 300


def test_zbuffer_brute_force_with_ties_and_duplicates():
    """Hard z-buffer = per-pixel minimum of (depth, sorted position) over all points."""
    rng = np.random.default_rng(7)
    W, H = 24, 20
    intr = synth.intrinsics_for(W, H)
    xyz, rgb, scan = _tiny_cloud(2000, rng, center_z=4.0, spread=1.5)
    xyz[1000:1300] = xyz[0:300]                   # exact duplicates: depth ties
    xyz[1300:1400, 2] = xyz[1400:1500, 2]         # equal depths, other positions
    R = np.eye(3)
    Cw = np.zeros(3)
    g = oracle.build_grid(xyz, rgb, scan, 0.5)
    keys, _ = oracle.splat(g, oracle.view_params(g, R, Cw), intr, W, H)
    u, v, z = _pinhole64(xyz, R, Cw, intr)
    _, _, pos = _stable_pos(xyz, g)
    inside = (z > intr.znear) & (z < intr.zfar) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    far_edge = (np.abs(u - np.round(u)) > 1e-3) & (np.abs(v - np.round(v)) > 1e-3)
    pix = np.floor(v).astype(np.int64) * W + np.floor(u).astype(np.int64)
    checked = 0
    for q in range(W * H):
        cand = np.nonzero(inside & (pix == q))[0]
        if len(cand) == 0:
            assert keys[q] == np.uint64(~np.uint64(0))
            continue
        if not far_edge[cand].all():
            continue
        zc = z[cand]
        best = cand[np.lexsort((pos[cand], zc))[0]]
        second = np.sort(np.unique(zc))
        if len(second) > 1 and (second[1] - second[0]) < 1e-5 * second[0]:
            continue                               # not resolvable in FP32
        checked += 1
        assert int(keys[q]) & 0xFFFFFFFF == pos[best]
    assert checked > 200


def _pixel_centre_point(intr, col, row, z):
    """World point (camera at the origin, identity rotation) projecting to the centre of
    pixel (col, row) at depth z."""
    return np.array([(col + 0.5 - intr.cx) / intr.fx * z, (row + 0.5 - intr.cy) / intr.fy * z, z])


def test_resolve_hand_case():
    """Resolve of a hand-written key buffer (Fig. 1; Sec. 3: the image holds the colour,
    the depth and the fill mask of each pixel's front point): a key is (float bits of z) << 32
    | sorted position; an empty key (all ones) gives RGB 0, D = +inf, A = 0; otherwise RGB is
    the point's colour (the scan byte of the packed colour is dropped), D = z and A = 1."""
    def key(z, pos):
        return (int(np.float32(z).view(np.uint32)) << 32) | pos
    empty = (1 << 64) - 1
    keys = np.array([[empty, key(2.5, 1), key(0.75, 0)],
                     [empty, key(100.0, 2), key(1e-3, 1)]], np.uint64)
    rgbs = np.array([0x07030201, 0x003264C8, 0x038000FF], np.uint32)   # (r, g, b, scan) packed
    rgb, D, A = oracle.resolve(keys, rgbs, 3, 2)
    assert rgb.tolist() == [[[0, 0, 0], [200, 100, 50], [1, 2, 3]],
                            [[0, 0, 0], [255, 0, 128], [200, 100, 50]]]
    assert A.tolist() == [[0, 1, 1], [0, 1, 1]]
    assert np.isinf(D[0, 0]) and np.isinf(D[1, 0])
    assert D[0, 1] == np.float32(2.5) and D[0, 2] == np.float32(0.75)
    assert D[1, 1] == np.float32(100.0) and D[1, 2] == np.float32(1e-3)


def test_soft_zbuffer_hand_case():
    """Soft z-buffer colours on a hand-built pixel (Sec. 3: colours of points arriving at
    similar depths are averaged): contributors are the points within z_front * (1 + rel)."""
    W, H = 64, 48
    intr = synth.intrinsics_for(W, H)
    pts = [(_pixel_centre_point(intr, 20, 10, 2.000), (10, 20, 30)),
           (_pixel_centre_point(intr, 20, 10, 2.015), (20, 40, 61)),
           (_pixel_centre_point(intr, 20, 10, 2.050), (250, 250, 250)),
           (_pixel_centre_point(intr, 40, 30, 3.000), (7, 8, 9))]
    xyz = np.round(np.array([p for p, _ in pts]) * 4096.0) / 4096.0
    rgb = np.array([c for _, c in pts], np.uint8)
    g = oracle.build_grid(xyz, rgb, None, 0.5)
    vp = oracle.view_params(g, np.eye(3), np.zeros(3))
    keys, _ = oracle.splat(g, vp, intr, W, H)
    expect = {0.0: (10, 20, 30),        # only the front point
              0.01: (15, 30, 46),       # front + 2.015 <= 2.02: (30 + 61 + 1) // 2 = 46
              0.03: (93, 103, 114)}     # all three: (280 + 1) // 3, (310 + 1) // 3, (341 + 1) // 3
    for rel, col in expect.items():
        c = oracle.soft_colours(g, vp, intr, W, H, keys, rel)
        assert tuple(int(v) for v in c[10, 20]) == col, rel
        assert tuple(int(v) for v in c[30, 40]) == (7, 8, 9)
        assert int(c.sum()) == sum(col) + 24          # every other pixel empty


def test_soft_zero_threshold_without_ties_equals_hard():
    """With rel = 0 and no two points at the same depth only the front point remains."""
    rng = np.random.default_rng(21)
    W, H = 40, 30
    intr = synth.intrinsics_for(W, H)
    n = 3000
    xyz, rgb, scan = _tiny_cloud(n, rng, center_z=4.0, spread=1.2)
    xyz[:, 2] = 3.0 + rng.permutation(n) / 4096.0          # distinct depths
    g = oracle.build_grid(xyz, rgb, scan, 0.5)
    vp = oracle.view_params(g, np.eye(3), np.zeros(3))
    keys, _ = oracle.splat(g, vp, intr, W, H)
    hard, _, A = oracle.resolve(keys, g.rgbs, W, H)
    soft = oracle.soft_colours(g, vp, intr, W, H, keys, 0.0)
    assert A.sum() > 500
    assert np.array_equal(soft, hard)


def test_soft_wide_threshold_is_mean_of_the_pixel():
    """With a threshold wider than the scene every point of a pixel contributes: the
    colour is the integer mean over the points the FP64 pinhole model puts there."""
    rng = np.random.default_rng(22)
    W, H = 32, 24
    intr = synth.intrinsics_for(W, H)
    xyz, rgb, scan = _tiny_cloud(4000, rng, center_z=4.0, spread=1.0)
    g = oracle.build_grid(xyz, rgb, scan, 0.5)
    vp = oracle.view_params(g, np.eye(3), np.zeros(3))
    keys, _ = oracle.splat(g, vp, intr, W, H)
    soft = oracle.soft_colours(g, vp, intr, W, H, keys, 1e6)
    u, v, z = _pinhole64(xyz, np.eye(3), np.zeros(3), intr)
    inside = (z > intr.znear) & (z < intr.zfar) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    far_edge = (np.abs(u - np.round(u)) > 1e-3) & (np.abs(v - np.round(v)) > 1e-3)
    pix = np.floor(v).astype(np.int64) * W + np.floor(u).astype(np.int64)
    checked = 0
    for q in range(W * H):
        cand = np.nonzero(inside & (pix == q))[0]
        if len(cand) < 2 or not far_edge[cand].all():
            continue
        n = len(cand)
        mean = (rgb[cand].astype(np.int64).sum(0) + n // 2) // n
        assert np.array_equal(soft.reshape(-1, 3)[q], mean), q
        checked += 1
    assert checked > 100


def test_training_input_hand_case():
    """Training-pair input (Sec. 3, "Training Data Generation") on four hand-built pixels:
    kept (foreground), filled but dropped (background), empty, kept."""
    inf = np.float32(np.inf)
    D = np.array([[2.0, 4.0], [inf, 10.0]], np.float32)
    U0 = np.array([[2.0, inf], [inf, 10.0]], np.float32)
    rgb = np.array([[[255, 0, 51], [102, 255, 0]], [[0, 0, 0], [1, 2, 3]]], np.uint8)
    gt = np.array([[[0.1, 0.2, 0.3], [0.4, 0.5, 0.6]], [[0.7, 0.8, 0.9], [1.0, 0.0, 0.5]]], np.float32)
    f = oracle.training_input(D, U0, rgb, gt, 100.0)
    u = oracle.training_input(D, U0, rgb, gt, 100.0, unfiltered=True)
    g32 = lambda *v: np.array(v, np.float32)
    assert np.array_equal(f[0, 0], g32(0.1, 0.2, 0.3, 0.02, 1.0))     # foreground: gt, z / zfar
    assert np.array_equal(f[0, 1], g32(0, 0, 0, 0, 0))                 # dropped: zero alpha
    assert np.array_equal(f[1, 0], g32(0, 0, 0, 0, 0))                 # empty
    assert np.array_equal(f[1, 1], g32(1.0, 0.0, 0.5, 0.1, 1.0))
    assert np.array_equal(u[0, 0], f[0, 0]) and np.array_equal(u[1, 1], f[1, 1])
    assert np.array_equal(u[0, 1], g32(0.4, 1.0, 0.0, 0.04, 1.0))      # background: point colour
    assert np.array_equal(u[1, 0], g32(0, 0, 0, 0, 0))


def test_georeferencing_offset_is_bit_exact():
    """Translating cloud and camera by a large exact offset leaves every key unchanged."""
    s = synth.room_scene(n_points=30000, seed=4)
    intr = synth.intrinsics_for(96, 64)
    T = np.array(synth.GEO_OFFSET)
    ga = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.25)
    gb = oracle.build_grid(s.xyz + T, s.rgb, s.scan_id, 0.25)
    fills = []
    for view in synth.random_poses(s, 3, seed=9):
        ka, _ = oracle.splat(ga, oracle.view_params(ga, view.R, view.C), intr, 96, 64)
        kb, _ = oracle.splat(gb, oracle.view_params(gb, view.R, view.C + T), intr, 96, 64)
        assert np.array_equal(ka, kb)
        fills.append((ka != np.uint64(~np.uint64(0))).mean())
    assert max(fills) > 0.2


# ------------------------------------------------------------------- cull ----

@pytest.mark.parametrize("which", ["room", "multiroom"])
def test_culling_never_changes_the_image(which):
    if which == "room":
        s = synth.room_scene()
        W, H, cell = 256, 256, 0.5
    else:
        s = synth.multiroom_scene(n_points=1_000_000)
        W, H, cell = 320, 180, 0.25
    intr = synth.intrinsics_for(W, H)
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, cell)
    for view in synth.random_poses(s, 3):
        vp = oracle.view_params(g, view.R, view.C)
        vis, nvis = oracle.cull(g, vp, intr, W, H)
        kc, npts = oracle.splat(g, vp, intr, W, H, vis)
        kb, nall = oracle.splat(g, vp, intr, W, H, None)
        assert np.array_equal(kc, kb)
        assert 0 < nvis < g.n_cells and npts < nall


def test_cull_rejects_cells_behind_and_beside():
    """A cell wholly behind the camera or outside the side planes is culled."""
    xyz = np.array([[0.1, 0.1, 5.1], [0.1, 0.1, -5.1], [40.1, 0.1, 5.1], [0.1, 0.1, 200.1]])
    g = oracle.build_grid(xyz, np.zeros((4, 3), np.uint8), None, 0.5)
    intr = synth.intrinsics_for(64, 64)
    vp = oracle.view_params(g, np.eye(3), np.zeros(3))
    vis, _ = oracle.cull(g, vp, intr, 64, 64)
    ijk = np.clip(np.floor((xyz - g.g0) / 0.5), 0, g.dims - 1).astype(np.int64)
    cid = (ijk[:, 2] * g.dims[1] + ijk[:, 1]) * g.dims[0] + ijk[:, 0]
    assert list(vis[cid]) == [1, 0, 0, 0]


# ----------------------------------------------------------------- filter ----

def _read_golden(name):
    blocks, cur = {}, None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            cur = blocks.setdefault(line, [])
            continue
        cur.append([float(t) for t in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def test_minpool_pyramid_never_increases_depth_and_is_block_min():
    rng = np.random.default_rng(3)
    D = rng.uniform(0.5, 20.0, size=(37, 53)).astype(np.float32)
    D[rng.random(D.shape) < 0.6] = np.inf
    M = [D]
    for _ in range(4):
        M.append(oracle.minpool(M[-1]))
    for l in range(1, 5):
        b = 1 << l
        Hc, Wc = M[l].shape
        pad = np.full((Hc * b, Wc * b), np.inf, np.float32)
        pad[:D.shape[0], :D.shape[1]] = D
        brute = pad.reshape(Hc, b, Wc, b).min(axis=(1, 3))
        assert np.array_equal(M[l], brute)
        up = np.repeat(np.repeat(M[l], 2, 0), 2, 1)[:M[l - 1].shape[0], :M[l - 1].shape[1]]
        assert np.all(up <= M[l - 1])


@pytest.mark.parametrize("name,n", [("filter_8x8_n1.txt", 1), ("filter_8x8_n2.txt", 2)])
def test_filter_hand_computed(name, n):
    g = _read_golden(name)
    D = g["depth"].astype(np.float32)
    U0 = oracle.depth_filter(D, n, 1.0)
    assert np.array_equal(np.isfinite(U0).astype(int), g["A"].astype(int))
    kept = np.isfinite(U0)
    assert np.array_equal(U0[kept], D[kept])
    if "U1" in g:
        M1 = oracle.minpool(D)
        M2 = oracle.minpool(M1)
        U1 = oracle.upsample(M1, M2, M2, np.float32(1) + np.float32(1) * np.float32(0.05), True)
        assert np.array_equal(U1, g["U1"].astype(np.float32))


def _scene_depth(W=256, H=256):
    s = synth.room_scene()
    g = oracle.build_grid(s.xyz, s.rgb, s.scan_id, 0.5)
    intr = synth.intrinsics_for(W, H)
    out = []
    for view in synth.random_poses(s, 3):
        keys, _ = oracle.splat(g, oracle.view_params(g, view.R, view.C), intr, W, H)
        out.append(oracle.resolve(keys, g.rgbs, W, H))
    return out


def test_filter_special_cases():
    dropped = 0
    for rgb, D, A in _scene_depth():
        fill = np.isfinite(D)
        assert np.array_equal(np.isfinite(oracle.depth_filter(D, 0, 1.0)), fill)
        assert np.array_equal(np.isfinite(oracle.depth_filter(D, 5, np.inf)), fill)
        prev = -1
        for fs in (0.0, 0.5, 1.0, 2.0):
            U0 = oracle.depth_filter(D, 4, fs)
            kept = np.isfinite(U0)
            assert np.all(fill[kept])                       # A is a subset of the fill mask
            assert np.array_equal(U0[kept], D[kept])        # kept depth unchanged
            assert kept.sum() >= prev                       # larger strength keeps more
            prev = kept.sum()
        dropped += fill.sum() - np.isfinite(oracle.depth_filter(D, 4, 0.0)).sum()
    assert dropped > 100


def test_filter_constant_plane_keeps_everything():
    rng = np.random.default_rng(1)
    D = np.full((64, 48), 3.25, np.float32)
    D[rng.random(D.shape) < 0.4] = np.inf
    for n in (1, 3, 5):
        for fs in (0.0, 0.5, 1.0):
            assert np.array_equal(np.isfinite(oracle.depth_filter(D, n, fs)), np.isfinite(D))


def test_filter_one_level_closed_form():
    """n = 1 brute force: edge from the 4-neighbour Laplacian of M1, reference M1 or 3x3 min."""
    rng = np.random.default_rng(2)
    for trial in range(20):
        D = rng.uniform(1.0, 10.0, size=(16, 16)).astype(np.float32)
        D[rng.random(D.shape) < 0.5] = np.inf
        fs = np.float32(rng.choice([0.0, 0.5, 1.0, 3.0]))
        S = np.float32(1) + fs * np.float32(0.05)
        M1 = D.reshape(8, 2, 8, 2).min(axis=(1, 3))
        A = np.zeros_like(D, dtype=bool)
        for y in range(16):
            for x in range(16):
                py, px = y // 2, x // 2
                d = M1[py, px]
                edge = False
                if np.isfinite(d):
                    lap = np.float32(0)
                    terms = []
                    for ny, nx in ((py, max(px - 1, 0)), (py, min(px + 1, 7)),
                                   (max(py - 1, 0), px), (min(py + 1, 7), px)):
                        nv = M1[ny, nx]
                        terms.append(np.float32(0) if not np.isfinite(nv) else np.float32(nv - d))
                    lap = np.float32(np.float32(terms[0] + terms[1]) + np.float32(terms[2] + terms[3]))
                    edge = abs(lap) > np.float32(0.1) * d
                if edge:
                    ref = M1[max(py - 1, 0):py + 2, max(px - 1, 0):px + 2].min()
                else:
                    ref = d
                A[y, x] = np.isfinite(D[y, x]) and D[y, x] <= np.float32(ref * S)
        assert np.array_equal(np.isfinite(oracle.depth_filter(D, 1, fs)), A), trial


def test_pack_input_channels():
    rgb = np.array([[[255, 0, 51], [10, 20, 30]]], np.uint8)
    U0 = np.array([[5.0, np.inf]], np.float32)
    x = oracle.pack_input(rgb, U0, 100.0)
    assert np.array_equal(x[0, 0], np.array([1.0, 0.0, np.float32(51) / np.float32(255),
                                              np.float32(5) / np.float32(100), 1.0], np.float32))
    assert np.array_equal(x[0, 1], np.zeros(5, np.float32))


# ------------------------------------------------------------------ U-Net ----

def _torch_unet(x, ch, w, in_ch=5, out_ch=3, has_bn=False):
    import torch.nn.functional as F
    shapes = synth.unet_layer_shapes(ch, in_ch, out_ch)
    wt = torch.from_numpy(w.astype(np.float64))
    off, params = 0, []
    for _, co, ci, k in shapes:
        W_ = wt[off:off + co * ci * k * k].reshape(co, ci, k, k); off += co * ci * k * k
        b_ = wt[off:off + co]; off += co
        params.append((W_, b_))
    bn = []
    if has_bn:
        for name, co, _, _ in shapes:
            if name.startswith("enc"):
                bn.append(wt[off:off + 4 * co].reshape(4, co)); off += 4 * co
    assert off == w.size
    L = len(ch)
    h = torch.from_numpy(x.astype(np.float64)).permute(2, 0, 1)[None]
    skips, i = [], 0

    def conv(h, i, bnp=None):
        y = F.conv2d(h, params[i][0], params[i][1], padding=1)
        if bnp is not None:
            y = F.batch_norm(y, bnp[2], bnp[3], bnp[0], bnp[1], training=False, eps=1e-5)
        return torch.relu(y)

    for l in range(L):
        h = conv(h, i, bn[i] if has_bn else None); i += 1
        h = conv(h, i, bn[i] if has_bn else None); i += 1
        if l < L - 1:
            skips.append(h)
            h = F.max_pool2d(h, 2)
    for l in range(L - 2, -1, -1):
        h = torch.cat([skips[l], F.interpolate(h, scale_factor=2, mode="nearest")], dim=1)
        h = conv(h, i); i += 1
        h = conv(h, i); i += 1
    y = torch.sigmoid(F.conv2d(h, params[i][0], params[i][1]))
    return y[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("ch,HW,has_bn", [((16, 32, 64), (32, 32), False),
                                           ((8, 16, 24, 32), (48, 64), False),
                                           ((16, 32, 64), (48, 32), True)])
def test_unet_fp64_matches_torch_float64(ch, HW, has_bn):
    rng = np.random.default_rng(4)
    H, W = HW
    x = rng.uniform(0, 1, size=(H, W, 5)).astype(np.float32)
    x[rng.random((H, W)) < 0.3] = 0
    w = synth.unet_weights(ch, seed=5, has_bn=has_bn)
    y = oracle.unet(x, ch, w, has_bn=has_bn)
    ref = _torch_unet(x, ch, w, has_bn=has_bn)
    assert np.max(np.abs(y - ref) / np.maximum(np.abs(ref), 1e-300)) < 1e-12
    assert 0.0 < y.min() and y.max() < 1.0


def test_unet_single_conv_hand_case():
    """A 1-level net whose convolutions are identity kernels reduces to sigmoid(b + w.x)."""
    ch = (4,)
    shapes = synth.unet_layer_shapes(ch, in_ch=5, out_ch=3)
    parts = []
    for name, co, ci, k in shapes:
        Wt = np.zeros((co, ci, k, k), np.float32)
        if k == 3:
            for c in range(min(co, ci)):
                Wt[c, c, 1, 1] = 1.0
        else:
            Wt[:, :, 0, 0] = np.arange(co * ci, dtype=np.float32).reshape(co, ci) / 8.0
        parts += [Wt.ravel(), np.zeros(co, np.float32)]
    w = np.concatenate(parts)
    x = np.random.default_rng(0).uniform(0, 1, size=(8, 8, 5)).astype(np.float32)
    y = oracle.unet(x, ch, w)
    hw = (np.arange(12, dtype=np.float64).reshape(3, 4) / 8.0)
    expect = 1.0 / (1.0 + np.exp(-(x[..., :4].astype(np.float64) @ hw.T)))
    assert np.allclose(y, expect, rtol=0, atol=1e-15)
