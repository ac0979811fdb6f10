"""Seeded multi-scanner LiDAR-like scenes (the inputs the method renders).

The paper's scans are merged clouds from several static scanner positions, with gaps
where foreground occludes background, density falling with distance from the scanner
and colour offsets between scans (Section 1).  These scenes reproduce those traits by
ray casting from each scanner position: directions are uniform on the sphere band of
elevations [-60, +90] degrees, so the surface density falls as cos(theta)/r^2, and each
ray keeps only its first hit, so occluded regions stay empty.

Geometry is a closed set of axis-aligned boxes: an outer enclosure (floor, walls and
optionally a ceiling), interior walls with doorways, and furniture boxes.  Coordinates
are quantised to a 2^-12 m lattice and may be shifted by a large georeferencing offset;
both steps are exact in float64.

The heavy arithmetic runs in torch float64 on any device (CPU for small scenes, CUDA
for 20M- and 100M-point scenes); every random draw comes from a seeded numpy PCG64
generator on the host, so the result does not depend on the device.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

# Georeferencing offset (metres) applied to the large scenes: UTM-like magnitudes,
# integers, so adding it is exact in float64 and the 2^-12 lattice is preserved.
GEO_OFFSET = (512000.0, 5600000.0, 100.0)
LATTICE = 4096.0  # coordinates are multiples of 1/LATTICE metres


@dataclasses.dataclass
class Scene:
    xyz: np.ndarray          # (N, 3) float64, world coordinates
    rgb: np.ndarray          # (N, 3) uint8
    scan_id: np.ndarray      # (N,) uint8, index of the scanner that produced the point
    scanners: np.ndarray     # (S, 3) float64 scanner positions (world)
    boxes_lo: np.ndarray     # (B, 3) solid boxes (interior walls + furniture), local frame
    boxes_hi: np.ndarray
    extent: tuple            # (X, Y, Z) of the enclosure, local frame
    offset: tuple            # world = local + offset
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    def free_space(self, p_local: np.ndarray, margin: float = 0.2) -> np.ndarray:
        """True where local points are inside the enclosure and outside every solid box."""
        X, Y, Z = self.extent
        ok = (p_local[:, 0] > margin) & (p_local[:, 0] < X - margin)
        ok &= (p_local[:, 1] > margin) & (p_local[:, 1] < Y - margin)
        ok &= (p_local[:, 2] > margin) & (p_local[:, 2] < Z - margin)
        for lo, hi in zip(self.boxes_lo, self.boxes_hi):
            inside = np.all((p_local > lo - margin) & (p_local < hi + margin), axis=1)
            ok &= ~inside
        return ok


def _walls_with_doorways(rng, X, Y, Z, nrx, nry, thick=0.1, door_w=1.0, door_h=2.0):
    """Interior walls of an nrx x nry grid of rooms, each wall segment with one doorway."""
    lo, hi = [], []
    door_h = min(door_h, Z - 0.2)

    def segment(axis, pos, a0, a1):
        # wall along the other horizontal axis, between a0 and a1, at coordinate pos
        d0 = rng.uniform(a0 + 0.4, a1 - 0.4 - door_w)
        pieces = [(a0, d0, 0.0, Z), (d0 + door_w, a1, 0.0, Z), (d0, d0 + door_w, door_h, Z)]
        for s0, s1, z0, z1 in pieces:
            if s1 - s0 <= 1e-9:
                continue
            if axis == 0:
                lo.append((pos - thick / 2, s0, z0)); hi.append((pos + thick / 2, s1, z1))
            else:
                lo.append((s0, pos - thick / 2, z0)); hi.append((s1, pos + thick / 2, z1))

    for i in range(1, nrx):
        x = i * X / nrx
        for j in range(nry):
            segment(0, x, j * Y / nry, (j + 1) * Y / nry)
    for j in range(1, nry):
        y = j * Y / nry
        for i in range(nrx):
            segment(1, y, i * X / nrx, (i + 1) * X / nrx)
    return lo, hi


def _furniture(rng, X, Y, Z, n):
    lo, hi = [], []
    for _ in range(n):
        sx, sy, sz = rng.uniform(0.3, 1.5, size=3)
        sz = min(sz, Z - 0.6)
        x0 = rng.uniform(0.15, X - 0.15 - sx)
        y0 = rng.uniform(0.15, Y - 0.15 - sy)
        lo.append((x0, y0, 0.0)); hi.append((x0 + sx, y0 + sy, sz))
    return lo, hi


def _place(rng, scene_like, n, z_range, tries=100000):
    X, Y, _ = scene_like.extent
    out = []
    for _ in range(tries):
        if len(out) == n:
            break
        p = np.array([[rng.uniform(0.3, X - 0.3), rng.uniform(0.3, Y - 0.3),
                       rng.uniform(*z_range)]])
        if scene_like.free_space(p, margin=0.3)[0]:
            out.append(p[0])
    if len(out) < n:
        raise RuntimeError("could not place points in free space")
    return np.stack(out)


def _cast(origin, dirs, extent, ceiling, blo, bhi):
    """First hit of rays from `origin` along `dirs` (M,3): returns t, surface id, normal axis.

    Surface ids: 0..5 are enclosure faces (axis*2 + (1 if the max face)), 6+b is box b.
    Rays that leave through a missing ceiling get t = inf.
    """
    dev = dirs.device
    o = torch.as_tensor(origin, dtype=torch.float64, device=dev)
    d = torch.where(dirs.abs() < 1e-12, torch.full_like(dirs, 1e-12), dirs)
    inv = 1.0 / d
    ext = torch.as_tensor(extent, dtype=torch.float64, device=dev)
    # exit through the enclosure
    bound = torch.where(d > 0, ext.expand_as(d), torch.zeros_like(d))
    t_axes = (bound - o) * inv
    t_best, axis = t_axes.min(dim=1)
    face = axis * 2 + (d.gather(1, axis[:, None])[:, 0] > 0).long()
    if not ceiling:
        t_best = torch.where(face == 5, torch.full_like(t_best, math.inf), t_best)
    sid = face.clone()
    nax = axis.clone()
    B = blo.shape[0]
    for b0 in range(0, B, 16):
        lo = torch.as_tensor(blo[b0:b0 + 16], dtype=torch.float64, device=dev)
        hi = torch.as_tensor(bhi[b0:b0 + 16], dtype=torch.float64, device=dev)
        t1 = (lo[None] - o) * inv[:, None]          # (M, b, 3)
        t2 = (hi[None] - o) * inv[:, None]
        tmin = torch.minimum(t1, t2)
        tmax = torch.maximum(t1, t2)
        tnear, nearax = tmin.max(dim=2)
        tfar = tmax.min(dim=2).values
        hit = (tnear <= tfar) & (tnear > 1e-9)
        tnear = torch.where(hit, tnear, torch.full_like(tnear, math.inf))
        tb, bi = tnear.min(dim=1)
        better = tb < t_best
        t_best = torch.where(better, tb, t_best)
        sid = torch.where(better, 6 + b0 + bi, sid)
        nax = torch.where(better, nearax.gather(1, bi[:, None])[:, 0], nax)
    return t_best, sid, nax


def _scan(rng, scene, n_points, ceiling, device, chunk):
    """Ray-cast n_points hits split over the scene's scanners; returns local xyz, rgb, scan."""
    S = scene.scanners.shape[0]
    nsurf = 6 + scene.boxes_lo.shape[0]
    albedo = rng.uniform(40.0, 220.0, size=(nsurf, 3))
    scan_off = rng.integers(-8, 9, size=(S, 1)).astype(np.float64)  # U{-8..8}, one per scan
    per = [n_points // S + (1 if s < n_points % S else 0) for s in range(S)]
    albedo_t = torch.as_tensor(albedo, device=device)
    xyz_parts, rgb_parts, sid_parts = [], [], []
    zmin = math.sin(math.radians(-60.0))
    for s in range(S):
        need = per[s]
        origin = scene.scanners[s] - np.asarray(scene.offset)
        while need > 0:
            m = min(chunk, need if ceiling else int(need * 1.6) + 1024)
            z = rng.uniform(zmin, 1.0, size=m)
            az = rng.uniform(0.0, 2 * math.pi, size=m)
            noise = rng.uniform(0.95, 1.05, size=m)
            zt = torch.as_tensor(z, device=device)
            azt = torch.as_tensor(az, device=device)
            r = torch.sqrt(torch.clamp(1.0 - zt * zt, min=0.0))
            dirs = torch.stack([r * torch.cos(azt), r * torch.sin(azt), zt], dim=1)
            t, sid, nax = _cast(origin, dirs, scene.extent, ceiling, scene.boxes_lo, scene.boxes_hi)
            ok = torch.isfinite(t)
            idx = torch.nonzero(ok)[:, 0][:need]
            t, sid, nax, dirs = t[idx], sid[idx], nax[idx], dirs[idx]
            nt = torch.as_tensor(noise, device=device)[idx]
            p = torch.as_tensor(origin, device=device) + t[:, None] * dirs
            p = torch.round(p * LATTICE) / LATTICE
            # checker texture on the two in-plane axes of the hit face
            cell = torch.floor(p / 0.25).long()
            csum = cell.sum(dim=1) - cell.gather(1, nax[:, None])[:, 0]
            tex = torch.where((csum & 1) == 1, 0.82, 1.0).to(torch.float64)
            col = albedo_t[sid] * (tex * nt)[:, None] + float(scan_off[s, 0])
            col = torch.clamp(torch.round(col), 0, 255).to(torch.uint8)
            xyz_parts.append(p.cpu().numpy())
            rgb_parts.append(col.cpu().numpy())
            sid_parts.append(np.full(p.shape[0], s, dtype=np.uint8))
            need -= p.shape[0]
    xyz = np.concatenate(xyz_parts)
    return xyz, np.concatenate(rgb_parts), np.concatenate(sid_parts)


def _finish(scene, xyz_local, rgb, sid, name):
    off = np.asarray(scene.offset, dtype=np.float64)
    scene.xyz = np.ascontiguousarray(xyz_local + off)
    scene.rgb = np.ascontiguousarray(rgb)
    scene.scan_id = np.ascontiguousarray(sid)
    scene.name = name
    return scene


def room_scene(n_points=200_000, seed=0, extent=(8.0, 6.0, 3.0), n_boxes=10, n_scanners=2,
               scanner_height=1.5, offset=(0.0, 0.0, 0.0), device="cpu", chunk=1 << 18):
    """One room: floor, four walls (no ceiling), n_boxes random boxes, scanners at 1.5 m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, Z = extent
    lo, hi = _furniture(rng, X, Y, Z, n_boxes)
    sc = Scene(None, None, None, None, np.array(lo).reshape(-1, 3), np.array(hi).reshape(-1, 3),
               extent, tuple(offset))
    sc.scanners = _place(rng, sc, n_scanners, (scanner_height, scanner_height)) + np.asarray(offset)
    xyz, rgb, sid = _scan(rng, sc, n_points, ceiling=False, device=device, chunk=chunk)
    return _finish(sc, xyz, rgb, sid, f"room{n_points}")


def multiroom_scene(n_points=20_000_000, seed=0, extent=(12.0, 12.0, 4.0), rooms=(3, 3),
                    n_boxes=30, n_scanners=8, offset=GEO_OFFSET, device="cpu", chunk=1 << 20):
    """A grid of rooms with doorways, ceiling, furniture, scanners at 1.5 m (geo-offset)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, Z = extent
    wlo, whi = _walls_with_doorways(rng, X, Y, Z, rooms[0], rooms[1])
    flo, fhi = _furniture(rng, X, Y, Z, n_boxes)
    sc = Scene(None, None, None, None, np.array(wlo + flo), np.array(whi + fhi), extent,
               tuple(offset))
    sc.scanners = _place(rng, sc, n_scanners, (1.5, 1.5)) + np.asarray(offset)
    xyz, rgb, sid = _scan(rng, sc, n_points, ceiling=True, device=device, chunk=chunk)
    return _finish(sc, xyz, rgb, sid, f"multiroom{n_points}")
