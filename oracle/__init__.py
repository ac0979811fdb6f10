"""CPU oracle of the per-frame render path (arXiv 2502.11618): Python view of lnr_oracle.c.

TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU-baseline leg
are the only callers.  Nothing here is imported by, or imports, the CUDA product path;
the two share nothing but the seeded input generators of the `synth` package.

Every function follows the passage named in lnr_oracle.c's header: grid and culling
(Sec. 3, "Point Cloud Projection"), the hard z-buffer splat, resolve to RGB/D/A
(Fig. 1), the depth filter (Fig. 2; Sec. 3, "Depth filtering"), the RGBDA packing and
the FP64 U-Net (Sec. 3, "U-Net Reconstruction").
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from .build import build

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        p = C.c_void_p
        L.orc_grid_dims.argtypes = [p, C.c_uint64, C.c_double, p, p]
        L.orc_grid_dims.restype = C.c_int
        L.orc_grid_build.argtypes = [p, p, p, C.c_uint64, C.c_double, p, p, p, p, p, p, p, p]
        L.orc_grid_build.restype = None
        L.orc_view_params.argtypes = [p, p, p, p, C.c_double, p, p, p, p]
        L.orc_view_params.restype = None
        L.orc_cull.argtypes = [p, p, p, p, p, C.c_int, C.c_int, p]
        L.orc_cull.restype = C.c_int64
        L.orc_splat.argtypes = [p, p, p, p, p, p, p, p, p, p, p, C.c_int, C.c_int, p]
        L.orc_splat.restype = C.c_uint64
        L.orc_soft_colours.argtypes = [p, p, p, p, p, p, p, p, p, p, p, p, C.c_int, C.c_int, p,
                                       C.c_float, p]
        L.orc_soft_colours.restype = None
        L.orc_resolve.argtypes = [p, p, C.c_int, C.c_int, p, p, p]
        L.orc_resolve.restype = None
        L.orc_minpool.argtypes = [p, C.c_int, C.c_int, p]
        L.orc_minpool.restype = None
        L.orc_upsample.argtypes = [p, C.c_int, C.c_int, p, p, C.c_float, C.c_int, p]
        L.orc_upsample.restype = None
        L.orc_filter.argtypes = [p, C.c_int, C.c_int, C.c_int, C.c_float, p]
        L.orc_filter.restype = C.c_int
        L.orc_pack_input.argtypes = [p, p, C.c_int, C.c_int, C.c_float, p]
        L.orc_pack_input.restype = None
        L.orc_unet_weight_count.argtypes = [C.c_int, p, C.c_int, C.c_int, C.c_int]
        L.orc_unet_weight_count.restype = C.c_int64
        L.orc_unet.argtypes = [p, C.c_int, C.c_int, C.c_int, p, C.c_int, C.c_int, C.c_int, p, p,
                               C.c_int]
        L.orc_unet.restype = C.c_int
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def intr_array(intr) -> np.ndarray:
    """{fx, fy, cx, cy, znear, zfar} as float32."""
    return np.array([intr.fx, intr.fy, intr.cx, intr.cy, intr.znear, intr.zfar], dtype=np.float32)


@dataclasses.dataclass
class Grid:
    cell: float
    g0: np.ndarray          # (3,) float64
    dims: np.ndarray        # (3,) int32
    cell_start: np.ndarray  # (C+1,) uint32
    order: np.ndarray       # (N,) uint32, input index at each sorted position
    ox: np.ndarray
    oy: np.ndarray
    oz: np.ndarray
    rgbs: np.ndarray        # (N,) uint32, r | g<<8 | b<<16 | scan<<24

    @property
    def n_cells(self):
        return int(np.prod(self.dims.astype(np.int64)))


def build_grid(xyz, rgb, scan_id, cell, frame=None) -> Grid:
    """Grid of the cloud; frame = (g0, dims) builds it in a given frame (another cloud's,
    e.g. the whole cloud's for a shard of it) instead of the cloud's own bounds."""
    L = lib()
    xyz = _c(xyz, np.float64)
    rgb = _c(rgb, np.uint8)
    scan = None if scan_id is None else _c(scan_id, np.uint8)
    n = xyz.shape[0]
    if frame is not None:
        g0 = _c(frame[0], np.float64).copy()
        dims = _c(frame[1], np.int32).copy()
    else:
        g0 = np.zeros(3, np.float64)
        dims = np.zeros(3, np.int32)
        if L.orc_grid_dims(_ptr(xyz), n, float(cell), _ptr(g0), _ptr(dims)) != 0:
            raise ValueError("bad cloud or cell size")
    nc = int(np.prod(dims.astype(np.int64)))
    cs = np.zeros(nc + 1, np.uint32)
    order = np.zeros(n, np.uint32)
    ox, oy, oz = (np.zeros(n, np.float32) for _ in range(3))
    rgbs = np.zeros(n, np.uint32)
    L.orc_grid_build(_ptr(xyz), _ptr(rgb), _ptr(scan), n, float(cell), _ptr(g0), _ptr(dims),
                     _ptr(cs), _ptr(order), _ptr(ox), _ptr(oy), _ptr(oz), _ptr(rgbs))
    return Grid(float(cell), g0, dims, cs, order, ox, oy, oz, rgbs)


@dataclasses.dataclass
class ViewParams:
    anchor: np.ndarray  # (3,) int32
    d0: np.ndarray      # (3,) float32
    s: np.ndarray       # (9,) float32, s[3k + r]
    Rf: np.ndarray      # (9,) float32


def view_params(grid: Grid, R, Cw) -> ViewParams:
    a = np.zeros(3, np.int32)
    d0 = np.zeros(3, np.float32)
    s = np.zeros(9, np.float32)
    Rf = np.zeros(9, np.float32)
    R = _c(R, np.float64).reshape(9)
    Cw = _c(Cw, np.float64)
    lib().orc_view_params(_ptr(R), _ptr(Cw), _ptr(grid.g0), _ptr(grid.dims), grid.cell, _ptr(a),
                          _ptr(d0), _ptr(s), _ptr(Rf))
    return ViewParams(a, d0, s, Rf)


def cull(grid: Grid, vp: ViewParams, intr, W, H):
    vis = np.zeros(grid.n_cells, np.uint8)
    ia = intr_array(intr)
    n = lib().orc_cull(_ptr(grid.dims), _ptr(vp.anchor), _ptr(vp.d0), _ptr(vp.s), _ptr(ia), W, H,
                       _ptr(vis))
    return vis, int(n)


def splat(grid: Grid, vp: ViewParams, intr, W, H, visible=None):
    keys = np.zeros(W * H, np.uint64)
    ia = intr_array(intr)
    vis = None if visible is None else _c(visible, np.uint8)
    nvis = lib().orc_splat(_ptr(vis), _ptr(grid.dims), _ptr(grid.cell_start), _ptr(grid.ox),
                           _ptr(grid.oy), _ptr(grid.oz), _ptr(vp.anchor), _ptr(vp.d0), _ptr(vp.s),
                           _ptr(vp.Rf), _ptr(ia), W, H, _ptr(keys))
    return keys, int(nvis)


def soft_colours(grid: Grid, vp: ViewParams, intr, W, H, keys, rel, visible=None):
    """Soft z-buffer colours (H, W, 3) uint8: per pixel the integer mean (rounded half up)
    of the colours of the points with z <= z_front * (1 + rel), z_front from keys."""
    rgb = np.zeros(W * H * 3, np.uint8)
    ia = intr_array(intr)
    vis = None if visible is None else _c(visible, np.uint8)
    scale = np.float32(1.0) + np.float32(rel)
    lib().orc_soft_colours(_ptr(vis), _ptr(grid.dims), _ptr(grid.cell_start), _ptr(grid.ox),
                           _ptr(grid.oy), _ptr(grid.oz), _ptr(grid.rgbs), _ptr(vp.anchor),
                           _ptr(vp.d0), _ptr(vp.s), _ptr(vp.Rf), _ptr(ia), W, H,
                           _ptr(_c(keys, np.uint64)), float(scale), _ptr(rgb))
    return rgb.reshape(H, W, 3)


def resolve(keys, rgbs, W, H):
    rgb = np.zeros(W * H * 3, np.uint8)
    D = np.zeros(W * H, np.float32)
    A = np.zeros(W * H, np.uint8)
    lib().orc_resolve(_ptr(_c(keys, np.uint64)), _ptr(_c(rgbs, np.uint32)), W, H, _ptr(rgb),
                      _ptr(D), _ptr(A))
    return rgb.reshape(H, W, 3), D.reshape(H, W), A.reshape(H, W)


def minpool(fine):
    fine = _c(fine, np.float32)
    H, W = fine.shape
    out = np.zeros(((H + 1) // 2, (W + 1) // 2), np.float32)
    lib().orc_minpool(_ptr(fine), W, H, _ptr(out))
    return out


def upsample(Mf, Mc, Uc, S, fill):
    Mf, Mc, Uc = _c(Mf, np.float32), _c(Mc, np.float32), _c(Uc, np.float32)
    H, W = Mf.shape
    out = np.zeros((H, W), np.float32)
    lib().orc_upsample(_ptr(Mf), W, H, _ptr(Mc), _ptr(Uc), float(S), int(fill), _ptr(out))
    return out


def depth_filter(D, n_levels, fs):
    """Kept depth per pixel (+inf where empty or filtered out)."""
    D = _c(D, np.float32)
    H, W = D.shape
    U0 = np.zeros((H, W), np.float32)
    if lib().orc_filter(_ptr(D), W, H, int(n_levels), float(fs), _ptr(U0)) != 0:
        raise ValueError("bad filter arguments")
    return U0


def pack_input(rgb, U0, zfar):
    rgb, U0 = _c(rgb, np.uint8), _c(U0, np.float32)
    H, W = U0.shape
    out = np.zeros((H, W, 5), np.float32)
    lib().orc_pack_input(_ptr(rgb), _ptr(U0), W, H, float(zfar), _ptr(out))
    return out


def unet_weight_count(ch, in_ch=5, out_ch=3, has_bn=False):
    chs = np.asarray(ch, np.int32)
    return int(lib().orc_unet_weight_count(len(ch), _ptr(chs), in_ch, out_ch, int(has_bn)))


def unet(x, ch, weights, in_ch=5, out_ch=3, has_bn=False, nthreads=0):
    """FP64 U-Net of one NHWC image x (H, W, in_ch) -> (H, W, out_ch) float64."""
    x = _c(x, np.float32)
    H, W, c = x.shape
    assert c == in_ch
    w = _c(weights, np.float32)
    if w.size != unet_weight_count(ch, in_ch, out_ch, has_bn):
        raise ValueError("weight count does not match the net")
    chs = np.asarray(ch, np.int32)
    out = np.zeros((H, W, out_ch), np.float64)
    if lib().orc_unet(_ptr(x), W, H, len(ch), _ptr(chs), in_ch, out_ch, int(has_bn), _ptr(w),
                      _ptr(out), int(nthreads)) != 0:
        raise ValueError("bad U-Net arguments")
    return out


def num_threads():
    return int(lib().orc_num_threads())


def training_input(D, U0, rgb, gt, zfar, unfiltered=False):
    """Network input (H, W, 5) FP32 of one synthetic training pair (Sec. 3, "Training Data
    Generation"): the projection's depth D and alpha A^s (the filter's kept mask, U0 finite)
    with the ground-truth photo gt zeroed where A^s = 0.  The unfiltered variant keeps every
    filled pixel (D finite): foreground (kept) pixels take gt, background (dropped) pixels
    the projected colour rgb / 255.  D channel z / zfar; zero where the pixel is not used."""
    D = np.asarray(D, np.float32)
    fg = np.isfinite(np.asarray(U0, np.float32))
    used = (fg | np.isfinite(D)) if unfiltered else fg
    out = np.zeros(D.shape + (5,), np.float32)
    col = np.where(fg[..., None], np.asarray(gt, np.float32),
                   np.asarray(rgb, np.uint8).astype(np.float32) / np.float32(255.0))
    out[..., :3] = np.where(used[..., None], col, np.float32(0.0))
    out[..., 3] = np.where(used, D / np.float32(zfar), np.float32(0.0))
    out[..., 4] = used.astype(np.float32)
    return out


def render(grid: Grid, view, intr, W, H, n_levels, fs, weights=None, ch=None, has_bn=False,
           brute=False, soft=0.0):
    """Every stage of one frame: keys, RGBDA before the filter, kept depth, U-Net input
    and (with weights) the FP64 output image.  soft > 0: soft z-buffer colours with
    relative depth threshold `soft`."""
    vp = view_params(grid, view.R, view.C)
    vis, nvis_cells = (None, grid.n_cells) if brute else cull(grid, vp, intr, W, H)
    keys, n_vis_points = splat(grid, vp, intr, W, H, vis)
    rgb, D, A = resolve(keys, grid.rgbs, W, H)
    if soft > 0:
        rgb = soft_colours(grid, vp, intr, W, H, keys, soft, vis)
    U0 = depth_filter(D, n_levels, fs)
    x = pack_input(rgb, U0, intr.zfar)
    out = dict(vp=vp, visible=vis, n_vis_cells=nvis_cells, n_vis_points=n_vis_points,
               keys=keys.reshape(H, W), rgb=rgb, D=D, A=A, U0=U0, x=x)
    if weights is not None:
        out["y"] = unet(x, ch, weights, has_bn=has_bn)
    return out
