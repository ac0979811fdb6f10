"""ctypes binding of liblnr.so (include/lnr.h): argument marshalling only.

Every step of the render path runs in the library's CUDA kernels; there is no Python or
CPU fallback.  Loading fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblnr.so")

FP32, BF16, FP8 = 0, 1, 2
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8}
STAGE_KEYS, STAGE_RGBDA_RAW, STAGE_FILTERED, STAGE_UNET_IN, STAGE_CULL = range(5)
STATUS = {0: "LNR_OK", -1: "LNR_E_ARG", -2: "LNR_E_STATE", -3: "LNR_E_OOM", -4: "LNR_E_CUDA",
          -5: "LNR_E_TIMEOUT", -6: "LNR_E_BUSY"}
E_BUSY = -6

# every entry point include/lnr.h declares
SYMBOLS = ["lnr_create", "lnr_destroy", "lnr_last_error", "lnr_load_cloud", "lnr_build_grid",
           "lnr_grid_info", "lnr_set_unet", "lnr_set_precision", "lnr_render", "lnr_render_stage",
           "lnr_render_batch", "lnr_serve_start", "lnr_serve_stop", "lnr_set_memory_budget",
           "lnr_submit", "lnr_submit_into", "lnr_poll", "lnr_serve_stats", "lnr_set_timing", "lnr_get_timing",
           "lnr_filter_static", "lnr_autotune", "lnr_calibrate", "lnr_calibrate_batch", "lnr_set_soft_zbuffer",
           "lnr_training_input", "lnr_build_grid_frame", "lnr_set_shard", "lnr_shard_resolve",
           "lnr_shard_finish", "lnr_probe_atomic_rate"]


class LnrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class View(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("C", C.c_double * 3)]


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("znear", C.c_float), ("zfar", C.c_float)]


class UnetDesc(C.Structure):
    _fields_ = [("levels", C.c_int), ("ch", C.c_int * 8), ("in_ch", C.c_int), ("out_ch", C.c_int),
                ("has_bn", C.c_int)]


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblnr.so is missing ({LIB_PATH}): build it with "
                               "paper_2502_11618_gb300.build.build() before use")
        L = C.CDLL(LIB_PATH)
        p, i, f, d, u64, sz = C.c_void_p, C.c_int, C.c_float, C.c_double, C.c_uint64, C.c_size_t
        st = C.c_int
        sig = {
            "lnr_create": ([C.POINTER(p), i, p], st),
            "lnr_destroy": ([p], st),
            "lnr_last_error": ([p], C.c_char_p),
            "lnr_load_cloud": ([p, p, p, p, u64], st),
            "lnr_build_grid": ([p, d], st),
            "lnr_grid_info": ([p, p, p], st),
            "lnr_set_unet": ([p, C.POINTER(UnetDesc), p, sz, i], st),
            "lnr_set_precision": ([p, i], st),
            "lnr_set_soft_zbuffer": ([p, f], st),
            "lnr_build_grid_frame": ([p, d, p, p], st),
            "lnr_set_shard": ([p, C.c_uint32], st),
            "lnr_shard_resolve": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, p, p], st),
            "lnr_shard_finish": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, i, f, p, p, p, i], st),
            "lnr_training_input": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, i, f, p, i, p], st),
            "lnr_render": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, i, f, p, i], st),
            "lnr_render_stage": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, i, f, i, p, i], st),
            "lnr_render_batch": ([p, i, p, p, i, i, i, p, p, i], st),
            "lnr_serve_start": ([p, i, i], st),
            "lnr_serve_stop": ([p], st),
            "lnr_set_memory_budget": ([p, sz], st),
            "lnr_submit": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, i, f, C.POINTER(u64)], st),
            "lnr_submit_into": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, i, f, p, C.POINTER(u64)], st),
            "lnr_poll": ([p, u64, p, C.POINTER(d)], st),
            "lnr_serve_stats": ([p, p], st),
            "lnr_set_timing": ([p, i], st),
            "lnr_get_timing": ([p, p], st),
            "lnr_probe_atomic_rate": ([p, u64, u64, i, C.POINTER(d)], st),
            "lnr_filter_static": ([p, i, i, i, f, p, p], st),
            "lnr_autotune": ([p, i, i, i], st),
            "lnr_calibrate": ([p, C.POINTER(View), C.POINTER(Intrinsics), i, i, i, f], st),
            "lnr_calibrate_batch": ([p, i, p, p, i, i, i, p], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def make_view(view) -> View:
    v = View()
    R = np.ascontiguousarray(view.R, dtype=np.float64).reshape(9)
    Cw = np.ascontiguousarray(view.C, dtype=np.float64).reshape(3)
    for k in range(9):
        v.R[k] = float(R[k])
    for k in range(3):
        v.C[k] = float(Cw[k])
    return v


def make_intr(intr) -> Intrinsics:
    return Intrinsics(intr.fx, intr.fy, intr.cx, intr.cy, intr.znear, intr.zfar)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t):
    """Device pointer of a tensor-like object (torch CUDA tensor), else None."""
    if hasattr(t, "data_ptr") and getattr(t, "is_cuda", False):
        return C.c_void_p(t.data_ptr())
    return None


class Renderer:
    """One lnr_ctx: a GPU, a stream, a resident cloud + grid and a U-Net."""

    def __init__(self, device: int = 0, stream=None):
        self._L = lib()
        self._c = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(stream))
        self._check(self._L.lnr_create(C.byref(self._c), int(device), s))
        self.levels = None

    def _check(self, status):
        if status != 0:
            msg = self._L.lnr_last_error(self._c).decode() if self._c else ""
            raise LnrError(status, msg)

    def close(self):
        if self._c:
            self._L.lnr_destroy(self._c)
            self._c = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- cloud, grid, network ----------------------------------------------------------
    def load_cloud(self, xyz, rgb, scan_id=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        sc = None if scan_id is None else np.ascontiguousarray(scan_id, dtype=np.uint8)
        self._check(self._L.lnr_load_cloud(self._c, _ptr(xyz), _ptr(rgb),
                                           None if sc is None else _ptr(sc), xyz.shape[0]))

    def build_grid(self, cell_size: float):
        self._check(self._L.lnr_build_grid(self._c, float(cell_size)))

    def build_grid_frame(self, cell_size, g0, dims):
        """Grid in a given frame (another context's grid_info): cloud shards share one."""
        g = np.ascontiguousarray(g0, dtype=np.float64)
        dm = np.ascontiguousarray(dims, dtype=np.int32)
        self._check(self._L.lnr_build_grid_frame(self._c, float(cell_size), _ptr(g), _ptr(dm)))

    def set_shard(self, pos_base):
        """Key positions offset by pos_base: this context holds a shard of a larger cloud."""
        self._check(self._L.lnr_set_shard(self._c, C.c_uint32(int(pos_base))))

    def shard_resolve(self, view, intr, W, H, keys_dev, rgba_dev):
        """Colours of this shard's front points for the whole cloud's keys (device tensors:
        keys uint64/int64 [H*W], rgba int32/uint32 [H*W], written)."""
        self._check(self._L.lnr_shard_resolve(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)), W, H,
                                               C.c_void_p(keys_dev.data_ptr()), C.c_void_p(rgba_dev.data_ptr())))

    def shard_finish(self, view, intr, W, H, n_levels, fs, keys_dev, rgba_dev, out=None):
        """The frame from the whole cloud's keys and colours (device tensors); (H, W, 3)."""
        host = out is None
        if host:
            out = np.empty((H, W, 3), np.float32)
        ptr = _ptr(out) if host else C.c_void_p(out.data_ptr())
        self._check(self._L.lnr_shard_finish(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)), W, H,
                                              n_levels, float(fs), C.c_void_p(keys_dev.data_ptr()),
                                              C.c_void_p(rgba_dev.data_ptr()), ptr, 0 if host else 1))
        return out

    def grid_info(self):
        g0 = np.zeros(3, np.float64)
        dims = np.zeros(3, np.int32)
        self._check(self._L.lnr_grid_info(self._c, _ptr(g0), _ptr(dims)))
        return g0, dims

    def set_unet(self, ch, weights, precision="fp32", in_ch=5, out_ch=3, has_bn=False):
        d = UnetDesc()
        d.levels = len(ch)
        for k, c in enumerate(ch):
            d.ch[k] = int(c)
        d.in_ch, d.out_ch, d.has_bn = in_ch, out_ch, int(has_bn)
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._check(self._L.lnr_set_unet(self._c, C.byref(d), _ptr(w), w.size,
                                         PRECISIONS.get(precision, precision)))
        self.levels = len(ch)

    def calibrate(self, view, intr, W, H, n_levels, fs):
        """Static E4M3 scales from BF16 frames; enables the FP8 precision.  `view` may be a
        list of views (calibrated as one batch; fs a scalar or one per view)."""
        if isinstance(view, (list, tuple)):
            n = len(view)
            va = (View * n)(*[make_view(v) for v in view])
            intrs = intr if isinstance(intr, (list, tuple)) else [intr] * n
            ia = (Intrinsics * n)(*[make_intr(k) for k in intrs])
            fsa = np.ascontiguousarray(np.broadcast_to(np.asarray(fs, np.float32), (n,)))
            self._check(self._L.lnr_calibrate_batch(self._c, n, C.cast(va, C.c_void_p), C.cast(ia, C.c_void_p),
                                                    W, H, n_levels, _ptr(fsa)))
            return
        self._check(self._L.lnr_calibrate(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)), W, H,
                                          n_levels, float(fs)))

    def autotune(self, W, H, batch=1):
        """Time every tensor-core conv configuration at (batch, W, H); keep the fastest."""
        self._check(self._L.lnr_autotune(self._c, int(W), int(H), int(batch)))

    def set_soft_zbuffer(self, rel):
        """0: hard z-buffer (default); rel > 0: soft z-buffer averaging the colours of the
        points within z_front * (1 + rel) of each pixel's front."""
        self._check(self._L.lnr_set_soft_zbuffer(self._c, float(rel)))

    def training_input(self, view, intr, W, H, n_levels, fs, gt_rgb, unfiltered=False):
        """(H, W, 5) FP32 network input of a synthetic training pair built from the
        ground-truth image gt_rgb (H, W, 3) at this view; see lnr_training_input."""
        gt = np.ascontiguousarray(gt_rgb, dtype=np.float32)
        if gt.shape != (H, W, 3):
            raise ValueError("gt_rgb must be (H, W, 3)")
        out = np.empty((H, W, 5), np.float32)
        self._check(self._L.lnr_training_input(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)),
                                               W, H, n_levels, float(fs), _ptr(gt), int(bool(unfiltered)),
                                               _ptr(out)))
        return out

    def set_precision(self, precision):
        self._check(self._L.lnr_set_precision(self._c, PRECISIONS.get(precision, precision)))

    # --- rendering ----------------------------------------------------------------------
    def render(self, view, intr, W, H, n_levels, fs, out=None):
        """One frame -> (H, W, 3) float32 in [0, 1].  `out` may be a CUDA tensor."""
        dp = _dev_ptr(out) if out is not None else None
        if dp is not None:
            self._check(self._L.lnr_render(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)),
                                           W, H, n_levels, float(fs), dp, 1))
            return out
        res = np.empty((H, W, 3), np.float32) if out is None else out
        self._check(self._L.lnr_render(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)),
                                       W, H, n_levels, float(fs), _ptr(res), 0))
        return res

    def render_batch(self, views, intrs, W, H, n_levels, fs, out=None):
        n = len(views)
        va = (View * n)(*[make_view(v) for v in views])
        if not isinstance(intrs, (list, tuple)):
            intrs = [intrs] * n
        ia = (Intrinsics * n)(*[make_intr(k) for k in intrs])
        fsa = np.ascontiguousarray(np.broadcast_to(np.asarray(fs, np.float32), (n,)))
        dp = _dev_ptr(out) if out is not None else None
        if dp is not None:
            self._check(self._L.lnr_render_batch(self._c, n, C.cast(va, C.c_void_p), C.cast(ia, C.c_void_p),
                                                 W, H, n_levels, _ptr(fsa), dp, 1))
            return out
        res = np.empty((n, H, W, 3), np.float32) if out is None else out
        self._check(self._L.lnr_render_batch(self._c, n, C.cast(va, C.c_void_p), C.cast(ia, C.c_void_p),
                                             W, H, n_levels, _ptr(fsa), _ptr(res), 0))
        return res

    def render_stage(self, view, intr, W, H, n_levels, fs, stage):
        P = W * H
        if stage == STAGE_KEYS:
            out = np.empty(P, np.uint64)
        elif stage == STAGE_RGBDA_RAW:
            out = np.empty(8 * P, np.uint8)
        elif stage == STAGE_FILTERED:
            out = np.empty(P, np.float32)
        elif stage == STAGE_UNET_IN:
            out = np.empty(P * 5, np.float32)
        elif stage == STAGE_CULL:
            out = np.empty(2, np.uint64)
        else:
            raise ValueError(stage)
        self._check(self._L.lnr_render_stage(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)),
                                             W, H, n_levels, float(fs), stage, _ptr(out), 0))
        if stage == STAGE_KEYS:
            return out.reshape(H, W)
        if stage == STAGE_RGBDA_RAW:
            raw = out.reshape(P, 8)
            D = raw[:, :4].copy().view(np.float32).reshape(H, W)
            rgb = raw[:, 4:7].reshape(H, W, 3).copy()
            A = raw[:, 7].reshape(H, W).copy()
            return rgb, D, A
        if stage == STAGE_FILTERED:
            return out.reshape(H, W)
        if stage == STAGE_UNET_IN:
            return out.reshape(H, W, 5)
        return int(out[0]), int(out[1])

    # --- serving ------------------------------------------------------------------------
    def serve_start(self, max_batch=4, slots=3):
        self._check(self._L.lnr_serve_start(self._c, max_batch, slots))

    def serve_stop(self):
        self._check(self._L.lnr_serve_stop(self._c))

    def set_memory_budget(self, nbytes):
        self._check(self._L.lnr_set_memory_budget(self._c, int(nbytes)))

    def submit(self, view, intr, W, H, n_levels, fs) -> int:
        t = C.c_uint64()
        self._check(self._L.lnr_submit(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)), W, H,
                                       n_levels, float(fs), C.byref(t)))
        return t.value

    def submit_into(self, view, intr, W, H, n_levels, fs, out) -> int:
        """Queue a request whose result goes to `out` (host, (H, W, 3) float32, kept alive
        by the caller until poll reports it done).  A page-locked `out` (e.g. a torch
        tensor from pin_memory()) receives the result straight from the device."""
        t = C.c_uint64()
        ptr = C.c_void_p(out.data_ptr()) if hasattr(out, "data_ptr") else _ptr(out)
        self._check(self._L.lnr_submit_into(self._c, C.byref(make_view(view)), C.byref(make_intr(intr)), W, H,
                                            n_levels, float(fs), ptr, C.byref(t)))
        return t.value

    def poll(self, ticket, out=None):
        """(image or None, latency_s); image None while the request is in flight."""
        lat = C.c_double()
        st = self._L.lnr_poll(self._c, C.c_uint64(ticket), None if out is None else _ptr(out), C.byref(lat))
        if st == E_BUSY:
            return None, None
        self._check(st)
        return out, lat.value

    def serve_stats(self):
        o = np.zeros(6, np.uint64)
        self._check(self._L.lnr_serve_stats(self._c, _ptr(o)))
        return dict(done=int(o[0]), launches=int(o[1]), max_batch=int(o[2]), peak_act_bytes=int(o[3]),
                    peak_alloc_bytes=int(o[4]), peak_busy_slots=int(o[5]))

    # --- measurement --------------------------------------------------------------------
    def set_timing(self, enable=True):
        self._check(self._L.lnr_set_timing(self._c, int(enable)))

    def probe_atomic_rate(self, n_slots, n_ops, coherent=True):
        """atomicMin operations per second into n_slots 64-bit keys (the splat's bound alone)."""
        r = C.c_double()
        self._check(self._L.lnr_probe_atomic_rate(self._c, C.c_uint64(n_slots), C.c_uint64(n_ops), int(coherent),
                                                  C.byref(r)))
        return r.value

    def get_timing(self):
        o = np.zeros(8, np.float64)
        self._check(self._L.lnr_get_timing(self._c, _ptr(o)))
        keys = ["cull", "splat", "resolve_pyramid", "upsample_pack", "unet", "frame", "visible_points", "kernels"]
        return dict(zip(keys, o.tolist()))
