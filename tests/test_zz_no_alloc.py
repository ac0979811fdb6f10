"""lnr_filter_static: the depth filter for callers that may not allocate device memory.

Some callers cannot call cudaMalloc -- a host application's real-time frame loop, where an
allocation can synchronise the whole device, or a plug-in whose host owns all device
memory.  lnr_filter_static serves them: it keeps its pyramid in a fixed array inside the
library.  This test checks, through the C ABI, that two calls in a row give exactly the
kept depth of the regular path (LNR_STAGE_FILTERED of lnr_render_stage, the bit-exact bar
of the other filter tests), and that an image beyond the array's capacity is refused.
It sits in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_filter_static_matches_render_stage_twice():
    import torch

    import paper_2502_11618_gb300 as lnr
    from paper_2502_11618_gb300 import build

    build.build()
    L = lnr.lib()
    s = synth.room_scene(n_points=120_000, seed=5)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.5)
    # n_levels 0 takes the no-pyramid branch (every filled pixel kept)
    cases = [(256, 192, 3, 1.0), (320, 200, 5, 0.5), (256, 192, 0, 1.0)]
    views = synth.random_poses(s, len(cases), seed=11)
    stream = torch.cuda.current_stream().cuda_stream
    for (W, H, nl, fs), view in zip(cases, views):
        intr = synth.intrinsics_for(W, H)
        _, D, _ = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_RGBDA_RAW)
        expect = r.render_stage(view, intr, W, H, nl, fs, lnr.STAGE_FILTERED)
        d_depth = torch.from_numpy(np.ascontiguousarray(D)).cuda()
        d_kept = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
        st = L.lnr_filter_static(ctypes.c_void_p(d_depth.data_ptr()), W, H, nl, ctypes.c_float(fs),
                                 ctypes.c_void_p(d_kept.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0
        torch.cuda.synchronize()
        got = d_kept.cpu().numpy()
        assert np.array_equal(got, expect)
        assert np.isfinite(got).sum() > 0
    r.close()


def test_filter_static_refuses_images_beyond_its_capacity():
    import torch

    import paper_2502_11618_gb300 as lnr

    L = lnr.lib()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    # 4096 x 4096 needs more pyramid than the fixed array holds: refused before any launch
    assert L.lnr_filter_static(p, 4096, 4096, 6, ctypes.c_float(1.0), p, None) == -1
    assert L.lnr_filter_static(None, 64, 64, 3, ctypes.c_float(1.0), p, None) == -1
    assert L.lnr_filter_static(p, 64, 64, 3, ctypes.c_float(-1.0), p, None) == -1
