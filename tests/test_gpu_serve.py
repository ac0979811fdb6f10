"""Serving: continuous batching through lnr_submit / lnr_poll.

Requests of mixed resolution, pyramid depth and filter strength are served in batches on
several streams; each result must equal the same request rendered alone (bit for bit: every
kernel treats the views of a batch independently), and admission must respect the
activation-memory budget.
"""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

CH = (16, 32, 64)


@pytest.fixture(scope="module")
def served():
    import paper_2502_11618_gb300 as lnr
    from paper_2502_11618_gb300 import build
    build.build()
    s = synth.room_scene(n_points=150_000, seed=3)
    r = lnr.Renderer(0)
    r.load_cloud(s.xyz, s.rgb, s.scan_id)
    r.build_grid(0.5)
    r.set_unet(CH, synth.unet_weights(CH, seed=1), "bf16")
    yield lnr, s, r
    r.close()


def _requests(s, n, seed=9):
    rng = np.random.default_rng(seed)
    sizes = [(128, 96), (160, 128), (96, 64)]
    views = synth.random_poses(s, n, seed=seed)
    out = []
    for i in range(n):
        W, H = sizes[rng.integers(0, 3)]
        out.append((views[i], W, H, int(rng.integers(2, 4)), float(rng.uniform(0.5, 1.5))))
    return out


def _wait(r, ticket, W, H, timeout=30.0):
    img = np.empty((H, W, 3), np.float32)
    t0 = time.time()
    while True:
        res, lat = r.poll(ticket, img)
        if res is not None:
            return res, lat
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(0.0005)


def test_served_results_equal_alone(served):
    lnr, s, r = served
    reqs = _requests(s, 24)
    alone = []
    for view, W, H, nl, fs in reqs:
        alone.append(r.render(view, synth.intrinsics_for(W, H), W, H, nl, fs))
    r.serve_start(max_batch=4, slots=3)
    try:
        tickets = [r.submit(view, synth.intrinsics_for(W, H), W, H, nl, fs) for view, W, H, nl, fs in reqs]
        for i, (t, (view, W, H, nl, fs)) in enumerate(zip(tickets, reqs)):
            img, lat = _wait(r, t, W, H)
            assert lat > 0
            assert np.array_equal(img, alone[i]), i
        st = r.serve_stats()
        assert st["done"] == len(reqs)
        assert st["launches"] < len(reqs) and st["max_batch"] > 1   # requests were batched
        assert st["peak_busy_slots"] >= 2                           # batches in flight side by side
    finally:
        r.serve_stop()


def test_admission_respects_memory_budget(served):
    """Under a budget of 2.5 requests of the largest size (measured: the buffers one such
    request alone makes a slot hold), batches shrink and slots release buffers so that the
    slots together never hold more than the budget; every request still completes."""
    lnr, s, r = served
    reqs = _requests(s, 12, seed=4)
    view = synth.random_poses(s, 1, seed=5)[0]
    r.serve_start(max_batch=4, slots=3)
    try:
        t = r.submit(view, synth.intrinsics_for(160, 128), 160, 128, 3, 1.0)
        _wait(r, t, 160, 128)
        one = r.serve_stats()["peak_alloc_bytes"]
    finally:
        r.serve_stop()
    assert one > 0
    budget = int(2.5 * one)
    r.serve_start(max_batch=4, slots=3)
    try:
        r.set_memory_budget(budget)
        tickets = [r.submit(v, synth.intrinsics_for(W, H), W, H, nl, fs) for v, W, H, nl, fs in reqs]
        for t, (v, W, H, nl, fs) in zip(tickets, reqs):
            _wait(r, t, W, H)
        st = r.serve_stats()
        assert st["done"] == len(reqs)
        assert st["peak_alloc_bytes"] <= budget, (st, budget)
        assert st["peak_act_bytes"] <= budget, (st, budget)
    finally:
        r.set_memory_budget(0)
        r.serve_stop()


def test_serving_errors(served):
    lnr, s, r = served
    view = synth.random_poses(s, 1)[0]
    intr = synth.intrinsics_for(64, 64)
    with pytest.raises(lnr.LnrError) as e:
        r.submit(view, intr, 64, 64, 2, 1.0)                 # not started
    assert e.value.status == -2
    r.serve_start(max_batch=2, slots=1)
    try:
        with pytest.raises(lnr.LnrError) as e:
            r.submit(view, intr, 66, 64, 2, 1.0)             # not a multiple of 4
        assert e.value.status == -1
        with pytest.raises(lnr.LnrError) as e:
            r.poll(12345678)
        assert e.value.status == -1
        t = r.submit(view, intr, 64, 64, 2, 1.0)
        img, lat = _wait(r, t, 64, 64)
        assert img.shape == (64, 64, 3) and 0 <= img.min() and img.max() <= 1
    finally:
        r.serve_stop()
