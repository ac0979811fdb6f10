"""Benchmark of the per-frame render path on the 20M-point multi-room scan at 1920x1080.

Workload (multiroom_20M): 20,000,000 seeded synthetic points (12x12x4 m, 3x3 rooms, 8
scanners, 1/r^2 density, per-scan colour offsets, georeferenced), grid cell 0.25 m,
n_levels 5, filter_strength alternating 0.5 / 1.0, 4-level U-Net 32/64/128/256 with
seeded He-init weights.  One step renders one batch of views through every stage of the
path (cull, splat, resolve + pyramid, filter, U-Net); the cloud, grid and weights are
resident in HBM before the timed region.  The grid build (once per cloud) is timed apart.

Paths:
  batched  : `--batch` views per launch, tensor-core U-Net (BF16) when the build has it,
             else FP32 -- the headline `value`;
  plain    : one view per call, FP32 U-Net -- reported beside it (`plain_fp32`).

`--impl reference` times the CPU oracle (the method as plainly written; no GPU) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s & p99 latency, 20M pts: BF16 served vs FP32 plain, 1 GB300"
W, H, NLEV, CELL = 1920, 1080, 5, 0.25
CH = (32, 64, 128, 256)
N_POINTS = 20_000_000
FS = (0.5, 1.0)
N_POSES = 16


def unet_flops_per_px(ch, in_ch=5, out_ch=3):
    """Algorithmic FLOPs of the U-Net per output pixel (2 per multiply-add)."""
    L = len(ch)
    mac = 0.0
    cin = in_ch
    for l in range(L):
        mac += (9 * cin * ch[l] + 9 * ch[l] * ch[l]) / 4 ** l
        cin = ch[l]
    for l in range(L - 2, -1, -1):
        mac += (9 * (ch[l] + ch[l + 1]) * ch[l] + 9 * ch[l] * ch[l]) / 4 ** l
    mac += ch[0] * out_ch
    return 2.0 * mac


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.dev = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_pose(i, rank, n_poses=N_POSES):
    """Pose index of view i on replica `rank`: every rank renders its own poses."""
    return (i * 7 + rank * 3) % n_poses


def aggregate(tot_ms, frames_per_rank, dist=None, device=None):
    """Whole-job throughput of independent replicas: the frames of all ranks divided by the
    slowest rank's time (max over ranks)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([tot_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    return frames_per_rank * world / (tot_ms / 1e3), tot_ms


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# DRAM traffic (read + write bytes) of all U-Net conv launches of one step of this workload
# (8 x 1080p views, BF16): ncu DRAM counters of the 13 conv launches of a 2-view step, x 4
# (scaled by the views processed).  It describes the conv kernels as captured: reported
# only while their sources are unchanged.
CONV_TRAFFIC = {"bytes_per_step": 10516.8e6,
                "sha256": {"paper_2502_11618_gb300/csrc/conv_tc.cu":
                           "7a9004f0b909af8054c3e420afef8d1cad3f622cb1e3cc30dd212568aa11f93e",
                           "paper_2502_11618_gb300/csrc/unet.cu":
                           "73ac1bad49f33b6771b5bc4f2b055aa06029aa1f464c4a4de00f1f36b4621dc2"}}


def conv_traffic():
    import hashlib
    for rel, digest in CONV_TRAFFIC["sha256"].items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return CONV_TRAFFIC["bytes_per_step"]


def make_workload(device):
    import synth
    from synth.workloads import MULTIROOM_20M, make_scene
    scene = make_scene(MULTIROOM_20M, device=device)
    views = synth.random_poses(scene, N_POSES, seed=2)
    weights = synth.unet_weights(CH, seed=1)
    return scene, views, weights


def oracle_grid(scene):
    import oracle
    return oracle.build_grid(scene.xyz, scene.rgb, scene.scan_id, CELL)


CONFIG = {"workload": "multiroom_20M", "W": W, "H": H, "n_points": N_POINTS, "views_per_step": 8,
          "n_levels": NLEV, "filter_strength": list(FS), "cell": CELL, "unet": list(CH)}


def cpu_sample(g, views, weights, crop=(480, 272)):
    """Oracle time of one 1080p frame, from a bounded sample: cull + splat + filter of a
    full view (one thread) and the FP64 U-Net on a crop (all cores), scaled by pixel count
    to the full frame.  The grid `g` is built once per cloud, outside the sample.  Returns
    the frame-rate estimate, the sample's own wall time and the fraction of a frame's work
    the sample did (by time)."""
    import oracle
    import synth
    intr = synth.intrinsics_for(W, H)
    t0 = time.perf_counter()
    ref = oracle.render(g, views[0], intr, W, H, NLEV, FS[0])
    t_raster = time.perf_counter() - t0
    cw, chh = crop
    x = ref["x"][(H - chh) // 2:(H - chh) // 2 + chh, (W - cw) // 2:(W - cw) // 2 + cw]
    t0 = time.perf_counter()
    oracle.unet(np.ascontiguousarray(x), CH, weights)
    t_crop = time.perf_counter() - t0
    t_unet = t_crop * (W * H) / (cw * chh)
    s_per_frame = t_raster + t_unet
    return {"value": 1.0 / s_per_frame, "unit": "frames/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample_s": t_raster + t_crop,
            "frames_per_sample": (t_raster + t_crop) / s_per_frame,
            "sample": (f"one 1920x1080 view: cull+splat+filter of the 20M-point scan on 1 core "
                       f"({t_raster:.2f} s) + FP64 U-Net on a {cw}x{chh} crop ({t_crop:.2f} s), "
                       f"scaled by pixel count to {t_unet:.1f} s per frame")}


def run_reference(args):
    """The oracle on the host cores, on this benchmark's workload: each step is one bounded
    sample (a whole 1080p view through cull, splat and filter; the FP64 U-Net on a crop).
    ms_per_step is the sample's measured wall time; value is the frame rate the samples give
    (frames_per_step = the fraction of a frame's work one sample does)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene, views, weights = make_workload("cpu")
    g = oracle_grid(scene)
    wall, frames = [], []
    for i in range(args.warmup + args.steps):
        r = cpu_sample(g, [views[i % len(views)]], weights)
        if i >= args.warmup:
            wall.append(r["sample_s"])
            frames.append(r["frames_per_sample"])
    v = sum(frames) / sum(wall)
    cb = {k: r[k] for k in ("unit", "cores", "kind", "sample")}
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(wall) / len(wall),
            "frames_per_step": sum(frames) / len(frames),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(CONFIG),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_accuracy(args, scene, views, weights, lnr, synth):
    """Max abs error and PSNR of each GPU precision against the oracle's FP64 U-Net (same
    bit-exact U-Net input on both sides) on `args.accuracy` 1080p views."""
    import oracle
    intr = synth.intrinsics_for(W, H)
    r = lnr.Renderer(0)
    r.load_cloud(scene.xyz, scene.rgb, scene.scan_id)
    r.build_grid(CELL)
    r.set_unet(CH, weights, "bf16")
    r.calibrate(synth.random_poses(scene, 4, seed=77), intr, W, H, NLEV, 1.0)
    g = oracle.build_grid(scene.xyz, scene.rgb, scene.scan_id, CELL)
    res = {p: {"max_abs": 0.0, "min_psnr": 1e9} for p in ("fp32", "bf16", "fp8")}
    vs = synth.random_poses(scene, args.accuracy, seed=2)
    for i, v in enumerate(vs):
        fs = FS[i % 2]
        ref = oracle.render(g, v, intr, W, H, NLEV, fs, weights, CH)["y"]
        for p in ("fp32", "bf16", "fp8"):
            r.set_precision(p)
            y = r.render(v, intr, W, H, NLEV, fs)
            d = np.abs(y.astype(np.float64) - ref)
            mse = float(np.mean(d * d))
            res[p]["max_abs"] = max(res[p]["max_abs"], float(d.max()))
            res[p]["min_psnr"] = min(res[p]["min_psnr"], 10 * np.log10(1.0 / max(mse, 1e-30)))
            res[p]["in_unit_range"] = bool(y.min() >= 0.0 and y.max() <= 1.0) and res[p].get("in_unit_range", True)
    print(json.dumps({"accuracy": res, "views": args.accuracy, "workload": "multiroom_20M", "W": W, "H": H,
                      "reference": "oracle FP64 U-Net on the bit-exact U-Net input"}), flush=True)
    r.close()


def run_sweep(args, lnr, synth):
    """Density / size sweep (the paper's output-sensitivity claim, Sec. 1, and its results figure's 10%
    decimation): the multiroom_20M scan decimated to 10..100% (seeded subset) and the
    100M-point scan, each rendered as 8 x 1080p views per step in BF16.  Per configuration:
    points, visible points per view, raster and U-Net milliseconds per step (library stage
    events), frames/s and visible points/s."""
    from synth.workloads import MULTIROOM_20M, MULTIROOM_100M, make_scene
    weights = synth.unet_weights(CH, seed=1)
    intr = synth.intrinsics_for(W, H)
    B = 8
    out = []

    def one(name, xyz, rgb, scan, views):
        r = lnr.Renderer(0)
        try:
            r.load_cloud(xyz, rgb, scan)
            r.build_grid(CELL)
            r.set_unet(CH, weights, "bf16")
            r.autotune(W, H, B)
            vis = [int(r.render_stage(v, intr, W, H, NLEV, 1.0, lnr.STAGE_CULL)[1]) for v in views[:B]]
            fs = [FS[k % 2] for k in range(B)]
            for i in range(3):
                r.render_batch(views[:B], intr, W, H, NLEV, fs)
            r.set_timing(True)
            tims = []
            for i in range(5):
                r.render_batch([views[(i + k) % len(views)] for k in range(B)], intr, W, H, NLEV, fs)
                tims.append(r.get_timing())
            r.set_timing(False)
            med = lambda k: float(np.median([t[k] for t in tims]))
            raster = med("cull") + med("splat") + med("resolve_pyramid") + med("upsample_pack")
            frame = med("frame")
            nvis = float(np.mean(vis))
            out.append({"config": name, "n_points": int(len(xyz)), "visible_points_per_view": nvis,
                        "raster_ms_per_step": raster, "splat_ms_per_step": med("splat"),
                        "unet_ms_per_step": med("unet"), "frame_ms_per_step": frame,
                        "frames_per_s": B / (frame * 1e-3),
                        "visible_points_per_s": nvis * B / (raster * 1e-3)})
        finally:
            r.close()

    s20 = make_scene(MULTIROOM_20M, device="cuda")
    views = synth.random_poses(s20, N_POSES, seed=2)
    rng = np.random.default_rng(0)
    order = rng.permutation(len(s20.xyz))
    for frac in (0.1, 0.25, 0.5, 1.0):
        keep = np.sort(order[:int(frac * len(order))])
        one(f"multiroom_20M at {int(frac * 100)}%", s20.xyz[keep], s20.rgb[keep], s20.scan_id[keep], views)
    del s20
    s100 = make_scene(MULTIROOM_100M, device="cuda")
    one("multiroom_100M", s100.xyz, s100.rgb, s100.scan_id, synth.random_poses(s100, N_POSES, seed=2))
    print(json.dumps({"sweep": out, "W": W, "H": H, "views_per_step": B, "precision": "bf16",
                      "n_levels": NLEV, "cell": CELL}), flush=True)


def run_atomic_ceiling(args, scene, views, weights, lnr):
    """The splat against its own bound: one 8-view step's z-buffer updates (one 64-bit
    atomicMin per visible point) timed inside the step, next to the same number of atomicMin
    on a fresh buffer of the step's size measured alone (coherent and hashed keys)."""
    import synth
    intr = synth.intrinsics_for(W, H)
    B = 8
    r = lnr.Renderer(0)
    try:
        r.load_cloud(scene.xyz, scene.rgb, scene.scan_id)
        r.build_grid(CELL)
        r.set_unet(CH, weights, "bf16")
        r.autotune(W, H, B)
        vis = [int(r.render_stage(v, intr, W, H, NLEV, 1.0, lnr.STAGE_CULL)[1]) for v in views[:B]]
        fs = [FS[k % 2] for k in range(B)]
        for _ in range(3):
            r.render_batch(views[:B], intr, W, H, NLEV, fs)
        r.set_timing(True)
        splat = []
        for _ in range(5):
            r.render_batch(views[:B], intr, W, H, NLEV, fs)
            splat.append(r.get_timing()["splat"])
        r.set_timing(False)
        n_ops = int(sum(vis))
        ceiling = {k: r.probe_atomic_rate(B * W * H, n_ops, k == "coherent") for k in ("coherent", "hashed")}
    finally:
        r.close()
    ms = float(np.median(splat))
    rate = n_ops / (ms * 1e-3)
    print(json.dumps({"atomic_ceiling": {"unit": "atomicMin/s", "n_ops": n_ops, "n_slots": B * W * H, **ceiling},
                      "splat": {"ms_per_step": ms, "visible_points": n_ops, "atomics_per_s": rate,
                                "frac_of_coherent": rate / ceiling["coherent"],
                                "frac_of_hashed": rate / ceiling["hashed"]},
                      "workload": "multiroom_20M", "W": W, "H": H, "views_per_step": B}), flush=True)


def spawn_replicas(n):
    """Re-run this command as n ranks, one GPU each (torch.distributed.run on 127.0.0.1);
    returns the launcher's exit status."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def run_replica_selftest(args):
    """The replica plumbing without a GPU: every rank (gloo) reports a step time of its own,
    and rank 0 prints the whole-job aggregate (frames of all ranks / slowest rank's time)."""
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    tot_ms = 10.0 * (1 + rank)
    value, slowest = aggregate(tot_ms, 8, dist if world > 1 else None, "cpu")
    if rank == 0:
        print(json.dumps({"replica_selftest": True, "world": world, "value": value, "slowest_ms": slowest}),
              flush=True)
    if world > 1:
        dist.destroy_process_group()


def stage_roofline(stage_ms, nvis, n_px, hbm_gbs):
    """HBM roofline of the raster stages from their algorithmic bytes: splat 12 B per
    visible point (FP32 offsets), resolve 28 B per pixel (key read + clear, colour gather,
    RGBDA write), filter 28 B per pixel (pyramid levels, the level-0 read and the network
    input).  stage_ms: library stage events of one step; nvis: visible points of the step."""
    parts = {"splat": (12.0 * nvis, stage_ms["splat"]),
             "splat_resolve": (12.0 * nvis + 28.0 * n_px, stage_ms["splat"] + stage_ms["resolve_pyramid"]),
             "filter": (28.0 * n_px, stage_ms["upsample_pack"])}
    out = {}
    for k, (b, ms) in parts.items():
        gbs = b / (ms * 1e-3) / 1e9
        out[k] = {"bound": "hbm", "algorithmic_bytes": b, "ms": ms, "achieved": gbs, "peak": hbm_gbs,
                  "unit": "GB/s", "frac": gbs / hbm_gbs}
    return out


def percentiles(lat_ms):
    a = np.asarray(lat_ms, np.float64)
    return {"p50": float(np.percentile(a, 50)), "p90": float(np.percentile(a, 90)), "p99": float(np.percentile(a, 99)),
            "max": float(a.max())}


_PINNED = {}   # (W, H) -> free page-locked result buffers, reused across serving runs


def serve_stream(r, lnr, synth, reqs, precision, max_batch, slots, realtime, window=48, session=True):
    """Serve `reqs` (synth.requests.Request) through lnr_submit_into / lnr_poll: at their
    arrival times when realtime, else closed loop with at most `window` requests
    outstanding.  Every result is copied by the device straight into a page-locked host
    buffer of the caller (a pool per resolution, reused once a result has been polled).
    session=False: serving is already started (and stays started).  Returns (frames/s,
    latencies in ms, serving stats of this run: requests, launches, mean batch, and the
    result buffers that had to be allocated inside the timed region)."""
    import torch
    if session:
        r.set_precision(precision)
    pools = _PINNED
    # page-locked buffers exist before the clock starts (pinning memory inside the timed
    # region would stall the client for milliseconds per buffer): `window` per resolution in
    # a closed loop; under arrivals, one per request, since past saturation every request
    # can be outstanding at once
    for key in {(q.W, q.H) for q in reqs}:
        free = pools.setdefault(key, [])
        count = sum(1 for q in reqs if (q.W, q.H) == key)
        need = count if realtime else min(window, count)
        while len(free) < need:
            free.append(torch.empty((key[1], key[0], 3), dtype=torch.float32, pin_memory=True))
    lat, pending = [], []
    allocs = [0]

    def buf(w_, h_):
        free = pools[(w_, h_)]
        if free:
            return free.pop()
        allocs[0] += 1
        return torch.empty((h_, w_, 3), dtype=torch.float32, pin_memory=True)

    if session:
        r.serve_start(max_batch=max_batch, slots=slots)
    import gc
    gc_was_enabled = gc.isenabled()
    gc.disable()    # no garbage-collector pause of the submitting client inside the timed region
    try:
        st0 = r.serve_stats()
        t0 = time.perf_counter()
        i, n = 0, len(reqs)
        while i < n or pending:
            now = time.perf_counter() - t0
            while i < n and (reqs[i].arrival_s <= now if realtime else len(pending) < window):
                q = reqs[i]
                b = buf(q.W, q.H)
                pending.append((r.submit_into(q.view, synth.intrinsics_for(q.W, q.H), q.W, q.H, q.n_levels, q.fs, b),
                                b, (q.W, q.H)))
                i += 1
            # poll every outstanding request: a batch whose results arrive late then holds
            # only its own requests, and the window keeps refilling behind it
            still = []
            for tk, b, key in pending:
                res, l = r.poll(tk)
                if l is None:
                    still.append((tk, b, key))
                else:
                    lat.append(1e3 * l)
                    pools[key].append(b)
            pending = still
        span = time.perf_counter() - t0
        st = r.serve_stats()
        nl = st["launches"] - st0["launches"]
        st = {**st, "run_requests": n, "run_launches": nl, "run_mean_batch": n / max(nl, 1),
              "run_buffer_allocs": allocs[0]}
    finally:
        if gc_was_enabled:
            gc.enable()
        if session:
            r.serve_stop()
    return n / span, lat, st


def run_100M(args, lnr, synth, torch, dev, B):
    """The 100M-point scene resident: batched BF16 at 8 x 1080p per launch (frames/s and
    visible points/s) and the mixed-resolution serving workload (a seeded Poisson stream of
    1280x720 / 1920x1080 / 2560x1440 requests, n_levels 4..6, filter_strength U[0.5, 1.5]):
    served BF16 against the plain per-request FP32 path, then the BF16 arrival rate stepped
    up to saturation."""
    from synth.requests import request_stream
    from synth.workloads import MULTIROOM_100M, make_scene
    t0 = time.perf_counter()
    scene = make_scene(MULTIROOM_100M, device=dev)
    gen_s = time.perf_counter() - t0
    weights = synth.unet_weights(CH, seed=1)
    views = synth.random_poses(scene, N_POSES, seed=2)
    intr = synth.intrinsics_for(W, H)
    stream = torch.cuda.Stream(device=dev)
    r = lnr.Renderer(dev.index, stream=stream.cuda_stream)
    res = {}
    try:
        r.load_cloud(scene.xyz, scene.rgb, scene.scan_id)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r.build_grid(CELL)
        grid_ms = 1e3 * (time.perf_counter() - t0)
        n_points = int(len(scene.xyz))
        r.set_unet(CH, weights, "bf16")
        for (w_, h_) in ((1280, 720), (1920, 1080), (2560, 1440)):
            r.autotune(w_, h_, B)
        vis = [r.render_stage(v, intr, W, H, NLEV, 1.0, lnr.STAGE_CULL)[1] for v in views]
        out = torch.empty((B, H, W, 3), dtype=torch.float32, device=dev)
        fs = [FS[k % 2] for k in range(B)]
        pick = lambda i: [views[(i * B + k) % len(views)] for k in range(B)]
        for i in range(3):
            r.render_batch(pick(i), intr, W, H, NLEV, fs, out=out)
        torch.cuda.synchronize()
        K = max(5, args.steps)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        nvis = 0
        for i in range(K):
            evs[i][0].record(stream)                 # on the library's stream
            r.render_batch(pick(3 + i), intr, W, H, NLEV, fs, out=out)
            evs[i][1].record(stream)
            nvis += sum(vis[(v_i) % len(views)] for v_i in [((3 + i) * B + k) % len(views) for k in range(B)])
        torch.cuda.synchronize()
        ms = float(np.sum([a.elapsed_time(b) for a, b in evs]))
        res["batched_100M"] = {"value": B * K / (ms * 1e-3), "unit": "frames/s", "steps": K, "views_per_step": B,
                               "ms_per_step": ms / K, "visible_points_per_s": nvis / (ms * 1e-3),
                               "visible_points_per_view": float(np.mean(vis)), "n_points": n_points,
                               "W": W, "H": H, "n_levels": NLEV, "precision": "bf16",
                               "grid_build_ms": grid_ms, "scene_generation_s": gen_s}
        del out
        # ---- mixed-resolution serving ------------------------------------------------
        # plain FP32 per request (one request per launch, one slot), closed loop then Poisson
        n_fp32 = max(60, 6 * args.steps)
        warm = request_stream(scene, 96, None, seed=7)
        serve_stream(r, lnr, synth, warm[:6], "fp32", 1, 1, False)
        fp32_fps, _, _ = serve_stream(r, lnr, synth, request_stream(scene, n_fp32, None, seed=3), "fp32", 1, 1, False)
        lam = 0.7 * fp32_fps
        n_open = max(60, int(4 * lam))
        open_reqs = request_stream(scene, n_open, lam, seed=3)
        _, f_lat, _ = serve_stream(r, lnr, synth, open_reqs, "fp32", 1, 1, True)
        # BF16 in one serving session: warm-up, closed loop, the same Poisson stream, then the
        # arrival rate stepped up to saturation
        n_bf16 = 2000
        r.set_precision("bf16")
        r.serve_start(max_batch=B, slots=3)
        try:
            serve_stream(r, lnr, synth, request_stream(scene, 400, None, seed=7), "bf16", B, 3, False, session=False)
            bf16_fps, bf16_lat, st = serve_stream(r, lnr, synth, request_stream(scene, n_bf16, None, seed=3), "bf16",
                                                  B, 3, False, session=False)
            _, b_lat, _ = serve_stream(r, lnr, synth, open_reqs, "bf16", B, 3, True, session=False)
            sweep = []
            for mult in (0.25, 0.5, 0.75, 0.9, 1.0, 1.25):
                lam_k = mult * bf16_fps
                n_k = 600
                fps_k, lat_k, st_k = serve_stream(r, lnr, synth, request_stream(scene, n_k, lam_k,
                                                                                seed=30 + int(100 * mult)),
                                                  "bf16", B, 3, True, session=False)
                sweep.append({"arrivals_per_s": lam_k, "of_closed_loop": mult, "requests": n_k,
                              "frames_per_s": fps_k, **percentiles(lat_k), "mean_batch": st_k["run_mean_batch"],
                              "buffer_allocs_timed": st_k["run_buffer_allocs"]})
            st = r.serve_stats()
        finally:
            r.serve_stop()
        res["served_mix"] = {
            "workload": "multiroom_100M resident; requests uniform over 1280x720 / 1920x1080 / 2560x1440, "
                        "n_levels uniform in 4..6, filter_strength U[0.5, 1.5], seeded poses",
            "served_bf16": {"value": bf16_fps, "unit": "frames/s", "requests": n_bf16, "closed_loop": True,
                            "max_batch": B, "slots": 3, **percentiles(bf16_lat),
                            "session_max_batch": st.get("max_batch"), "session_peak_slots_busy": st.get("peak_busy_slots")},
            "plain_fp32": {"value": fp32_fps, "unit": "frames/s", "requests": n_fp32, "closed_loop": True},
            "poisson": {"arrivals_per_s": lam, "requests": n_open, "rule": "0.7 x plain FP32 closed-loop rate",
                        "served_bf16": percentiles(b_lat), "plain_fp32": percentiles(f_lat)},
            "bf16_rate_sweep": sweep}
    finally:
        r.close()
    return res


def density_sweep(lnr, synth, torch, dev, scene, B, fractions=(0.05, 0.1, 0.25, 0.5)):
    """Output sensitivity (the paper's claim that cost follows the visible points, Sec. 1):
    the multiroom_20M scan decimated to a seeded subset of its points (1M to 10M), 8 x 1080p
    views per step, BF16; per configuration the visible points per view and per second of
    frame time, raster and U-Net time (library stage events) and frames/s."""
    weights = synth.unet_weights(CH, seed=1)
    intr = synth.intrinsics_for(W, H)
    views = synth.random_poses(scene, N_POSES, seed=2)
    order = np.random.default_rng(0).permutation(len(scene.xyz))
    out = []
    for frac in fractions:
        keep = np.sort(order[:int(frac * len(order))])
        r = lnr.Renderer(dev.index)
        try:
            r.load_cloud(scene.xyz[keep], scene.rgb[keep], scene.scan_id[keep])
            r.build_grid(CELL)
            r.set_unet(CH, weights, "bf16")
            r.autotune(W, H, B)
            fs = [FS[k % 2] for k in range(B)]
            for _ in range(3):
                r.render_batch(views[:B], intr, W, H, NLEV, fs)
            r.set_timing(True)
            tims = []
            for i in range(5):
                r.render_batch([views[(i + k) % len(views)] for k in range(B)], intr, W, H, NLEV, fs)
                tims.append(r.get_timing())
            r.set_timing(False)
        finally:
            r.close()
        med = lambda k: float(np.median([t[k] for t in tims]))
        raster = med("cull") + med("splat") + med("resolve_pyramid") + med("upsample_pack")
        nvis = float(np.mean([t["visible_points"] for t in tims]))   # per step, the library's count
        out.append({"points": int(len(keep)), "fraction": frac, "visible_points_per_view": nvis / B,
                    "visible_points_per_s": nvis / (med("frame") * 1e-3),
                    "raster_ms_per_step": raster, "splat_ms_per_step": med("splat"), "unet_ms_per_step": med("unet"),
                    "frames_per_s": B / (med("frame") * 1e-3)})
    return out


def accuracy_crops(r, lnr, synth, views, weights, precisions, crop=256, margin=64):
    """Error of each U-Net precision against the oracle's FP64 U-Net on the precision
    workload (the 16 poses at 1920x1080): per view three aligned crops (two image corners, one
    interior window), compared where the crop's cut edges are farther than the receptive
    field; max abs error and the minimum over views of the PSNR of the compared pixels."""
    import oracle
    intr = synth.intrinsics_for(W, H)
    fs = [FS[i % 2] for i in range(len(views))]
    ys = {}
    for p in precisions:
        r.set_precision(p)
        ys[p] = np.concatenate([r.render_batch(views[k:k + 8], intr, W, H, NLEV, fs[k:k + 8])
                                for k in range(0, len(views), 8)])
    res = {p: {"max_abs": 0.0, "min_psnr": 1e9, "in_unit_range": True} for p in precisions}
    for i, v in enumerate(views):
        x = r.render_stage(v, intr, W, H, NLEV, fs[i], lnr.STAGE_UNET_IN)
        exp, got = [], {p: [] for p in precisions}
        for x0, y0 in [(0, 0), (W - crop, H - crop), (832, 416)]:
            ref = oracle.unet(np.ascontiguousarray(x[y0:y0 + crop, x0:x0 + crop]), CH, weights)
            xa, ya = (0 if x0 == 0 else margin), (0 if y0 == 0 else margin)
            xb, yb = (crop if x0 + crop == W else crop - margin), (crop if y0 + crop == H else crop - margin)
            exp.append(ref[ya:yb, xa:xb].ravel())
            for p in precisions:
                got[p].append(ys[p][i][y0 + ya:y0 + yb, x0 + xa:x0 + xb].ravel())
        e = np.concatenate(exp)
        for p in precisions:
            d = np.concatenate(got[p]).astype(np.float64) - e
            res[p]["max_abs"] = max(res[p]["max_abs"], float(np.abs(d).max()))
            res[p]["min_psnr"] = min(res[p]["min_psnr"], float(10 * np.log10(1.0 / max(float(np.mean(d * d)), 1e-30))))
            res[p]["in_unit_range"] &= bool(ys[p][i].min() >= 0.0 and ys[p][i].max() <= 1.0)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-100m", action="store_true", help="skip the 100M-point batched and serving legs")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the density sweep and the accuracy summary (FP64 oracle on crops)")
    ap.add_argument("--accuracy", type=int, default=0, metavar="VIEWS",
                    help="report max abs error and PSNR of the FP32 / BF16 / FP8 U-Nets against the "
                         "oracle's FP64 U-Net on VIEWS 1080p views (slow: the oracle runs on the host)")
    ap.add_argument("--sweep", action="store_true",
                    help="density / size sweep (decimated 20M scan, 100M scan): raster and U-Net "
                         "time, frames/s and visible points/s per configuration")
    ap.add_argument("--atomic-ceiling", action="store_true",
                    help="the splat's z-buffer update rate in the step against atomicMin throughput "
                         "measured alone on a buffer of the same size")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the batched path only (no stage timing, plain, serving or CPU legs), "
                         "e.g. under a profiler")
    ap.add_argument("--replica-selftest", action="store_true",
                    help="check the multi-rank plumbing on CPU ranks (gloo); no GPU work")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_replicas(args.gpus))
    if args.replica_selftest:
        return run_replica_selftest(args)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    import synth
    import paper_2502_11618_gb300 as lnr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if args.sweep:
        return run_sweep(args, lnr, synth)
    scene, views, weights = make_workload(dev)
    if args.accuracy:
        return run_accuracy(args, scene, views, weights, lnr, synth)
    if args.atomic_ceiling:
        return run_atomic_ceiling(args, scene, views, weights, lnr)
    stream = torch.cuda.Stream(device=dev)
    r = lnr.Renderer(local, stream=stream.cuda_stream)
    r.load_cloud(scene.xyz, scene.rgb, scene.scan_id)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r.build_grid(CELL)
    grid_ms = 1e3 * (time.perf_counter() - t0)
    intr = synth.intrinsics_for(W, H)
    have_tc = True
    try:
        r.set_unet(CH, weights, "bf16")
    except lnr.LnrError:
        have_tc = False
        r.set_unet(CH, weights, "fp32")
    prec = "bf16" if have_tc else "fp32"
    B = args.batch
    t0 = time.perf_counter()
    r.autotune(W, H, B)          # per-layer conv kernel choice (outside every timed region)
    tune_s = time.perf_counter() - t0
    # every rank renders its own poses (replicas: views are independent)
    pose_idx = lambda i: replica_pose(i, rank, len(views))
    pose = lambda i: views[pose_idx(i)]
    out = torch.empty((B, H, W, 3), dtype=torch.float32, device=dev)
    nlev_run = [NLEV]

    def step(i):
        vs = [pose(i * B + k) for k in range(B)]
        fs = [FS[(i * B + k) % 2] for k in range(B)]
        r.render_batch(vs, intr, W, H, nlev_run[0], fs, out=out)

    def timed(fn, K, Wm):
        for i in range(Wm):
            fn(i)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.nvtx.range_push("timed")     # ncu captures select launches inside this range
        t0 = time.perf_counter()
        for i in range(K):
            with torch.cuda.stream(stream):
                evs[i][0].record(stream)
            fn(Wm + i)
            with torch.cuda.stream(stream):
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        if world > 1:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, wall

    # ---- headline: batched path, device-timed --------------------------------------
    clocks = Clocks(local)
    clocks.start()
    step_ms, wall = timed(step, args.steps, args.warmup)
    value, tot_ms = aggregate(float(np.sum(step_ms)), B * args.steps, dist if world > 1 else None, dev)

    if args.only_batched:
        clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                              "mode": "only-batched", "config": {"views_per_step": B, "precision": prec}}))
        r.close()
        return

    # ---- stage timing of the batched path (library stage events on its stream) -------
    def stage_times(nlev, n=3):
        """Median stage times of n timed steps, their mean visible points and the kernels
        one step launches (the library's own counts)."""
        nlev_run[0] = nlev
        r.set_timing(True)
        tims = []
        for i in range(n):
            step(i)
            torch.cuda.synchronize()
            tims.append(r.get_timing())
        r.set_timing(False)
        nlev_run[0] = NLEV
        med = {k: float(np.median([t[k] for t in tims]))
               for k in ["cull", "splat", "resolve_pyramid", "upsample_pack", "unet", "frame"]}
        return med, float(np.mean([t["visible_points"] for t in tims])), int(max(t["kernels"] for t in tims))

    stages, nvis_step, launches_per_step = stage_times(NLEV)
    stages0, _, _ = stage_times(0)
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6784.5)
    unet_ms = stages["unet"]
    flops = unet_flops_per_px(CH) * W * H * B
    if have_tc:
        peak = pk.get("bf16_tflops_sustained", 1713.8)
        roof = {"kernel": "conv3x3 tcgen05 (all U-Net conv launches of a step)", "bound": "tensor",
                "achieved": flops / (unet_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "measured (bf16_tflops_sustained)"}
    else:
        smax = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * smax * 1e6 / 1e12
        roof = {"kernel": "conv3x3 FP32 SIMT (all U-Net conv launches of a step)", "bound": "alu",
                "achieved": flops / (unet_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = conv_traffic() if have_tc else None
    roof["traffic_scope"] = ("DRAM bytes read + written by all U-Net conv launches of one step (ncu at 2 views, "
                             "scaled by the views processed)")
    roof_stages = stage_roofline(stages, nvis_step, W * H * B, hbm)
    filter_cost = {"n_levels": [0, NLEV],
                   "filter_ms_per_step": [stages0["upsample_pack"], stages["upsample_pack"]],
                   "resolve_pyramid_ms_per_step": [stages0["resolve_pyramid"], stages["resolve_pyramid"]],
                   "frame_ms_per_step": [stages0["frame"], stages["frame"]],
                   "frames_per_s": [B / (stages0["frame"] * 1e-3), B / (stages["frame"] * 1e-3)]}

    # ---- plain per-frame FP32 path (device-timed) ----------------------------------
    r.set_precision("fp32")
    out1 = torch.empty((H, W, 3), dtype=torch.float32, device=dev)

    def step_plain(i):
        r.render(pose(i), intr, W, H, NLEV, FS[i % 2], out=out1)

    plain_ms, _ = timed(step_plain, max(3, args.steps // 2), 3)
    plain_fps = 1e3 / float(np.mean(plain_ms))

    # ---- FP8 variant of the batched path (device-timed) ------------------------------
    fp8 = None
    if have_tc:
        try:
            r.calibrate(synth.random_poses(scene, 4, seed=77), intr, W, H, NLEV, 1.0)
            r.set_precision("fp8")
            r.autotune(W, H, B)
            fp8_ms, _ = timed(step, args.steps, args.warmup)
            fp8 = {"value": B * args.steps / (float(np.sum(fp8_ms)) / 1e3), "unit": "frames/s",
                   "calibration": "static per-tensor scales from 4 BF16 frames of other poses",
                   "bf16_layers": "encoder level 0 (enc0a, enc0b) and decoder levels 0-1 (dec1a, dec1b, "
                                  "dec0a, dec0b)"}
        except lnr.LnrError as e:
            fp8 = {"unavailable": str(e)}
        r.set_precision(prec)

    # ---- served paths through the public serving API (host result buffers) --------
    from synth.requests import Request

    def req_list(n, lam, seed, first):
        arr = np.zeros(n) if lam is None else np.cumsum(np.random.default_rng(seed).exponential(1.0 / lam, size=n))
        return [Request(float(arr[k]), pose(first + k), W, H, NLEV, FS[k % 2]) for k in range(n)]

    def serve_run(precision, max_batch, slots, n, lam, seed):
        """n 1080p requests (all at once when lam is None, else Poisson arrivals at rate
        lam) after a warm-up of the configuration in the same serving session; frames/s and
        latencies (ms).  The warm-up gives every slot about eight full batches, so that each
        slot's frame graphs (one per view block) are captured before the clock starts."""
        r.set_precision(precision)
        r.serve_start(max_batch=max_batch, slots=slots)
        try:
            serve_stream(r, lnr, synth, req_list(8 * max_batch * slots, None, seed, 0), precision, max_batch, slots,
                         False, session=False)
            fps, lat, st = serve_stream(r, lnr, synth, req_list(n, lam, seed, 1000), precision, max_batch, slots,
                                        lam is not None, session=False)
        finally:
            r.serve_stop()
        return fps, np.asarray(lat), st

    def serve_closed_runs(precision, max_batch, slots, n, runs, seed):
        """`runs` closed-loop runs of n 1080p requests in one warmed serving session (as a
        server runs: slots, buffers and frame graphs stay between requests)."""
        r.set_precision(precision)
        r.serve_start(max_batch=max_batch, slots=slots)
        try:
            serve_stream(r, lnr, synth, req_list(8 * max_batch * slots, None, seed, 0), precision, max_batch, slots,
                         False, session=False)
            return [serve_stream(r, lnr, synth, req_list(n, None, seed + k, 1000 + n * k), precision, max_batch, slots,
                                 False, session=False) for k in range(runs)]
        finally:
            r.serve_stop()

    lam = 0.7 * plain_fps                      # both paths stable at this arrival rate
    n_open = max(40, int(3 * lam))             # about 3 s of arrivals
    prec_fast = "bf16" if have_tc else "fp32"
    # closed loop: 640 requests, 48 outstanding at a time (about 0.4 s of work), median of
    # five runs in one serving session; measured before the legs that load the host cores
    srv = serve_closed_runs(prec_fast, 8, 3, 16 * max(40, args.steps), 5, 11)
    srv_runs = [x[0] for x in srv]
    srv_fps = float(np.median(srv_runs))
    _, srv_lat, _ = serve_run(prec_fast, 8, 3, n_open, lam, 12)
    plain_srv_fps, _, _ = serve_run("fp32", 1, 1, max(10, args.steps), None, 13)
    _, plain_lat, _ = serve_run("fp32", 1, 1, n_open, lam, 12)
    clk = clocks.stop()
    r.set_precision(prec)
    e2e = {"value": srv_fps, "unit": "frames/s",
           "path": "serving API (lnr_submit_into / lnr_poll), BF16, closed loop with 48 requests outstanding, "
                   "median of 5 runs in one serving session, "
                   "results copied by the device into page-locked host buffers of the caller",
           "h2d_bytes_per_step": 96 + 24 + 4, "d2h_bytes_per_step": W * H * 3 * 4, "step": "one request",
           "runs": [round(float(x), 1) for x in srv_runs], "requests_per_run": 16 * max(40, args.steps),
           "peak_slots_busy": max(x[2].get("peak_busy_slots") or 0 for x in srv)}

    # ---- accuracy of every precision on the precision workload (16 views, crops) -----
    accuracy = None
    if have_tc and rank == 0 and not args.no_extras and fp8 and "value" in fp8:
        accuracy = accuracy_crops(r, lnr, synth, views, weights, ("fp32", "bf16", "fp8"))
        accuracy["views"] = len(views)
        accuracy["compared"] = ("three 256x256 crops per view (two corners, one interior) against the oracle's "
                                "FP64 U-Net on the bit-exact U-Net input, 64-px margins at cut edges")
        r.set_precision(prec)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(oracle_grid(scene), views, weights)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
    r.close()
    sweep = None
    if have_tc and rank == 0 and world == 1 and not args.no_extras:
        sweep = density_sweep(lnr, synth, torch, dev, scene, B)
        sweep.append({"points": N_POINTS, "fraction": 1.0, "visible_points_per_view": nvis_step / B,
                      "visible_points_per_s": nvis_step / (stages["frame"] * 1e-3),
                      "raster_ms_per_step": stages["cull"] + stages["splat"] + stages["resolve_pyramid"] +
                      stages["upsample_pack"], "splat_ms_per_step": stages["splat"],
                      "unet_ms_per_step": stages["unet"], "frames_per_s": B / (stages["frame"] * 1e-3)})
    del scene

    big = {}
    if have_tc and not args.no_100m and world == 1:
        big = run_100M(args, lnr, synth, torch, dev, B)

    if rank == 0:
        cfg = dict(CONFIG)
        cfg.update({"views_per_step": B, "precision": prec, "parallelism": f"replicas{world}",
                    "l2": "inputs larger than L2: per-step working set > 1 GB, every step new poses"})
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if have_tc else "f32", "data": "synthetic",
            "config": cfg,
            "latency_ms": {"batched_step": percentiles(step_ms),
                           "served_bf16": {**percentiles(srv_lat), "arrivals_per_s": lam, "requests": int(n_open)},
                           "plain_fp32": {**percentiles(plain_lat), "arrivals_per_s": lam, "requests": int(n_open)}},
            "plain_fp32": {"value": plain_fps, "unit": "frames/s", "served_value": plain_srv_fps},
            "served_bf16": {"value": srv_fps, "unit": "frames/s"},
            "batched_fp8": fp8,
            "stages_ms_per_batch": {k: round(v, 4) for k, v in stages.items()},
            "visible_points_per_step": nvis_step,
            "roofline_stages": roof_stages,
            "filter_cost": filter_cost,
            "accuracy_16_views": accuracy,
            "density_sweep": sweep,
            "grid_build_ms": grid_ms,
            "autotune_s": tune_s,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches_per_step * args.steps,
            "wall_s_timed": wall,
            **big,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
