"""Benchmark: one step = the whole hot path on one image pair of the oriented and
scaled workload (two 1920x1080 images, 10,000 keypoints each over 32 angle bins
and 3 scales): extract both descriptor sets, then match 10,000 x 10,000 top-2
with the 0.8 ratio test.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--path auto|popc|tensor]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Under torchrun each rank runs its own replica of the pair (independent pairs, no
collective on the data path); rank 0 prints units of all ranks / max-over-ranks
time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LATCH descriptors/s + Hamming Gpairs/s (bit-exact); serve p50/p99 latency"
WORKLOAD = "oriented_scaled_1920x1080_10k"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="latch", choices=["latch", "reference"])
    p.add_argument("--path", default="auto", choices=["auto", "popc", "tensor"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrivals per second")
    p.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    p.add_argument("--workload", default="pair", choices=["pair", "gallery", "sfm_batch", "serve"],
                   help="pair: the default one-pair step; gallery: 16,384 x 1,048,576 matching; "
                        "sfm_batch: 64 images x 476 neighbour pairs, batched vs one call per image / pair")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"latch_clocks_gpu{self.gpu}_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


def max_over_ranks(x: float, ws: int, device) -> float:
    """Largest value of x over the ranks (the job's time is its slowest rank's)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, seconds: float) -> float:
    """Units processed by all ranks (each runs its own replica) per second of the
    slowest rank."""
    return ws * units_per_rank / seconds


def _workload():
    from paper_1609_03986_gb300 import synth
    return synth.pair(WORKLOAD)


# ------------------------------------------------------------------ CPU oracle timing

def _oracle_train(wl):
    """The oracle's descriptors of the second image (the train set), computed once."""
    import oracle
    from paper_1609_03986_gb300 import synth
    return oracle.extract(wl["images"][1], wl["width"], wl["height"], wl["kps"][1], wl["triplets"], synth.SCALES)


def _oracle_rates(wl, train, n_extract: int, n_match: int, offset: int = 0):
    """Time the oracle (single-threaded C) on a bounded sample: seconds per
    descriptor extracted and per query matched against the full train set."""
    import oracle
    from paper_1609_03986_gb300 import synth
    img, kps = wl["images"][0], wl["kps"][0]
    sel = (np.arange(n_extract) + offset) % len(kps)
    t0 = time.perf_counter()
    d0 = oracle.extract(img, wl["width"], wl["height"], kps[sel], wl["triplets"], synth.SCALES)
    t1 = time.perf_counter()
    oracle.match(d0[:n_match], train, 2, 0.8)
    t2 = time.perf_counter()
    return (t1 - t0) / n_extract, (t2 - t1) / n_match


def _cpu_step_seconds(wl, per_desc, per_query):
    n0, n1 = len(wl["kps"][0]), len(wl["kps"][1])
    return per_desc * (n0 + n1) + per_query * n0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = _workload()
    n_desc = len(wl["kps"][0]) + len(wl["kps"][1])
    train = _oracle_train(wl)
    # warm-up and timed steps, each a bounded sample scaled to one full step
    times = []
    for i in range(args.warmup + args.steps):
        per_desc, per_query = _oracle_rates(wl, train, 50, 3, offset=50 * i)
        if i >= args.warmup:
            times.append(_cpu_step_seconds(wl, per_desc, per_query))
    step_s = statistics.mean(times)
    value = n_desc / step_s
    line = {
        "metric": METRIC, "value": value, "unit": "descriptors/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "images": "2 x 1920x1080 u8", "keypoints_per_image": 10000,
                   "angle_bins": 32, "scales": [1.0, 1.5, 2.25], "match": "10000 x 10000 top-2 ratio 0.8"},
        "cpu_baseline": {"value": value, "unit": "descriptors/s", "cores": 1, "kind": "oracle",
                         "sample": "per step: 50 descriptors extracted + 3 queries matched against the 10,000 "
                                   "train descriptors, single-threaded C oracle, scaled to the full step "
                                   "(20,000 descriptors extracted + 10,000 queries matched)"},
        "e2e": {"value": value, "unit": "descriptors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm

def run_latch(args):
    import torch
    import torch.distributed as dist

    import paper_1609_03986_gb300 as P

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    path = {"auto": P.PATH_AUTO, "popc": P.PATH_POPC, "tensor": P.PATH_TENSOR}[args.path]

    wl = _workload()
    w, h = wl["width"], wl["height"]
    ctx = P.Context(local, triplets=wl["triplets"])
    n0, n1 = len(wl["kps"][0]), len(wl["kps"][1])
    tuning = P.latch_autotune(ctx.handle, w, h, max(n0, n1), n0, n1)  # tile shapes / path, measured here
    P.latch_reserve(ctx.handle, max(n0, n1), n0, n1)
    imgs_h = [torch.from_numpy(im).pin_memory() for im in wl["images"]]
    kps_h = torch.from_numpy(np.concatenate([P.pack_keypoints(k) for k in wl["kps"]])).pin_memory()
    imgs = [t.to(dev) for t in imgs_h]
    kps = kps_h.to(dev)
    desc = torch.empty((n0 + n1, 64), dtype=torch.uint8, device=dev)
    matches = torch.empty((n0, 16), dtype=torch.uint8, device=dev)
    matches_h = torch.empty((n0, 16), dtype=torch.uint8).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    s = int(stream.cuda_stream)
    # the pair as a batch of 2 images and 1 pair: both images bucketed and extracted
    # in one launch each, descriptors expanded once, one match launch
    batch = P.BatchDesc([(t, w, h, t.stride(0)) for t in imgs], [n0, n1], kps, desc, [(0, 1)], 2, 0.8, matches)
    P.latch_reserve_batch(ctx.handle, batch)
    if path != P.PATH_AUTO and path != P.PATH_TENSOR:
        raise SystemExit("the batched step matches on the tensor cores; use --path auto|tensor")

    def step():
        P.latch_batch_run(ctx.handle, batch, s)

    def plain_step():
        P.latch_extract(ctx.handle, imgs[0], w, h, imgs[0].stride(0), kps[:n0], n0, None, desc[:n0], s)
        P.latch_extract(ctx.handle, imgs[1], w, h, imgs[1].stride(0), kps[n0:], n1, None, desc[n0:], s)
        P.hamming_match(ctx.handle, desc[:n0], n0, desc[n0:], n1, 2, 0.8, matches, P.PATH_TENSOR, s)

    # end to end through the C ABI from pinned host memory: latch_batch_run_host
    # uploads the images and keypoints, runs the batch and downloads the matches;
    # consecutive calls overlap (the uploads of step i+1 run during step i's kernels)
    host_batch = P.HostBatchDesc([(t, w, h, t.stride(0)) for t in imgs_h], [n0, n1], kps_h, None, [(0, 1)], 2, 0.8,
                                 matches_h)

    def e2e_step():
        P.latch_batch_run_host(ctx.handle, host_batch, s)

    # correctness gate: the batched step gives the bytes of the plain calls
    plain_step()
    ref = (desc.clone(), matches.clone())
    step()
    torch.cuda.synchronize()
    ctx.check()
    if not (torch.equal(ref[0], desc) and torch.equal(ref[1], matches)):
        raise SystemExit("batched and plain results differ")

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clocks.start()
    time.sleep(0.5)  # let the sampler take its first readings
    launches0 = P.latch_kernel_launches()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the step's events)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall1 = time.perf_counter()
    launches = P.latch_kernel_launches() - launches0
    clk = clocks.stop()

    # per-phase times from the library's own CUDA events, in a separate traced loop
    # (an event between the extraction and the matching launch would keep the latter
    # from starting early, so the timed loop above records none)
    P.latch_trace_enable(ctx.handle, args.steps)
    for i in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    phases = P.latch_trace_collect(ctx.handle, args.steps)
    P.latch_trace_enable(ctx.handle, 0)

    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    ms_per_step = total_ms / args.steps
    n_desc = n0 + n1
    value = whole_job_rate(n_desc * args.steps, ws, total_ms / 1e3)

    # the plain form (one latch_extract per image, one hamming_match) on the same GPU
    plain_steps = max(3, args.steps // 5)
    plain_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(plain_steps)]
    for i in range(plain_steps):
        flush.zero_()
        plain_ev[i][0].record(stream)
        plain_step()
        plain_ev[i][1].record(stream)
    torch.cuda.synchronize()
    plain_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in plain_ev)

    # end to end through the C ABI: pinned host inputs -> device -> matches back in
    # host memory, K calls enqueued back to back, timed to the last download
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    if not torch.equal(matches_h, matches.cpu()):
        raise SystemExit("end-to-end matches differ from the device batch")
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    stream.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    h2d = sum(x.numel() for x in imgs_h) + kps_h.numel()
    d2h = matches_h.numel()

    # roofline of the dominant phase (per-phase CUDA events recorded by the library)
    ext_ms = float(np.mean(phases[:, 0]))
    mat_ms = float(np.mean(phases[:, 1]))
    from paper_1609_03986_gb300 import roofline
    rf = roofline.report(ext_ms, n0 + n1, mat_ms, n0 * n1, "tensor", os.path.join(ROOT, "MEASURED_PEAKS.json"))
    used_name = "tensor"

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline:
        t_cpu = time.perf_counter()
        train = _oracle_train(wl)
        per_desc, per_query = _oracle_rates(wl, train, 2000, 3000)
        cpu_s = _cpu_step_seconds(wl, per_desc, per_query)
        cpu = {"value": n_desc / cpu_s, "unit": "descriptors/s", "cores": 1, "kind": "oracle",
               "sample": "single-threaded C oracle: 2,000 descriptors extracted (+ the 10,000 train "
                         "descriptors) and 3,000 queries matched against 10,000, scaled to one full step",
               "seconds": time.perf_counter() - t_cpu}

    line = {
        "metric": METRIC, "value": value, "unit": "descriptors/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "images": "2 x 1920x1080 u8", "keypoints_per_image": 10000,
                   "angle_bins": 32, "scales": [1.0, 1.5, 2.25], "match": "10000 x 10000 top-2 ratio 0.8",
                   "match_path": used_name, "entry": "latch_batch_run (2 images, 1 pair)",
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"{ws} independent replicas", "tuning": tuning},
        "extract_desc_per_s": n_desc / (ext_ms / 1e3),
        "match_gpairs_per_s": n0 * n1 / (mat_ms / 1e3) / 1e9,
        "phase_ms": {"extract_both_images": ext_ms, "match": mat_ms},
        "plain_form": {"ms_per_step": plain_ms, "value": n_desc / (plain_ms / 1e3),
                       "note": "one latch_extract per image + one hamming_match, same GPU"},
        "wall_s_timed": wall1 - wall0,
        "e2e": {"value": whole_job_rate(n_desc * args.steps, ws, e2e_s), "unit": "descriptors/s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": rf,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _timed(fn, steps, warmup, flush=None):
    """CUDA-event time (ms) per call of fn on the current stream, L2 flushed between calls."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        if flush is not None:
            flush.zero_()
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def run_gallery(args):
    """16,384 queries against 1,048,576 gallery descriptors, top-2 ratio 0.8."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import synth
    torch.cuda.set_device(0)
    q, g, slots, hs = synth.gallery_workload()
    dq, dg = torch.from_numpy(q).cuda(), torch.from_numpy(g).cuda()
    out = torch.empty((q.shape[0], 16), dtype=torch.uint8, device="cuda")
    ctx = P.Context(0)
    s = int(torch.cuda.current_stream().cuda_stream)
    res = {}
    for name, path in (("tensor", P.PATH_TENSOR), ("popc", P.PATH_POPC)):
        if args.path != "auto" and args.path != name:
            continue
        fn = lambda: P.hamming_match(ctx.handle, dq, q.shape[0], dg, g.shape[0], 2, 0.8, out, path, s)
        ms = _timed(fn, args.steps, args.warmup)
        got = P.matches_from_bytes(out.cpu().numpy())
        ok = bool((got["idx1"] == slots).all() and (got["dist1"].astype(np.int32) == hs).all())
        res[name] = {"ms": ms, "gpairs_per_s": q.shape[0] * g.shape[0] / (ms / 1e3) / 1e9, "planted_ok": ok}
    ctx.close()
    print(json.dumps({"metric": METRIC, "workload": "gallery_16384x1048576", "unit": "Gpairs/s", "paths": res,
                      "steps": args.steps, "warmup": args.warmup}))
    return 0


def run_sfm_batch(args):
    """64 images of 4000x3000 (5k-50k keypoints) x 476 neighbour pairs: the batched
    entry point (captured in a CUDA graph) against one call per image and per pair."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import synth
    torch.cuda.set_device(0)
    wl = synth.sfm_batch()
    w, h = wl["width"], wl["height"]
    n = [len(k) for k in wl["kps"]]
    ctx = P.Context(0, triplets=wl["triplets"])
    # extraction tiles chosen by the autotuner on this workload's image size and the
    # median keypoint count (the batch always matches on the tensor cores)
    tuning = P.latch_autotune(ctx.handle, w, h, int(np.median(n)), 0, 0)
    imgs = [torch.from_numpy(im).cuda() for im in wl["images"]]
    d_kps = torch.from_numpy(np.concatenate([P.pack_keypoints(k) for k in wl["kps"]])).cuda()
    d_desc = torch.zeros((sum(n), 64), dtype=torch.uint8, device="cuda")
    pairs = wl["pairs"]
    nout = sum(n[a] for a, _ in pairs)
    d_m = torch.zeros((nout, 16), dtype=torch.uint8, device="cuda")
    b = P.BatchDesc([(t, w, h, t.stride(0)) for t in imgs], n, d_kps, d_desc, pairs, 2, 0.8, d_m)
    P.latch_reserve_batch(ctx.handle, b)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = int(stream.cuda_stream)
        P.latch_batch_run(ctx.handle, b, s)  # warm-up outside capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            P.latch_batch_run(ctx.handle, b, int(torch.cuda.current_stream().cuda_stream))
        batched_ms = _timed(lambda: graph.replay(), args.steps, args.warmup)
        batched_ref = d_m.clone()
        # plain form: one latch_extract per image, one hamming_match per pair
        off = np.concatenate([[0], np.cumsum(n)])
        mo = b.match_offsets()
        P.latch_reserve(ctx.handle, max(n), max(n), max(n))

        def plain():
            for i in range(len(imgs)):
                P.latch_extract(ctx.handle, imgs[i], w, h, imgs[i].stride(0), d_kps[off[i]:off[i + 1]], n[i], None,
                                d_desc[off[i]:off[i + 1]], s)
            for p, (qi, ti) in enumerate(pairs):
                P.hamming_match(ctx.handle, d_desc[off[qi]:off[qi + 1]], n[qi], d_desc[off[ti]:off[ti + 1]], n[ti],
                                2, 0.8, d_m[mo[p]:mo[p + 1]], P.PATH_TENSOR, s)
        plain_ms = _timed(plain, max(1, args.steps // 4), 1)
    same = bool(torch.equal(batched_ref, d_m))
    ctx.check()
    pairs_total = sum(n[a] * n[c] for a, c in pairs)
    print(json.dumps({"metric": METRIC, "workload": "sfm_batch_64x4000x3000_476pairs", "unit": "descriptors/s",
                      "batched": {"ms": batched_ms, "desc_per_s": sum(n) / (batched_ms / 1e3),
                                  "gpairs_per_s": pairs_total / (batched_ms / 1e3) / 1e9},
                      "plain": {"ms": plain_ms, "desc_per_s": sum(n) / (plain_ms / 1e3),
                                "gpairs_per_s": pairs_total / (plain_ms / 1e3) / 1e9},
                      "identical_results": same, "descriptors": sum(n), "pairs": pairs_total,
                      "tuning": tuning, "steps": args.steps, "warmup": args.warmup}))
    return 0


def run_serve(args):
    """Poisson stream of extract-and-match requests (images from 640x480 to
    4000x3000, 1k-64k oriented keypoints) against 32 resident galleries of 10k-200k
    descriptors, through the session API (continuous batching)."""
    import threading
    import queue as _q
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import synth
    torch.cuda.set_device(0)
    sizes = [(640, 480), (1280, 720), (1920, 1080), (2560, 1440), (4000, 3000)]
    per_size = 4
    pool = {}
    for si, (w, h) in enumerate(sizes):
        for j in range(per_size):
            im = P.pinned_copy(synth.image(synth.seed(5, si * per_size + j, synth.KIND_IMAGE), w, h))
            kp = synth.keypoints(synth.seed(5, si * per_size + j, synth.KIND_KEYPOINTS), w, h, 64000, 32, True, 3)
            pool[(si, j)] = (im, w, h, P.pinned_copy(P.pack_keypoints(kp)))
    gal_n = synth.batch_keypoint_counts(32, 10000, 200000, config=5)
    gals = [synth.random_descriptors(synth.seed(5, 1000 + g, synth.KIND_GALLERY), int(n)) for g, n in enumerate(gal_n)]
    t_arr, size_i, kps_n, gal_i = synth.arrivals(synth.seed(5, 0, synth.KIND_ARRIVALS), args.rate, args.duration,
                                                 len(sizes), 1000, 64000, 32)
    sess = P.Session(synth.triplets(), hbm_budget=12 << 30, max_gallery_rows=int(gal_n.sum()) + 1, max_batch=16,
                     max_batch_kps=1 << 18)
    for g in gals:
        sess.add_gallery(g)
    # warm-up
    for i in range(8):
        im, w, h, kp = pool[(i % len(sizes), 0)]
        sess.wait(sess.submit(im, w, h, kp[:4000], i % 32))
    tickets = _q.Queue()
    n_req = len(t_arr)

    def submitter():
        t0 = time.perf_counter()
        for i in range(n_req):
            dt = t_arr[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            im, w, h, kp = pool[(int(size_i[i]), i % per_size)]
            tickets.put((sess.submit(im, w, h, kp[:int(kps_n[i])], int(gal_i[i])), int(kps_n[i])))

    th = threading.Thread(target=submitter)
    wall0 = time.perf_counter()
    th.start()
    lat, first, last, ndesc, bsz = [], None, None, 0, []
    for _ in range(n_req):
        t, n = tickets.get()
        r, m, _ = sess.wait(t)
        lat.append((r.done_s - r.submit_s) * 1e3)
        first = r.submit_s if first is None else min(first, r.submit_s)
        last = r.done_s if last is None else max(last, r.done_s)
        ndesc += n
        bsz.append(r.batch_size)
    th.join()
    wall = time.perf_counter() - wall0
    st = sess.stats()
    sess.close()
    lat = np.array(lat)
    pairs = float(sum(int(kps_n[i]) * int(gal_n[gal_i[i]]) for i in range(n_req)))
    print(json.dumps({"metric": METRIC, "workload": f"serve_poisson_{args.rate:g}rps_{args.duration:g}s",
                      "requests": n_req, "offered_rps": args.rate,
                      "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                     "max": float(lat.max()), "mean": float(lat.mean())},
                      "sustained_desc_per_s": ndesc / (last - first), "sustained_gpairs_per_s": pairs / (last - first) / 1e9,
                      "achieved_rps": n_req / (last - first), "mean_batch": float(np.mean(bsz)),
                      "max_batch": int(np.max(bsz)), "wall_s": wall, "stats": st}))
    return 0


def main():
    args = _args()
    if args.workload == "serve":
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "gallery":
        return run_gallery(args)
    if args.workload == "sfm_batch":
        return run_sfm_batch(args)
    return run_latch(args)


if __name__ == "__main__":
    sys.exit(main())
