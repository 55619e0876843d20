"""Benchmark of the LATCH extraction + Hamming matching hot path on one GPU.

Headline step (the largest single-GPU workload): the batched structure-from-motion
workload -- 64 grey images of 4000x3000, 5k-50k oriented and scaled keypoints each
(32 angle bins, 3 scales), every image matched top-2 (ratio 0.8) against its next 8
images (476 pairs) -- as one latch_batch_run replayed from a CUDA graph.  `value` is
descriptors/s of that step.  The same JSON line carries sub-records for the other
workloads, each timed on its own with its own roofline fraction and clocks:
  plain_640x480_2k        one upright pair, latch_extract x 2 + hamming_match in a graph
  oriented_1920x1080_10k  one oriented / scaled pair on both matching paths
  gallery_16k_x_1M        16,384 queries x 1,048,576 descriptors on both paths
  detect_extract          oriented FAST on a 4000x3000 image, alone and fused with extraction
  weighted_8x8            the oriented pair's extraction with Gaussian-weighted 8x8 patches
  serve_poisson           a Poisson request stream through the serving session and
                          through the plain per-request calls

  python bench.py [--gpus N] [--steps K] [--warmup W]
  python bench.py --workload sfm_batch|pair|plain_pair|gallery|serve   # one workload alone
  python bench.py --impl reference ...   # the CPU oracle on bounded samples of the headline

Under torchrun each rank runs its own replica of the headline step (independent
images, no collective on the data path); rank 0 prints units of all ranks divided by
the slowest rank's time, and only a single-GPU run adds the sub-records.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LATCH descriptors/s + Hamming Gpairs/s (bit-exact); serve p50/p99 latency"
HEADLINE = "sfm_batch_64x4000x3000_476pairs"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="latch", choices=["latch", "reference"])
    p.add_argument("--workload", default="all",
                   choices=["all", "sfm_batch", "pair", "plain_pair", "gallery", "detect", "weighted", "dense",
                            "serve"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrivals per second")
    p.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during a timed region."""

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
        time.sleep(0.4)  # first readings before the timed region

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


def _gpu_index(local):
    import torch
    return torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local


def _timed(fn, steps, warmup, flush=None, stream=None):
    """Mean CUDA-event time (ms) of fn on the current stream, L2 flushed (outside the
    events) between calls."""
    import torch
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        if flush is not None:
            flush.zero_()
        fn()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        evs[i][0].record(stream)
        fn()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return statistics.mean(e[0].elapsed_time(e[1]) for e in evs)


def _phase_ms(calls, steps, flush):
    """Per-call CUDA-event times (ms) of a sequence of calls, averaged over steps (an
    event between two chained launches keeps the second from starting early, so
    these are taken in a loop of their own)."""
    import torch
    stream = torch.cuda.current_stream()
    tot = np.zeros(len(calls))
    for _ in range(steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)]
        ev[0].record(stream)
        for j, c in enumerate(calls):
            c()
            ev[j + 1].record(stream)
        torch.cuda.synchronize()
        tot += [ev[j].elapsed_time(ev[j + 1]) for j in range(len(calls))]
    return tot / steps


# ------------------------------------------------------------------ CPU oracle timing

def _oracle_pool_run(fns, threads):
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda f: f(), fns))


def oracle_sample(wl, threads: int, n_extract: int, n_rows: int, train_desc=None):
    """Time the unchanged single-threaded oracle on a bounded sample of the batched
    workload, sharded over `threads` host threads (ctypes releases the GIL): the
    train image 1 extracted in full (unless given), n_extract keypoints of image 0
    extracted, and n_rows of them matched against image 1's descriptors.  Returns
    (seconds per descriptor, seconds per pair, wall seconds, train descriptors)."""
    import oracle
    from paper_1609_03986_gb300 import synth
    w, h, trip = wl["width"], wl["height"], wl["triplets"]

    def ext(img, kps, per):
        return [lambda a=a: oracle.extract(img, w, h, kps[a:a + per], trip, synth.SCALES)
                for a in range(0, len(kps), per)]

    t_all = time.perf_counter()
    n_ext = n_extract
    t0 = time.perf_counter()
    if train_desc is None:
        k1 = wl["kps"][1]
        train_desc = np.concatenate(_oracle_pool_run(ext(wl["images"][1], k1, max(1, -(-len(k1) // (4 * threads)))),
                                                     threads))
        n_ext += len(k1)
    k0 = wl["kps"][0][:n_extract]
    q = np.concatenate(_oracle_pool_run(ext(wl["images"][0], k0, max(1, -(-len(k0) // (4 * threads)))), threads))
    t1 = time.perf_counter()
    rows = q[:n_rows]
    per = max(1, -(-n_rows // (2 * threads)))
    _oracle_pool_run([lambda a=a: oracle.match(rows[a:a + per], train_desc, 2, 0.8) for a in range(0, n_rows, per)],
                     threads)
    t2 = time.perf_counter()
    return (t1 - t0) / n_ext, (t2 - t1) / (n_rows * len(train_desc)), time.perf_counter() - t_all, train_desc


def _sfm_counts(wl):
    n = [len(k) for k in wl["kps"]]
    return n, sum(n), float(sum(n[a] * n[b] for a, b in wl["pairs"]))


def cpu_baseline(wl):
    """The oracle on host cores for the headline step: one core, then all cores."""
    n, n_desc, pairs = _sfm_counts(wl)
    out = {}
    for threads in (1, os.cpu_count() or 1):
        n_ext, n_rows = (4000, 800) if threads == 1 else (16000, 4000)
        per_desc, per_pair, wall, _ = oracle_sample(wl, threads, n_ext, n_rows)
        step_s = per_desc * n_desc + per_pair * pairs
        out[threads] = {"value": n_desc / step_s, "unit": "descriptors/s", "cores": threads, "kind": "oracle",
                        "sample": f"image 1 extracted in full + {n_ext} keypoints of image 0 extracted and {n_rows} "
                                  f"of them matched against image 1; per-descriptor and per-pair times scaled to the "
                                  f"full step ({n_desc} descriptors, {pairs:.3e} pairs)",
                        "s_per_descriptor": per_desc, "ns_per_pair": per_pair * 1e9, "seconds": wall}
    allc = out[max(out)]
    allc["single_core"] = out[1]
    return allc


def run_reference(args):
    """The CPU oracle as the reference arm: each step a bounded sample of the headline
    workload on all host cores, scaled to the full step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1609_03986_gb300 import synth
    wl = synth.sfm_batch()
    n, n_desc, pairs = _sfm_counts(wl)
    threads = os.cpu_count() or 1
    train = None
    times = []
    for i in range(args.warmup + args.steps):
        per_desc, per_pair, _, train = oracle_sample(wl, threads, 4096, 64 * threads, train)
        if i >= args.warmup:
            times.append(per_desc * n_desc + per_pair * pairs)
    step_s = statistics.mean(times)
    value = n_desc / step_s
    sample = (f"per step: 4,096 keypoints of image 0 extracted and {64 * threads} of them matched against image 1's "
              f"{len(train)} oracle descriptors (extracted once in setup), sharded over {threads} host threads, "
              f"scaled to the full step ({n_desc} descriptors, {pairs:.3e} pairs)")
    line = {
        "metric": METRIC, "value": value, "unit": "descriptors/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": _sfm_config(wl),
        "cpu_baseline": {"value": value, "unit": "descriptors/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "descriptors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ headline: batched SfM step

def _sfm_config(wl):
    n, n_desc, pairs = _sfm_counts(wl)
    return {"workload": HEADLINE, "images": f"{len(wl['images'])} x {wl['width']}x{wl['height']} u8",
            "keypoints": f"{min(n)}-{max(n)} per image, {n_desc} in all, 32 angle bins, scales 1/1.5/2.25",
            "pairs": f"{len(wl['pairs'])} (each image against its next 8), top-2 ratio 0.8, {pairs:.4e} pairs",
            "entry": "latch_batch_run (one sort, one extraction, one tensor-core matching launch and its merge pass) replayed "
                     "from a CUDA graph",
            "l2": "inputs (768 MB of images) larger than L2; a 256 MB L2 flush between timed steps as well",
            "match_path": "tensor (tcgen05 kind::mxf4, E2M1 +-1, block scales 2^0)"}


def bench_sfm_batch(args, local, ws):
    import torch
    import torch.distributed as dist
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth

    dev = torch.device("cuda", local)
    wl = synth.sfm_batch()
    w, h = wl["width"], wl["height"]
    n, n_desc, pairs_total = _sfm_counts(wl)
    ctx = P.Context(local, triplets=wl["triplets"])
    tuning = P.latch_autotune(ctx.handle, w, h, int(np.median(n)), 0, 0)
    imgs_h = [torch.from_numpy(im).pin_memory() for im in wl["images"]]
    kps_h = torch.from_numpy(np.concatenate([P.pack_keypoints(k) for k in wl["kps"]])).pin_memory()
    imgs = [t.to(dev) for t in imgs_h]
    d_kps = kps_h.to(dev)
    pairs = wl["pairs"]
    nout = sum(n[a] for a, _ in pairs)
    d_desc = torch.zeros((n_desc, 64), dtype=torch.uint8, device=dev)
    d_m = torch.zeros((nout, 16), dtype=torch.uint8, device=dev)
    m_h = torch.empty((nout, 16), dtype=torch.uint8).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    b = P.BatchDesc([(t, w, h, t.stride(0)) for t in imgs], n, d_kps, d_desc, pairs, 2, 0.8, d_m)
    P.latch_reserve_batch(ctx.handle, b)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        s = int(stream.cuda_stream)
        P.latch_batch_run(ctx.handle, b, s)
        torch.cuda.synchronize()
        ctx.check()
        ref_desc, ref_m = d_desc.clone(), d_m.clone()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            P.latch_batch_run(ctx.handle, b, s)
        for _ in range(args.warmup):
            flush.zero_()
            graph.replay()
        torch.cuda.synchronize()
        clocks = ClockSampler(_gpu_index(local))
        clocks.start()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            graph.replay()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        clk = clocks.stop()
        # a replay launches the captured kernels: count them from one eager run
        launches0 = P.latch_kernel_launches()
        P.latch_batch_run(ctx.handle, b, s)
        torch.cuda.synchronize()
        per_step_launches = P.latch_kernel_launches() - launches0
        if not (torch.equal(ref_desc, d_desc) and torch.equal(ref_m, d_m)):
            raise SystemExit("graph replay changed the results")
        step_ms = [e[0].elapsed_time(e[1]) for e in evs]
        total_ms = max_over_ranks(sum(step_ms), ws, dev)
        ms_per_step = total_ms / args.steps

        # per-phase times from the library's own CUDA events (a separate, traced loop)
        P.latch_trace_enable(ctx.handle, args.steps)
        for _ in range(args.steps):
            flush.zero_()
            P.latch_batch_run(ctx.handle, b, s)
        torch.cuda.synchronize()
        ph = P.latch_trace_collect(ctx.handle, args.steps)
        P.latch_trace_enable(ctx.handle, 0)
        ext_ms, mat_ms = float(np.mean(ph[:, 0])), float(np.mean(ph[:, 1]))

        # the plain form: one latch_extract per image, one hamming_match per pair
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
        plain_ms = _timed(plain, max(2, args.steps // 5), 1, flush, stream)
        same_plain = bool(torch.equal(ref_desc, d_desc) and torch.equal(ref_m, d_m))

        # end to end through the C ABI: pinned host images and keypoints in, matches back
        # in pinned host memory, calls enqueued back to back, timed to the last download
        hb = P.HostBatchDesc([(t, w, h, t.stride(0)) for t in imgs_h], n, kps_h, None, pairs, 2, 0.8, m_h)
        for _ in range(2):
            P.latch_batch_run_host(ctx.handle, hb, s)
        stream.synchronize()
        if not torch.equal(m_h, ref_m.cpu()):
            raise SystemExit("end-to-end matches differ from the device batch")
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            P.latch_batch_run_host(ctx.handle, hb, s)
        stream.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    ctx.check()
    rf = roofline.dominant([
        (mat_ms, roofline.tensor_match(mat_ms, pairs_total, HEADLINE, PEAKS, sustained=True)),
        (ext_ms, roofline.extraction(ext_ms, n_desc, HEADLINE, PEAKS))])
    res = {
        "value": whole_job_rate(n_desc * args.steps, ws, total_ms / 1e3), "ms_per_step": ms_per_step,
        "gpairs_per_s": whole_job_rate(pairs_total * args.steps, ws, total_ms / 1e3) / 1e9,
        "phase_ms": {"extract_all_images": ext_ms, "match_all_pairs": mat_ms},
        "extract_desc_per_s": n_desc / (ext_ms / 1e3), "match_gpairs_per_s": pairs_total / (mat_ms / 1e3) / 1e9,
        "plain_form": {"ms_per_step": plain_ms, "value": n_desc / (plain_ms / 1e3),
                       "speedup_of_batched": plain_ms / ms_per_step, "identical_results": same_plain,
                       "note": "one latch_extract per image + one hamming_match per pair, same GPU"},
        "e2e": {"value": whole_job_rate(n_desc * args.steps, ws, e2e_s), "unit": "descriptors/s",
                "h2d_bytes_per_step": int(sum(x.numel() for x in imgs_h) + kps_h.numel()),
                "d2h_bytes_per_step": int(m_h.numel()), "entry": "latch_batch_run_host"},
        "gpu_launches": per_step_launches * args.steps,
        "roofline": rf, "clocks": clk, "tuning": tuning, "config": _sfm_config(wl), "wl": wl,
    }
    del graph
    ctx.close()
    return res


# ------------------------------------------------------------------ sub-records

def _sub_clocks(local):
    c = ClockSampler(_gpu_index(local))
    c.start()
    return c


def bench_plain_pair(args, local):
    """Upright 640x480 pair, 2,000 keypoints each: latch_extract x 2 + hamming_match
    (path chosen per shape) captured in one CUDA graph."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth
    dev = torch.device("cuda", local)
    name = "plain_640x480_2k"
    wl = synth.pair(name)
    w, h = wl["width"], wl["height"]
    ctx = P.Context(local, triplets=wl["triplets"])
    n0, n1 = (len(k) for k in wl["kps"])
    P.latch_reserve(ctx.handle, max(n0, n1), n0, n1)
    imgs = [torch.from_numpy(im).to(dev) for im in wl["images"]]
    kps = [torch.from_numpy(P.pack_keypoints(k)).to(dev) for k in wl["kps"]]
    desc = [torch.empty((nn, 64), dtype=torch.uint8, device=dev) for nn in (n0, n1)]
    m = torch.empty((n0, 16), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    path = P.hamming_match_path(ctx.handle, n0, n1)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        s = int(stream.cuda_stream)
        calls = [lambda i=i: P.latch_extract(ctx.handle, imgs[i], w, h, imgs[i].stride(0), kps[i], len(kps[i]), None,
                                             desc[i], s) for i in range(2)]
        calls.append(lambda: P.hamming_match(ctx.handle, desc[0], n0, desc[1], n1, 2, 0.8, m, path, s))
        for c in calls:
            c()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for c in calls:
                c()
        clocks = _sub_clocks(local)
        ms = _timed(graph.replay, args.steps, args.warmup, flush, stream)
        clk = clocks.stop()
        ph = _phase_ms(calls, args.steps, flush)
    ctx.check()
    ext_ms = float(ph[0] + ph[1])
    mrf = (roofline.tensor_match(ph[2], n0 * n1, name, PEAKS, sustained=False)
           if path == P.PATH_TENSOR else roofline.popc_match(ph[2], n0 * n1, name, PEAKS))
    rf = roofline.dominant([(ext_ms, roofline.extraction(ext_ms, n0 + n1, name, PEAKS)), (ph[2], mrf)])
    del graph
    ctx.close()
    return {"workload": name, "entry": "latch_extract x 2 + hamming_match, CUDA graph",
            "match_path": {1: "popc", 2: "tensor"}[path], "ms_per_step": ms, "desc_per_s": (n0 + n1) / (ms / 1e3),
            "gpairs_per_s": n0 * n1 / (ms / 1e3) / 1e9,
            "phase_ms": {"extract_image0": ph[0], "extract_image1": ph[1], "match": ph[2]},
            "roofline": rf, "clocks": clk}


def bench_oriented_pair(args, local):
    """Oriented and scaled 1920x1080 pair, 10,000 keypoints each: the batched step on
    the tensor cores, and the plain calls with the CUDA-core (XOR + popc) matcher."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth
    dev = torch.device("cuda", local)
    name = "oriented_scaled_1920x1080_10k"
    wl = synth.pair(name)
    w, h = wl["width"], wl["height"]
    ctx = P.Context(local, triplets=wl["triplets"])
    n0, n1 = (len(k) for k in wl["kps"])
    tuning = P.latch_autotune(ctx.handle, w, h, max(n0, n1), n0, n1)
    P.latch_reserve(ctx.handle, max(n0, n1), n0, n1)
    imgs = [torch.from_numpy(im).to(dev) for im in wl["images"]]
    kps = torch.from_numpy(np.concatenate([P.pack_keypoints(k) for k in wl["kps"]])).to(dev)
    desc = torch.empty((n0 + n1, 64), dtype=torch.uint8, device=dev)
    m = torch.empty((n0, 16), dtype=torch.uint8, device=dev)
    m2 = torch.empty((n0, 16), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    b = P.BatchDesc([(t, w, h, t.stride(0)) for t in imgs], [n0, n1], kps, desc, [(0, 1)], 2, 0.8, m)
    P.latch_reserve_batch(ctx.handle, b)
    s = int(torch.cuda.current_stream().cuda_stream)
    out = {"workload": name, "tuning": tuning}
    # tensor path: the pair as a batch (2 images, 1 pair)
    P.latch_batch_run(ctx.handle, b, s)
    clocks = _sub_clocks(local)
    ms_t = _timed(lambda: P.latch_batch_run(ctx.handle, b, s), args.steps, args.warmup, flush)
    clk = clocks.stop()
    P.latch_trace_enable(ctx.handle, args.steps)
    for _ in range(args.steps):
        flush.zero_()
        P.latch_batch_run(ctx.handle, b, s)
    torch.cuda.synchronize()
    ph = P.latch_trace_collect(ctx.handle, args.steps)
    P.latch_trace_enable(ctx.handle, 0)
    ext_ms, mat_ms = float(np.mean(ph[:, 0])), float(np.mean(ph[:, 1]))
    out["tensor"] = {"entry": "latch_batch_run (2 images, 1 pair)", "ms_per_step": ms_t,
                     "desc_per_s": (n0 + n1) / (ms_t / 1e3), "gpairs_per_s": n0 * n1 / (ms_t / 1e3) / 1e9,
                     "phase_ms": {"extract_both_images": ext_ms, "match": mat_ms},
                     "roofline": roofline.dominant([
                         (ext_ms, roofline.extraction(ext_ms, n0 + n1, name, PEAKS)),
                         (mat_ms, roofline.tensor_match(mat_ms, n0 * n1, name, PEAKS, sustained=False))]),
                     "clocks": clk}
    # popc path: plain calls, per-call phases
    calls = [lambda: P.latch_extract(ctx.handle, imgs[0], w, h, imgs[0].stride(0), kps[:n0], n0, None, desc[:n0], s),
             lambda: P.latch_extract(ctx.handle, imgs[1], w, h, imgs[1].stride(0), kps[n0:], n1, None, desc[n0:], s),
             lambda: P.hamming_match(ctx.handle, desc[:n0], n0, desc[n0:], n1, 2, 0.8, m2, P.PATH_POPC, s)]
    clocks = _sub_clocks(local)
    ms_p = _timed(lambda: [c() for c in calls], args.steps, args.warmup, flush)
    clk = clocks.stop()
    php = _phase_ms(calls, args.steps, flush)
    same = bool(torch.equal(m, m2))
    out["popc"] = {"entry": "latch_extract x 2 + hamming_match (PATH_POPC)", "ms_per_step": ms_p,
                   "desc_per_s": (n0 + n1) / (ms_p / 1e3), "gpairs_per_s": n0 * n1 / (ms_p / 1e3) / 1e9,
                   "phase_ms": {"extract_image0": php[0], "extract_image1": php[1], "match": php[2]},
                   "roofline": roofline.dominant([
                       (php[0] + php[1], roofline.extraction(php[0] + php[1], n0 + n1, name, PEAKS)),
                       (php[2], roofline.popc_match(php[2], n0 * n1, name, PEAKS))]),
                   "clocks": clk, "identical_to_tensor": same}
    ctx.check()
    ctx.close()
    return out


def bench_gallery(args, local):
    """16,384 queries against 1,048,576 descriptors, top-2 ratio 0.8, on both paths."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth
    dev = torch.device("cuda", local)
    q, g, slots, hs = synth.gallery_workload()
    dq, dg = torch.from_numpy(q).to(dev), torch.from_numpy(g).to(dev)
    out_t = torch.empty((q.shape[0], 16), dtype=torch.uint8, device=dev)
    out_p = torch.empty((q.shape[0], 16), dtype=torch.uint8, device=dev)
    ctx = P.Context(local)
    P.latch_reserve(ctx.handle, 0, q.shape[0], g.shape[0])
    s = int(torch.cuda.current_stream().cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    pairs = q.shape[0] * g.shape[0]
    name = "gallery_16384x1048576"
    res = {"workload": name, "entry": "hamming_match"}
    for pname, path, out in (("tensor", P.PATH_TENSOR, out_t), ("popc", P.PATH_POPC, out_p)):
        def fn(path=path, out=out):
            P.hamming_match(ctx.handle, dq, q.shape[0], dg, g.shape[0], 2, 0.8, out, path, s)
        clocks = _sub_clocks(local)
        ms = _timed(fn, args.steps, args.warmup, flush)
        clk = clocks.stop()
        got = P.matches_from_bytes(out.cpu().numpy())
        ok = bool((got["idx1"] == slots).all() and (got["dist1"].astype(np.int32) == hs).all()
                  and got["accepted"].all())
        rf = (roofline.tensor_match(ms, pairs, name, PEAKS, sustained=False) if path == P.PATH_TENSOR
              else roofline.popc_match(ms, pairs, name, PEAKS))
        res[pname] = {"ms": ms, "gpairs_per_s": pairs / (ms / 1e3) / 1e9, "planted_matches_exact": ok,
                      "roofline": rf, "clocks": clk}
    res["paths_identical"] = bool(torch.equal(out_t, out_p))
    ctx.check()
    ctx.close()
    return res


def bench_dense(args, local):
    """Dense per-pixel LATCH (Sec. 6): the descriptor of every pixel of two 640x480
    images (the second the first shifted by (3, -2)), then every pixel of the first
    matched against the second within radius 8 (up to 289 candidates each)."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth
    dev = torch.device("cuda", local)
    w, h, r = 640, 480, 8
    name = "dense_640x480_r8"
    base = synth.image(synth.seed(6, 0, synth.KIND_IMAGE), w + 16, h + 16)
    imgs = [torch.from_numpy(np.ascontiguousarray(base[8:8 + h, 8:8 + w])).to(dev),
            torch.from_numpy(np.ascontiguousarray(base[10:10 + h, 5:5 + w])).to(dev)]
    ctx = P.Context(local, triplets=synth.triplets())
    da = torch.empty((w * h, 64), dtype=torch.uint8, device=dev)
    db = torch.empty((w * h, 64), dtype=torch.uint8, device=dev)
    out = torch.empty((w * h, 16), dtype=torch.uint8, device=dev)
    s = int(torch.cuda.current_stream().cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def ext():
        P.latch_dense_extract(ctx.handle, imgs[0], w, h, w, da, s)
        P.latch_dense_extract(ctx.handle, imgs[1], w, h, w, db, s)

    def mat():
        P.latch_dense_match(ctx.handle, da, db, w, h, r, 2, 0.8, out, s)

    clocks = _sub_clocks(local)
    ms_ext = _timed(ext, args.steps, args.warmup, flush)
    ms_mat = _timed(mat, args.steps, args.warmup, flush)
    clk = clocks.stop()
    ctx.check()
    got = P.matches_from_bytes(out.cpu().numpy())
    yy, xx = np.mgrid[0:h, 0:w]
    inner = (yy >= 26) & (yy < h - 26) & (xx >= 26) & (xx < w - 26)
    shift_found = bool((got["dist1"].reshape(h, w)[inner] == 0).all())
    side_x = np.minimum(np.arange(w) + r, w - 1) - np.maximum(np.arange(w) - r, 0) + 1
    side_y = np.minimum(np.arange(h) + r, h - 1) - np.maximum(np.arange(h) - r, 0) + 1
    pairs = int(side_x.sum()) * int(side_y.sum())
    ctx.close()
    return {"workload": name, "entry": "latch_dense_extract x 2, latch_dense_match (radius 8)",
            "pixels": w * h, "candidate_pairs": pairs, "ms_extract_two_images": ms_ext, "ms_match": ms_mat,
            "desc_per_s": 2 * w * h / (ms_ext / 1e3), "match_gpairs_per_s": pairs / (ms_mat / 1e3) / 1e9,
            "shift_recovered_inside": shift_found,
            "roofline": roofline.dominant([(ms_ext, roofline.dense_extraction(ms_ext, 2 * w * h, name, PEAKS)),
                                           (ms_mat, roofline.dense_match(ms_mat, pairs, name, PEAKS))]),
            "clocks": clk}


def bench_detect(args, local):
    """Oriented FAST on one 4000x3000 image of the batched workload (threshold 20):
    detection alone, and detection + extraction of every keypoint found in one call
    (no host round trip)."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth
    dev = torch.device("cuda", local)
    name = "detect_extract_4000x3000_t20"
    w, h = synth.BATCH_W, synth.BATCH_H
    img = torch.from_numpy(synth.image(synth.seed(3, 0, synth.KIND_IMAGE), w, h)).to(dev)
    ctx = P.Context(local, triplets=synth.triplets())
    max_kps = 1 << 18
    kps = torch.empty((max_kps, 12), dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    desc = torch.empty((max_kps, 64), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s = int(torch.cuda.current_stream().cuda_stream)
    P.latch_reserve(ctx.handle, max_kps, 0, 0)

    def det():
        P.latch_detect(ctx.handle, img, w, h, img.stride(0), 20, 0, max_kps, kps, cnt, s)

    def det_ext():
        P.latch_detect_extract(ctx.handle, img, w, h, img.stride(0), 20, 0, max_kps, kps, cnt, desc, s)

    def pyr_ext():
        P.latch_detect_pyramid(ctx.handle, img, w, h, img.stride(0), 20, 3, max_kps, kps, cnt, desc, s)

    clocks = _sub_clocks(local)
    ms_p = _timed(pyr_ext, args.steps, args.warmup, flush)
    n_p = int(cnt.item())
    ms_d = _timed(det, args.steps, args.warmup, flush)
    ms_de = _timed(det_ext, args.steps, args.warmup, flush)
    clk = clocks.stop()
    n = int(cnt.item())
    ctx.check()
    ctx.close()
    ext_ms = ms_de - ms_d
    rf = roofline.dominant([
        (ext_ms, roofline.extraction(ext_ms, n, name, PEAKS)),
        (ms_d, roofline.detection(ms_d, w * h, name, PEAKS))])
    return {"workload": name, "keypoints": n, "detect_ms": ms_d, "detect_extract_ms": ms_de,
            "detect_mpix_per_s": w * h / (ms_d / 1e3) / 1e6, "desc_per_s": n / (ms_de / 1e3),
            "pyramid": {"levels": "scales 1, 1.5, 2.25", "keypoints": n_p, "detect_extract_ms": ms_p,
                        "desc_per_s": n_p / (ms_p / 1e3), "entry": "latch_detect_pyramid with descriptors"},
            "entry": "latch_detect; latch_detect_extract", "roofline": rf, "clocks": clk}


def bench_weighted(args, local):
    """The oriented 1920x1080 pair's extraction with Gaussian-weighted 8x8 patches
    against the plain 7x7 patches (triplets drawn in [3, 43] for both)."""
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth
    dev = torch.device("cuda", local)
    name = "weighted_8x8_oriented_1920x1080_10k"
    wl = synth.pair("oriented_scaled_1920x1080_10k")
    w, h = wl["width"], wl["height"]
    ctx = P.Context(local, triplets=synth.triplets(synth.seed(2, 0, synth.KIND_TRIPLETS), hi=43))
    n = sum(len(k) for k in wl["kps"])
    imgs = [torch.from_numpy(im).to(dev) for im in wl["images"]]
    kps = torch.from_numpy(np.concatenate([P.pack_keypoints(k) for k in wl["kps"]])).to(dev)
    desc = torch.empty((n, 64), dtype=torch.uint8, device=dev)
    b = P.BatchDesc([(t, w, h, t.stride(0)) for t in imgs], [len(k) for k in wl["kps"]], kps, desc, [], 2, 0.8, None)
    P.latch_reserve_batch(ctx.handle, b)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s = int(torch.cuda.current_stream().cuda_stream)
    gauss = np.array([[int(round(255 * np.exp(-((i - 3.5) ** 2 + (j - 3.5) ** 2) / 8.0))) for j in range(8)]
                      for i in range(8)], np.uint8)
    clocks = _sub_clocks(local)
    ms7 = _timed(lambda: P.latch_batch_run(ctx.handle, b, s), args.steps, args.warmup, flush)
    P.latch_set_patch_weights(ctx.handle, gauss)
    ms8 = _timed(lambda: P.latch_batch_run(ctx.handle, b, s), args.steps, args.warmup, flush)
    P.latch_set_patch_weights(ctx.handle, None)
    clk = clocks.stop()
    ctx.check()
    ctx.close()
    rf = roofline.extraction_weighted(ms8, n, name, PEAKS)
    return {"workload": name, "entry": "latch_batch_run (2 images, extraction only)", "weights": "Gaussian 8x8",
            "ms_weighted": ms8, "ms_7x7": ms7, "desc_per_s_weighted": n / (ms8 / 1e3), "desc_per_s_7x7": n / (ms7 / 1e3),
            "roofline": rf, "clocks": clk}


def _serve_inputs(args):
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import synth
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
    return sizes, per_size, pool, gal_n, gals


def _serve_arrivals(rate, duration, n_sizes, stream=0):
    from paper_1609_03986_gb300 import synth
    return synth.arrivals(synth.seed(5, stream, synth.KIND_ARRIVALS), rate, duration, n_sizes, 1000, 64000, 32)


def _latency_summary(lat_ms, first, last, ndesc, pairs, n_req):
    lat = np.array(lat_ms)
    span = last - first
    return {"latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max()), "mean": float(lat.mean())},
            "achieved_rps": n_req / span, "sustained_desc_per_s": ndesc / span,
            "sustained_gpairs_per_s": pairs / span / 1e9}


def _drive(n_req, t_arr, submit, wait):
    """Submits request i at its arrival time from one thread and waits in this one;
    returns per-request latencies (ms), the first submit and last completion times,
    and the micro-batch size each request ran in."""
    import queue as _q
    tickets = _q.Queue()

    def submitter():
        t0 = time.perf_counter()
        for i in range(n_req):
            dt = t_arr[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.put((submit(i), time.perf_counter()))

    th = threading.Thread(target=submitter)
    th.start()
    lat, first, last, bsz = [], None, None, []
    for _ in range(n_req):
        tk, t_sub = tickets.get()
        t_done, b = wait(tk)
        lat.append((t_done - t_sub) * 1e3)
        first = t_sub if first is None else min(first, t_sub)
        last = t_done if last is None else max(last, t_done)
        bsz.append(b)
    th.join()
    return lat, first, last, bsz


def _serve_session(local, inputs, arr, lanes, name, sustained_roof=True):
    """One request stream through a session with `lanes` lanes (continuous batching)."""
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import roofline, synth
    sizes, per_size, pool, gal_n, gals = inputs
    t_arr, size_i, kps_n, gal_i = arr
    n_req = len(t_arr)
    pairs = float(sum(int(kps_n[i]) * int(gal_n[gal_i[i]]) for i in range(n_req)))
    sess = P.Session(synth.triplets(), device=local, hbm_budget=12 << 30, max_gallery_rows=int(gal_n.sum()) + 1,
                     max_batch=16, max_batch_kps=1 << 18, lanes=lanes)
    for g in gals:
        sess.add_gallery(g)
    for i in range(8):
        im, w, h, kp = pool[(i % len(sizes), 0)]
        sess.wait(sess.submit(im, w, h, kp[:4000], i % 32))

    def s_submit(i):
        im, w, h, kp = pool[(int(size_i[i]), i % per_size)]
        return sess.submit(im, w, h, kp[:int(kps_n[i])], int(gal_i[i]))

    def s_wait(t):
        r, _, _ = sess.wait(t)
        return time.perf_counter(), r.batch_size

    clocks = _sub_clocks(local)
    lat, first, last, bsz = _drive(n_req, t_arr, s_submit, s_wait)
    clk = clocks.stop()
    st = sess.stats()
    sess.close()
    rec = _latency_summary(lat, first, last, int(kps_n.sum()), pairs, n_req)
    rec.update({"entry": f"latch_session_* (continuous batching, {lanes} lanes)", "lanes": lanes,
                "mean_batch": float(np.mean(bsz)), "max_batch": int(np.max(bsz)), "stats": st, "clocks": clk})
    if sustained_roof:
        rec["roofline"] = roofline.tensor_match((last - first) * 1e3, pairs, name, PEAKS, sustained=True)
        rec["roofline"]["note"] = "pairs over the whole stream's span: a latency workload at this offered rate"
    return rec


def _serve_plain(local, inputs, arr):
    """The same stream through the plain per-request calls (upload, latch_extract,
    hamming_match against the resident gallery, download), one request at a time in
    arrival order."""
    import queue as _q
    import torch
    import paper_1609_03986_gb300 as P
    from paper_1609_03986_gb300 import synth
    dev = torch.device("cuda", local)
    sizes, per_size, pool, gal_n, gals = inputs
    t_arr, size_i, kps_n, gal_i = arr
    n_req = len(t_arr)
    pairs = float(sum(int(kps_n[i]) * int(gal_n[gal_i[i]]) for i in range(n_req)))
    ctx = P.Context(local, triplets=synth.triplets())
    P.latch_reserve(ctx.handle, 64000, 64000, int(gal_n.max()))
    d_gals = [torch.from_numpy(g_).to(dev) for g_ in gals]
    d_img = torch.empty(3000 * 4000, dtype=torch.uint8, device=dev)
    d_kps = torch.empty((64000, 12), dtype=torch.uint8, device=dev)
    d_desc = torch.empty((64000, 64), dtype=torch.uint8, device=dev)
    d_m = torch.empty((64000, 16), dtype=torch.uint8, device=dev)
    h_m = torch.empty((64000, 16), dtype=torch.uint8).pin_memory()
    stream = torch.cuda.Stream(device=dev)
    s = int(stream.cuda_stream)
    work = _q.Queue()
    done = {}
    cv = threading.Condition()

    def worker():
        torch.cuda.set_device(local)
        with torch.cuda.stream(stream):
            while True:
                i = work.get()
                if i is None:
                    return
                im, w, h, kp = pool[(int(size_i[i]), i % per_size)]
                nk = int(kps_n[i])
                pitch = im.strides[0]
                d_img[:h * pitch].view(h, pitch).copy_(torch.from_numpy(im), non_blocking=True)
                d_kps[:nk].copy_(torch.from_numpy(kp[:nk]), non_blocking=True)
                P.latch_extract(ctx.handle, d_img, w, h, pitch, d_kps, nk, None, d_desc, s)
                g = int(gal_i[i])
                P.hamming_match(ctx.handle, d_desc, nk, d_gals[g], len(gals[g]), 2, 0.8, d_m, P.PATH_AUTO, s)
                h_m[:nk].copy_(d_m[:nk], non_blocking=True)
                stream.synchronize()
                with cv:
                    done[i] = time.perf_counter()
                    cv.notify_all()

    th = threading.Thread(target=worker)
    th.start()
    for i in range(4):  # warm-up
        work.put(i)
    with cv:
        cv.wait_for(lambda: len(done) >= 4)
        done.clear()

    def p_submit(i):
        work.put(i)
        return i

    def p_wait(i):
        with cv:
            cv.wait_for(lambda: i in done)
            return done.pop(i), 1

    clocks = _sub_clocks(local)
    lat, first, last, _ = _drive(n_req, t_arr, p_submit, p_wait)
    clk = clocks.stop()
    work.put(None)
    th.join()
    ctx.check()
    ctx.close()
    rec = _latency_summary(lat, first, last, int(kps_n.sum()), pairs, n_req)
    rec.update({"entry": "per request: upload, latch_extract, hamming_match (path per shape) against the "
                         "resident packed gallery, download; one request at a time in arrival order",
                "clocks": clk})
    return rec


def bench_serve(args, local):
    """The Poisson request stream (--rate, --duration) through the session (continuous
    batching, 2 lanes) and through the plain per-request calls; then an overload stream
    (1,000 req/s for 6 s, beyond one-at-a-time capacity) through sessions of 2 and 4
    lanes and the plain calls, where requests queue and micro-batches form."""
    inputs = _serve_inputs(args)
    sizes = inputs[0]
    arr = _serve_arrivals(args.rate, args.duration, len(sizes))
    name = f"serve_poisson_{args.rate:g}rps_{args.duration:g}s"
    out = {"workload": name, "requests": len(arr[0]), "offered_rps": args.rate,
           "request_mix": "640x480..4000x3000 images, 1k-64k oriented keypoints, 32 resident galleries of "
                          "10k-200k descriptors"}
    out["session"] = _serve_session(local, inputs, arr, 2, name)
    out["plain_per_request"] = _serve_plain(local, inputs, arr)
    over_rate, over_s = 1000.0, 6.0
    arr_o = _serve_arrivals(over_rate, over_s, len(sizes), stream=1)
    over = {"offered_rps": over_rate, "duration_s": over_s, "requests": len(arr_o[0])}
    for lanes in (2, 4):
        over[f"session_{lanes}_lanes"] = _serve_session(local, inputs, arr_o, lanes, name, sustained_roof=False)
    over["plain_per_request"] = _serve_plain(local, inputs, arr_o)
    out["overload"] = over
    return out


# ------------------------------------------------------------------ driver

def run_latch(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    single = {"pair": bench_oriented_pair, "plain_pair": bench_plain_pair, "gallery": bench_gallery,
              "detect": bench_detect, "weighted": bench_weighted, "dense": bench_dense, "serve": bench_serve}
    if args.workload in single:
        print(json.dumps({"metric": METRIC, **single[args.workload](args, local)}))
        return 0
    head = bench_sfm_batch(args, local, ws)
    wl = head.pop("wl")
    sub = {}
    if ws == 1 and args.workload == "all":
        torch.cuda.empty_cache()
        for key, fn in (("plain_640x480_2k", bench_plain_pair), ("oriented_scaled_1920x1080_10k", bench_oriented_pair),
                        ("gallery_16384x1048576", bench_gallery), ("detect_extract_4000x3000", bench_detect),
                        ("weighted_8x8_1920x1080", bench_weighted), ("dense_640x480_r8", bench_dense),
                        ("serve", bench_serve)):
            sub[key] = fn(args, local)
            torch.cuda.empty_cache()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    cpu = None if args.no_cpu_baseline else cpu_baseline(wl)
    cfg = head.pop("config")
    cfg["parallelism"] = f"{ws} independent replicas"
    cfg["tuning"] = head.pop("tuning")
    line = {
        "metric": METRIC, "value": head.pop("value"), "unit": "descriptors/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": cfg,
        "gpu_launches": head.pop("gpu_launches"), "roofline": head.pop("roofline"), "clocks": head.pop("clocks"),
        "e2e": head.pop("e2e"), "cpu_baseline": cpu, **head, "configs": sub,
    }
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_latch(args)


if __name__ == "__main__":
    sys.exit(main())
