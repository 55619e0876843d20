"""Roofline bookkeeping for the benchmark: algorithmic work per launch of each
kernel and the peak it is bounded by.

Algorithmic work (independent of how a kernel computes it):
  extraction  per descriptor: 512 triplets x 2 patch distances x 49 pixels x
              2 integer ops (subtract, multiply-add) = 100,352 int32 ops;
              bytes: the 2,304 window samples it reads + 64 bytes written.
  popc match  per pair: 16 x 32-bit population counts (512 bits), the
              quarter-rate pipe that bounds the XOR+POPC kernel.
  tensor match per pair: 2 x 512 multiply-adds of 0/1 values = 1,024 flop.
Peaks: int32 issue = 152 SMs x 128 lanes x SM clock; POPC = 152 x 16 x clock;
8-bit-float tensor = measured dense bf16 x 2 (nominal fp8/bf16 ratio);
clock = the maximum SM clock measured by the driver.
"""
from __future__ import annotations

import hashlib
import json
import os

SMS = 152
INT_LANES_PER_SM = 128
POPC_PER_SM = 16
EXTRACT_OPS_PER_DESC = 512 * 2 * 49 * 2
POPC_PER_PAIR = 16
TENSOR_FLOP_PER_PAIR = 2 * 512
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _peaks(path):
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def source_hash(name: str) -> str:
    with open(os.path.join(HERE, "csrc", name), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def traffic(kernel: str, source: str):
    """dram read+write bytes per launch from the committed ncu summary, if it was
    taken on the current source of the kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(p).read().splitlines()
    except OSError:
        return None
    h = source_hash(source)
    for line in lines:
        parts = line.split("#", 1)[0].split()
        if len(parts) >= 3 and parts[0] == kernel and parts[2] == h:
            return float(parts[1])
    return None


def report(extract_ms: float, n_desc: int, match_ms: float, pairs: int, path: str, peaks_path: str):
    """Roofline of the dominant phase (the other under "other").  extract_ms: time of
    the extraction launches over n_desc descriptors; match_ms: time of the matching
    launches over `pairs` pairs."""
    peaks, kind = _peaks(peaks_path)
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    ext = {"bound": "alu", "achieved": EXTRACT_OPS_PER_DESC * n_desc / (extract_ms / 1e3) / 1e12,
           "peak": SMS * INT_LANES_PER_SM * clk / 1e12, "unit": "Tops/s (int32)",
           "kernel": "extract", "units_per_launch": n_desc, "traffic": traffic("extract", "extract.cu"),
           "note": "bound in practice by the shared-memory data pipe and instruction issue together (each about "
                   "68-70% busy under ncu: conflict-free patch loads, 1,322 wavefronts per descriptor), not int32 "
                   "throughput"}
    if path == "tensor":
        mat = {"bound": "tensor", "achieved": TENSOR_FLOP_PER_PAIR * pairs / (match_ms / 1e3) / 1e12,
               "peak": 2.0 * float(peaks["bf16_tflops"]), "unit": "TFLOP/s (fp8 e4m3)", "kernel": "match_tensor",
               "units_per_launch": pairs, "traffic": traffic("match_tensor", "match_tc.cu")}
    else:
        mat = {"bound": "alu", "achieved": POPC_PER_PAIR * pairs / (match_ms / 1e3) / 1e12,
               "peak": SMS * POPC_PER_SM * clk / 1e12, "unit": "Tpopc/s", "kernel": "match_popc",
               "units_per_launch": pairs, "traffic": traffic("match_popc", "match_popc.cu")}
    for r in (ext, mat):
        r["frac"] = r["achieved"] / r["peak"]
        r["peak_source"] = f"{kind} (MEASURED_PEAKS.json clock / bf16)" if kind == "measured" else "fallback"
    dominant = ext if extract_ms >= match_ms else mat
    out = dict(dominant)
    out["other"] = mat if dominant is ext else ext
    return out
