"""Roofline bookkeeping for the benchmark: the algorithmic work per launch of each
kernel and the measured ceiling it is judged against.

Algorithmic work (independent of how a kernel computes it):
  extraction   per descriptor: 512 triplets x 2 patch distances x 49 pixels x 2
               integer ops (subtract, multiply-add) = 100,352 int32 ops (Eq. 1).
  popc match   per pair: the 512-bit XOR and population count, 16 words each
               (Sec. 4's Hamming distance).
  tensor match per pair: 2 x 512 multiply-adds of +-1 values = 1,024 flop.

Ceilings:
  int32 ops    the measured issue rate of the plain integer add (IADD3) per SM per
               clock x SMs x the maximum SM clock; the extraction also reports the
               same work against the measured dp4a rate (4 multiply-adds per lane).
  popc match   the best split of a pair's 16 words between the population-count
               pipe (one POPC per word) and the logic pipe (carry-save adders, which
               fold words with LOP3 and leave fewer POPC), from the measured rates of
               both pipes (`popc_pair_ceiling`).
  tensor       4-bit float (E2M1): the measured dense bf16 GEMM throughput
               x 6 (the nominal dense fp4 / bf16 ratio), burst for a kernel timed
               alone and sustained for one timed inside a long step; beside it the
               measured issue rate of the block-scaled E2M1 MMA (4x bf16 per clock).
Per-clock pipe rates come from a throughput probe on this GPU, stored in
``pipe_rates.json``; the clocks and the bf16 / HBM figures from the driver's
measured-peaks file.
"""
from __future__ import annotations

import hashlib
import json
import os

EXTRACT_OPS_PER_DESC = 512 * 2 * 49 * 2
EXTRACT_WEIGHTED_OPS_PER_DESC = 512 * 2 * 64 * 3
EXTRACT_DP4A_PER_DESC = 512 * 4 * 49 // 4  # D1 - D2 as four 49-term u8 dot products, 4 multiply-adds per dp4a
# dense per pixel and triplet: the product (C2 - C1)(2A - C1 - C2) (4 ops), its 7x7 box
# sum by running sums along rows and columns (2 + 2 ops) and the comparison (1 op)
DENSE_OPS_PER_PIXEL = 512 * 9
POPC_WORDS_PER_PAIR = 16
TENSOR_FLOP_PER_PAIR = 2 * 512
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
RATES_PATH = os.path.join(HERE, "pipe_rates.json")

# used only when pipe_rates.json is absent (marked "nominal" in every report)
_NOMINAL_RATES = {"sm_count": 152, "per_sm_per_clock": {"iadd3": 128.0, "lop3": 128.0, "imad": 64.0, "dp4a": 64.0,
                                                         "popc": 16.0}}


def _peaks(path):
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def pipe_rates():
    """(rates dict, source) with rates["per_sm_per_clock"][pipe] in lane operations."""
    try:
        with open(RATES_PATH) as f:
            return json.load(f), "measured (pipe_rates.json)"
    except OSError:
        return _NOMINAL_RATES, "nominal (no pipe_rates.json)"


def popc_pair_ceiling(logic: float, popc: float):
    """Pairs per SM per clock for the best split of 16 words: w words counted by POPC
    (1 XOR + 1 POPC + 1 add each), the other 16 - w folded by a carry-save adder tree
    (1 XOR + 2 LOP3 per word folded, then one POPC and one shift-add per weight level
    of the tree, ceil(log2(16 - w + 1)) levels).  The two pipes issue in parallel,
    so a split costs max(logic ops / logic rate, POPC / POPC rate) clocks per pair."""
    best, best_w = None, None
    for w in range(0, 17):
        f = 16 - w
        levels = 0 if f == 0 else (f).bit_length()
        logic_ops = 16 + w + 2 * f + levels
        popc_ops = w + levels
        clk = max(logic_ops / logic, popc_ops / popc)
        if best is None or clk < best:
            best, best_w = clk, w
    return 1.0 / best, best_w


def source_hash(name: str) -> str:
    with open(os.path.join(HERE, "csrc", name), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def traffic(kernel: str, source: str, workload: str):
    """dram read+write bytes per launch from the committed ncu summary for this kernel
    and workload, if it was taken on the current source of the kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(p).read().splitlines()
    except OSError:
        return None
    h = source_hash(source)
    for line in lines:
        parts = line.split("#", 1)[0].split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[3] == h:
            return float(parts[2])
    return None


def _finish(r, src):
    r["frac"] = r["achieved"] / r["peak"]
    r["peak_source"] = src
    return r


def extraction(ms: float, n_desc: int, workload: str, peaks_path: str):
    """Extraction launch(es) of `ms` over n_desc descriptors."""
    peaks, pk = _peaks(peaks_path)
    rates, rk = pipe_rates()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    sms = rates["sm_count"]
    r = {"bound": "alu", "kernel": "extract_lanes", "unit": "Tops/s (int32)", "units_per_launch": n_desc,
         "achieved": EXTRACT_OPS_PER_DESC * n_desc / (ms / 1e3) / 1e12,
         "peak": rates["per_sm_per_clock"]["iadd3"] * sms * clk / 1e12,
         "traffic": traffic("extract_lanes", "extract.cu", workload)}
    dp4a_peak = rates["per_sm_per_clock"]["dp4a"] * sms * clk
    r["dp4a_view"] = {"achieved_dp4a_per_s": EXTRACT_DP4A_PER_DESC * n_desc / (ms / 1e3),
                      "peak_dp4a_per_s": dp4a_peak,
                      "frac": EXTRACT_DP4A_PER_DESC * n_desc / (ms / 1e3) / dp4a_peak}
    return _finish(r, f"{rk}; clock {pk} (measured-peaks file)")


def extraction_weighted(ms: float, n_desc: int, workload: str, peaks_path: str):
    """Weighted 8x8 extraction: per descriptor 512 triplets x 2 distances x 64 pixels x
    3 int32 ops (subtract, square, weight-multiply-add) = 196,608 ops."""
    peaks, pk = _peaks(peaks_path)
    rates, rk = pipe_rates()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    r = {"bound": "alu", "kernel": "extract_lanes (weighted)", "unit": "Tops/s (int32)", "units_per_launch": n_desc,
         "achieved": EXTRACT_WEIGHTED_OPS_PER_DESC * n_desc / (ms / 1e3) / 1e12,
         "peak": rates["per_sm_per_clock"]["iadd3"] * rates["sm_count"] * clk / 1e12, "traffic": None}
    return _finish(r, f"{rk}; clock {pk} (measured-peaks file)")


def dense_extraction(ms: float, pixels: int, workload: str, peaks_path: str):
    """Dense descriptors: per pixel 512 triplets x 9 int32 ops of the box-sum form of
    Eq. 1 (every pixel shares its neighbours' patch sums)."""
    peaks, pk = _peaks(peaks_path)
    rates, rk = pipe_rates()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    r = {"bound": "alu", "kernel": "dense_extract", "unit": "Tops/s (int32)", "units_per_launch": pixels,
         "achieved": DENSE_OPS_PER_PIXEL * pixels / (ms / 1e3) / 1e12,
         "peak": rates["per_sm_per_clock"]["iadd3"] * rates["sm_count"] * clk / 1e12,
         "traffic": traffic("dense_extract", "dense.cu", workload)}
    return _finish(r, f"{rk}; clock {pk} (measured-peaks file)")


def dense_match(ms: float, pairs: float, workload: str, peaks_path: str):
    """Windowed dense matching on the CUDA cores: the popc matcher's ceiling per pair."""
    r = popc_match(ms, pairs, workload, peaks_path)
    r["kernel"] = "dense_match"
    r["traffic"] = traffic("dense_match", "dense.cu", workload)
    return r


def detection(ms: float, pixels: int, workload: str, peaks_path: str):
    """FAST detection: reads every pixel of the image once (1 byte) from HBM."""
    peaks, pk = _peaks(peaks_path)
    r = {"bound": "hbm", "kernel": "detect_cells", "unit": "GB/s", "units_per_launch": pixels,
         "achieved": pixels / (ms / 1e3) / 1e9, "peak": float(peaks["hbm_gbs"]),
         "traffic": traffic("detect_cells", "detect.cu", workload)}
    return _finish(r, f"{pk} HBM copy bandwidth")


def tensor_match(ms: float, pairs: float, workload: str, peaks_path: str, sustained: bool):
    """Tensor matcher: 1,024 flop per pair on the block-scaled E2M1 MMA.  `peak` is
    the measured bf16 GEMM x 6, the nominal dense fp4 / bf16 ratio (13.5 / 2.25
    PFLOP/s); `issue_view` compares with the measured issue rate of the MMA form the
    kernel uses (kind::mxf4, one CTA per MMA), 4x the bf16 rate per clock."""
    peaks, pk = _peaks(peaks_path)
    rates, rk = pipe_rates()
    bf16 = float(peaks["bf16_tflops_sustained" if sustained else "bf16_tflops"])
    achieved = TENSOR_FLOP_PER_PAIR * pairs / (ms / 1e3) / 1e12
    r = {"bound": "tensor", "kernel": "match_tc", "unit": "TFLOP/s (fp4 e2m1)", "units_per_launch": pairs,
         "achieved": achieved, "peak": 6.0 * bf16,
         "traffic": traffic("match_tc", "match_tc.cu", workload)}
    pr = rates["per_sm_per_clock"]
    if "mma_mxf4_flop" in pr and "mma_bf16_flop" in pr:
        ratio = pr["mma_mxf4_flop"] / pr["mma_bf16_flop"]
        r["issue_view"] = {"peak": ratio * bf16, "frac": achieved / (ratio * bf16),
                           "peak_model": f"bf16 {'sustained' if sustained else 'burst'} x {ratio:.2f}, the measured "
                                         "kind::mxf4 / kind::f16 issue ratio"}
    return _finish(r, f"{pk} bf16 {'sustained' if sustained else 'burst'} x 6 (nominal fp4/bf16)")


def popc_match(ms: float, pairs: float, workload: str, peaks_path: str):
    peaks, pk = _peaks(peaks_path)
    rates, rk = pipe_rates()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    pr = rates["per_sm_per_clock"]
    per_clk, w = popc_pair_ceiling(pr["lop3"], pr["popc"])
    peak = per_clk * rates["sm_count"] * clk / 1e9
    r = {"bound": "alu", "kernel": "match_popc", "unit": "Gpairs/s", "units_per_launch": pairs,
         "achieved": pairs / (ms / 1e3) / 1e9, "peak": peak,
         "peak_model": f"best split of 16 words between POPC ({pr['popc']:g}/clk/SM) and carry-save LOP3 "
                       f"({pr['lop3']:g}/clk/SM): {w} words counted directly",
         "popc_only_peak": pr["popc"] / POPC_WORDS_PER_PAIR * rates["sm_count"] * clk / 1e9,
         "traffic": traffic("match_popc", "match_popc.cu", workload)}
    return _finish(r, f"{rk}; clock {pk} (measured-peaks file)")


def dominant(parts):
    """The roofline record of the longest phase, with the others under "other"."""
    parts = sorted(parts, key=lambda p: -p[0])
    out = dict(parts[0][1])
    if len(parts) > 1:
        out["other"] = [p[1] for p in parts[1:]] if len(parts) > 2 else parts[1][1]
    return out
