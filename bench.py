#!/usr/bin/env python3
"""Throughput benchmark of the batched MIMO tree-search detectors.

One step = one pass of the detection path over one batch of synthetic
received vectors resident in device memory: FP64 QR, (for the learned
workloads) the network's features and tensor-core forward pass giving each
vector's initial radius, the tree search (FP32 partial distances), FP64
re-scoring of the final leaves, and the Gray-coded bit/symbol error count of
the batch.  The default workload is 16x16 MIMO, 16-QAM, exact sphere
decoding from the learned radius and first leaf (the trained model in
paper_2002_09561_gb300/models), 100,000 vectors per step with the SNR points
4, 6, ..., 20 dB interleaved (vector b at point b mod 9); the same batch is
also timed with the paper's radius r^2 = N M sigma^2 ("plain"), and both
arms' decisions (hence BER) must be identical.

Prints one JSON line (rank 0).  Launch: python bench.py [--gpus N] [--steps K]
[--warmup W] [--workload NAME] [--impl mdx|reference]; for N > 1 under
torch.distributed.run, one rank per GPU, each rank detecting its own shard.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEP_16 = [4.0, 6.0, 8.0, 10.0, 12.0, 14.0, 16.0, 18.0, 20.0]
WORKLOADS = {
    "16x16-16qam-sd-learned": dict(n=16, qam=16, snr=SWEEP_16, vectors=100_000, detector="sd", radius="paper",
                                   K=0, depth=0, learned=True),
    "16x16-16qam-sd": dict(n=16, qam=16, snr=SWEEP_16, vectors=100_000, detector="sd", radius="paper",
                           K=0, depth=0),
    "16x16-16qam-kbest64": dict(n=16, qam=16, snr=SWEEP_16, vectors=100_000, detector="kbest",
                                radius=math.inf, K=64, depth=0),
    "16x16-16qam-kbest256": dict(n=16, qam=16, snr=SWEEP_16, vectors=100_000, detector="kbest",
                                 radius=math.inf, K=256, depth=0),
    "100x100-64qam-hybrid32": dict(n=100, qam=64, snr=[20.0, 24.0, 28.0, 32.0], vectors=10_000,
                                   detector="hybrid", radius="paper", K=32, depth=4),
    "100x100-64qam-hybrid32-learned": dict(n=100, qam=64, snr=[20.0, 24.0, 28.0, 32.0], vectors=10_000,
                                           detector="hybrid", radius="paper", K=32, depth=4, learned=True),
    "100x100-64qam-hybrid128": dict(n=100, qam=64, snr=[20.0, 24.0, 28.0, 32.0], vectors=10_000,
                                    detector="hybrid", radius="paper", K=128, depth=4),
    # complex tree (one level per complex antenna, Q children): exact SD with the
    # learned radius and K-best on the paper's 16x16 64-QAM configuration
    # (the complex-tree SD runs one warp per vector without subtree splitting, so
    # its low-SNR tail is one warp's: the sweep starts at 12 dB, 20,000 vectors
    # per step, and the Babai control, whose open first sphere leaves that tail
    # unbounded, is not run)
    "16x16-16qam-sd-complex-learned": dict(n=16, qam=16, snr=[12.0, 14.0, 16.0, 18.0, 20.0], vectors=20_000,
                                           detector="sd", radius="paper", K=0, depth=0, learned=True,
                                           complex=True),
    "16x16-64qam-kbest32-complex": dict(n=16, qam=64, snr=[16.0, 20.0, 24.0, 28.0], vectors=100_000,
                                        detector="kbest", radius=math.inf, K=32, depth=0, complex=True),
    # the paper's controls: unsorted depth-first SD and the linear detectors
    "16x16-16qam-sd-natural": dict(n=16, qam=16, snr=[18.0, 20.0], vectors=100_000, detector="sd",
                                   radius="paper", K=0, depth=0, natural=True),
    "16x16-16qam-zf": dict(n=16, qam=16, snr=SWEEP_16, vectors=100_000, detector="linear", radius=math.inf,
                           K=0, depth=0),
    "16x16-16qam-mmse": dict(n=16, qam=16, snr=SWEEP_16, vectors=100_000, detector="linear", radius=math.inf,
                             K=0, depth=0, mmse=True),
    # uneven batch: n_tx = n_rx in {8, 16, 32, 64, 100}, {4, 16, 64}-QAM, SNR U(6, 30) dB,
    # half exact SD (paper radius, node budget) and half K-best K=64, one detect_mixed call
    "mixed-50k": dict(mixed=True, n=100, qam=64, antennas=(8, 16, 32, 64, 100), qams=(4, 16, 64),
                      snr=[6.0, 30.0], vectors=50_000, detector="mixed", radius="paper (SD) / none (K-best)",
                      K=64, depth=0, budget=20_000),
}
DEFAULT_WORKLOAD = "16x16-16qam-sd-learned"
METRIC = "decoded vectors/s at matched BER (16x16 16QAM, 100x100 64QAM), learned vs plain"
# DRAM bytes (read + write) of the dominant kernel per vector, from one ncu
# capture of the same kernel on a smaller run of the same workload (traffic
# grows with the number of vectors), with the capture it comes from and the
# code hash (code_hash: comments and spacing aside) of the kernel's sources
# it was taken on.  When the sources no longer hash to that value, the line
# reports no traffic until the kernel is captured again.
KERNEL_SOURCES = {
    "16x16-16qam-sd-learned": ("sd_group.cu", "sd_common.cuh", "mdx_internal.cuh"),
    "100x100-64qam-hybrid32-learned": ("kbest.cu", "warp_kbest.cuh", "mdx_internal.cuh"),
}
TRAFFIC_PER_VECTOR = {
    "16x16-16qam-sd-learned": ((225.208576e6 + 6.209024e6) / 30000,
                               "ncu capture of sd_group_kernel, 30,000 vectors of the learned 16x16 sweep "
                               "(profiles/sd_group_kernel_16x16_16qam_sweep_30k.md), scaled by vectors",
                               "41cf9bf6e4c91aa7"),
    "100x100-64qam-hybrid32-learned": ((516.954880e6 + 4.081664e6) / 2000,
                                       "ncu capture of hybrid_kernel, 2,000 vectors of the learned 100x100 "
                                       "workload (profiles/hybrid_kernel_100x100_64qam_2k.md), scaled by vectors",
                                       "e4500e2afb5bc28e"),
}


def code_hash(files, csrc=None):
    """sha256 (first 16 hex digits) of the given kernel sources with comments
    removed and white space collapsed, so that a comment edit keeps a
    capture's figures and a code change drops them."""
    csrc = csrc or os.path.join(ROOT, "paper_2002_09561_gb300", "csrc")
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(csrc, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


# Warp instructions the search kernel executes per branched node (all of the
# launch's instructions over its nodes), from the same kind of capture and
# tied to the sources in the same way: with the live node rate this gives the
# kernel's instruction-issue rate, the resource that bounds it.
INSTRUCTIONS_PER_NODE = {
    "16x16-16qam-sd-learned": (1.2128964723e10 / 297008606,
                               "ncu capture of sd_group_kernel, 30,000 vectors of the learned 16x16 sweep: "
                               "smsp__inst_executed.sum over the launch's branched nodes "
                               "(profiles/sd_group_kernel_16x16_16qam_sweep_30k.md)",
                               "41cf9bf6e4c91aa7"),
}


def _captured(table, workload):
    """(value, source) of the workload's entry in a table of ncu-captured
    figures if the kernel's sources are still the ones the capture was taken
    on, else (None, why)."""
    entry = table.get(workload)
    if not entry:
        return None, "no capture of the current kernel"
    if code_hash(KERNEL_SOURCES[workload]) != entry[2]:
        return None, f"the kernel changed since its capture ({entry[1]})"
    return entry[0], entry[1]


def instructions_per_node(workload):
    """(warp instructions per node, source) of the workload's capture, or
    (None, why)."""
    return _captured(INSTRUCTIONS_PER_NODE, workload)


def traffic_per_vector(workload):
    """(DRAM bytes per vector, source) of the workload's capture, or
    (None, why)."""
    return _captured(TRAFFIC_PER_VECTOR, workload)


FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (4 sub-partitions x 32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mdx", choices=["mdx", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-radius comparison arm")
    ap.add_argument("--vectors", type=int, default=0, help="override vectors per step (per GPU)")
    ap.add_argument("--snr", type=str, default="", help="comma-separated SNR points (override)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline duration")
    ap.add_argument("--no-autotune", action="store_true", help="uneven batch: keep the default tuning")
    ap.add_argument("--no-hybrid", action="store_true",
                    help="default workload: skip the 100x100 64-QAM hybrid record")
    return ap.parse_args()


def workload_of(args):
    w = dict(WORKLOADS[args.workload])
    if args.vectors:
        w["vectors"] = args.vectors
    if args.snr:
        w["snr"] = [float(s) for s in args.snr.split(",")]
    return w


def generate(w, seed, count, start=0):
    from paper_2002_09561_gb300 import workload as wl

    snr = np.asarray(w["snr"])[np.arange(start, start + count) % len(w["snr"])]
    return wl.generate(seed, count, w["n"], w["n"], w["qam"], snr, start=start)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


_MIXED_CACHE = {}


def mixed_table(w, seed, count):
    key = (seed, count, tuple(w["antennas"]), tuple(w["qams"]), tuple(w["snr"]), w["K"], w["budget"])
    if key not in _MIXED_CACHE:
        _MIXED_CACHE.clear()
        _MIXED_CACHE[key] = _mixed_table(w, seed, count)
    return _MIXED_CACHE[key]


def _mixed_table(w, seed, count):
    from paper_2002_09561_gb300 import mdx
    from paper_2002_09561_gb300 import workload as wl

    d = wl.generate_mixed_inputs(seed, count, antennas=w["antennas"], qams=w["qams"], snr_range=tuple(w["snr"]))
    reqs = mdx.make_requests(d["n"], d["n"], d["qam"], d["algo"], K=w["K"], budget=w["budget"],
                             h_offset=d["h_offset"], y_offset=d["y_offset"], sym_offset=d["sym_offset"])
    return d, reqs


def cpu_baseline_mixed(w, seed, target_s):
    """The FP64 oracle on the host cores over a bounded sample of the mix:
    chunks of requests spread over the whole table (every 97th request from
    a rotating start) until target_s seconds have been spent."""
    import oracle

    cores = host_cores()
    d, reqs = mixed_table(w, seed, w["vectors"])
    done = 0
    t0 = time.perf_counter()
    start = 0
    while time.perf_counter() - t0 < target_s and done < len(reqs):
        idx = np.arange(start, len(reqs), 97)[:max(cores, 16)]
        oracle.detect_mixed(reqs[idx], d["H"], d["y"], d["noise_var"][idx], want_gap=False)
        done += idx.size
        start += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "requests/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} requests spread over the {len(reqs)}-request mix (same seed) in {dt:.1f} s "
                      f"on {cores} threads"}


# The oracle's CPU baseline and error check run on a FIXED sample of the
# workload: its first PER_POINT[workload] vectors of every SNR point (vector b
# is at point b mod len(snr), so the sample is the first per_point * len(snr)
# vectors of the seed), the same vectors in both arms of the benchmark.
ORACLE_PER_POINT = {"16x16": 64, "100x100": 16}
ORACLE_PER_POINT_1CORE = {"16x16": 8, "100x100": 2}


def _size_key(w):
    return "100x100" if w["n"] > 32 else "16x16"


def oracle_sample(w, seed, per_point):
    return generate(w, seed, per_point * len(w["snr"]), start=0)


_HOST_CORES = []


def host_cores():
    """The oracle's OpenMP thread count before any single-core run changed it."""
    import oracle

    if not _HOST_CORES:
        _HOST_CORES.append(oracle.max_threads())
    return _HOST_CORES[0]


def oracle_detect(w, d, nthreads=0, want_gap=False):
    import oracle

    nthreads = nthreads or host_cores()
    algo = w["detector"] + ("_complex" if w.get("complex") else "")
    if algo == "linear":
        r = oracle.detect_linear("mmse" if w.get("mmse") else "zf", d["H"], d["y"], d["noise_var"], w["qam"])
        r["gap"] = r["margin"]
        return r
    return oracle.detect_batch(algo, d["H"], d["y"], d["noise_var"], w["qam"], radius=w["radius"],
                               K=max(w["K"], 1), depth=w["depth"], order="natural" if w.get("natural") else "se",
                               want_gap=want_gap, nthreads=nthreads)


def cpu_baseline(w, seed):
    """The FP64 oracle as it stands, on the host cores, over the fixed sample
    (all cores), and over a smaller fixed sample on one core."""
    import oracle

    if w.get("mixed"):
        return cpu_baseline_mixed(w, seed, 15.0)
    key = _size_key(w)
    cores = 1 if w["detector"] == "linear" else host_cores()
    d = oracle_sample(w, seed, ORACLE_PER_POINT[key])
    t0 = time.perf_counter()
    ref = oracle_detect(w, d)
    dt = time.perf_counter() - t0
    d1 = oracle_sample(w, seed, ORACLE_PER_POINT_1CORE[key])
    t1 = time.perf_counter()
    oracle_detect(w, d1)
    dt1c = time.perf_counter() - t1
    t1 = time.perf_counter()
    oracle_detect(w, d1, nthreads=1)
    dt1 = time.perf_counter() - t1
    B = len(d["noise_var"])
    algo = w["detector"] + ("_complex" if w.get("complex") else "")
    return {"value": B / dt, "unit": "vectors/s", "cores": cores, "kind": "oracle",
            "sample": f"fixed: the first {ORACLE_PER_POINT[key]} vectors of each of the {len(w['snr'])} SNR points "
                      f"({B} vectors, seed {seed}; {w['n']}x{w['n']} {w['qam']}-QAM {algo}, "
                      f"radius {w['radius'] if w['radius'] == 'paper' else 'none'}) in {dt:.2f} s on {cores} threads",
            "single_core": {"value": len(d1["noise_var"]) / dt1, "unit": "vectors/s", "cores": 1,
                            "all_cores_same_sample": len(d1["noise_var"]) / dt1c,
                            "sample": f"the first {ORACLE_PER_POINT_1CORE[key]} vectors of each SNR point "
                                      f"({len(d1['noise_var'])} vectors) in {dt1:.2f} s on one thread "
                                      f"({dt1c:.2f} s on {cores})"}}, d, ref


def gray_bit_errors(a, b, qam):
    """Bit errors per vector between complex indices a and b (Gray code per
    PAM dimension of q = k_re P + k_im)."""
    P = int(round(qam ** 0.5))
    ones = np.array([bin(v).count("1") for v in range(256)], dtype=np.int64)
    a = a.astype(np.int64)
    b = b.astype(np.int64)
    g = lambda k: k ^ (k >> 1)  # noqa: E731
    x = ones[g(a // P) ^ g(b // P)] + ones[g(a % P) ^ g(b % P)]
    return x.sum(axis=1)


def per_snr(w, outs, truth):
    """Per SNR point: BER, SER, mean / p99 visited nodes, radius-doubling and
    budget rates (vector b is at point b mod len(snr))."""
    sym, vst, st = outs
    B = sym.shape[0]
    pts = np.arange(B) % len(w["snr"])
    be = gray_bit_errors(sym, truth, w["qam"])
    se = (sym != truth).sum(axis=1)
    bits_per_vec = 2 * w["n"] * int(round(math.log2(int(round(w["qam"] ** 0.5)))))
    rows = []
    for i, s in enumerate(w["snr"]):
        m = pts == i
        nodes = st[m, 0].astype(np.float64)
        rows.append({"snr_db": s, "vectors": int(m.sum()), "ber": float(be[m].sum() / (m.sum() * bits_per_vec)),
                     "ser": float(se[m].sum() / (m.sum() * w["n"])), "mean_nodes": float(nodes.mean()),
                     "p99_nodes": float(np.percentile(nodes, 99)),
                     "radius_doubling_rate": float((vst[m] == 1).mean()),
                     "budget_rate": float((vst[m] == 2).mean())})
    return rows


def oracle_check(w, d, ref_gap, gpu_sym, gpu_met, seed):
    """The GPU's answers on the oracle's fixed sample against the oracle's:
    mismatches outside near-ties (SD: best/second-best gap < 1e-6; K-best,
    hybrid: a K / K+1 cut or final gap < 1e-5), near-tie fraction, largest
    relative metric error where the indices agree, and BER of both per SNR
    point."""
    tol = 1e-6 if w["detector"] == "sd" else (1e-8 if w["detector"] == "linear" else 1e-5)
    B = len(d["noise_var"])
    same = (gpu_sym[:B] == ref_gap["sym"]).all(axis=1)
    near = ref_gap["gap"] < tol
    rel = np.abs(gpu_met[:B] - ref_gap["metric"]) / np.maximum(ref_gap["metric"], 1e-300)
    pts = np.arange(B) % len(w["snr"])
    bits_per_vec = 2 * w["n"] * int(round(math.log2(int(round(w["qam"] ** 0.5)))))
    gb = gray_bit_errors(gpu_sym[:B], d["sym"], w["qam"])
    ob = gray_bit_errors(ref_gap["sym"], d["sym"], w["qam"])
    return {"vectors": int(B), "sample": f"the oracle's fixed sample (seed {seed})",
            "identical": int(same.sum()), "mismatches_outside_near_ties": int((~same & ~near).sum()),
            "differing_near_ties": int((~same & near).sum()), "near_tie_fraction": float(near.mean()),
            "near_tie_rule": f"gap < {tol:g} relative",
            "max_rel_metric_error": float(rel[same].max()) if same.any() else None,
            "ber_per_snr": [{"snr_db": s, "gpu": float(gb[pts == i].sum() / ((pts == i).sum() * bits_per_vec)),
                             "oracle": float(ob[pts == i].sum() / ((pts == i).sum() * bits_per_vec))}
                            for i, s in enumerate(w["snr"])]}


def run_reference(args, w, rank, world):
    """The oracle arm: every step detects the fixed sample on all host cores
    (the same vectors the GPU arm's cpu_baseline times)."""
    if rank != 0:
        return
    import oracle

    steps, warm = args.steps, args.warmup
    if w.get("mixed"):
        target = max(2.0, min(args.cpu_seconds, 60.0 / max(1, steps + warm)))
        for _ in range(warm):
            cpu_baseline_mixed(w, args.seed, target / 4)
        vals = []
        t0 = time.perf_counter()
        for _ in range(steps):
            vals.append(cpu_baseline_mixed(w, args.seed, target))
        wall = time.perf_counter() - t0
        value = float(np.mean([v["value"] for v in vals]))
        base = dict(vals[-1])
        base["value"] = value
    else:
        key = _size_key(w)
        d = oracle_sample(w, args.seed, ORACLE_PER_POINT[key])
        B = len(d["noise_var"])
        warm_d = oracle_sample(w, args.seed, 1)
        for _ in range(warm):
            oracle_detect(w, warm_d)
        t0 = time.perf_counter()
        for _ in range(steps):
            oracle_detect(w, d)
        wall = time.perf_counter() - t0
        value = B * steps / wall
        cores = 1 if w["detector"] == "linear" else host_cores()
        base = {"value": value, "unit": "vectors/s", "cores": cores, "kind": "oracle",
                "sample": f"fixed: the first {ORACLE_PER_POINT[key]} vectors of each of the {len(w['snr'])} SNR "
                          f"points ({B} vectors, seed {args.seed}) per step, {steps} steps on {cores} threads"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": base["unit"], "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * wall / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, w, world), "cpu_baseline": base,
            "e2e": {"value": value, "unit": base["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(args, w, world):
    if w.get("mixed"):
        return {"workload": args.workload, "n_tx = n_rx": list(w["antennas"]), "qam": list(w["qams"]),
                "snr_db": f"uniform {w['snr'][0]}..{w['snr'][1]}",
                "detectors": f"half exact SD (r^2 = N M sigma^2, node budget {w['budget']}), half K-best "
                             f"K={w['K']} (no radius)",
                "requests_per_step_per_gpu": w["vectors"], "global_batch": w["vectors"] * world,
                "launch": "one captured CUDA graph per step (QR per antenna class + one persistent search kernel)",
                "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                "l2": "inputs larger than L2 (no flush)"}
    return {"workload": args.workload, "n_tx": w["n"], "n_rx": w["n"], "qam": w["qam"],
            "detector": w["detector"] + (" (complex tree)" if w.get("complex") else "")
            + (" (natural child order)" if w.get("natural") else "") + (" MMSE" if w.get("mmse") else "")
            + (" ZF" if w["detector"] == "linear" and not w.get("mmse") else ""), "K": w["K"] or None, "hybrid_depth": w["depth"] or None,
            "initial_radius": "r^2 = N M sigma^2" if w["radius"] == "paper" else "none",
            "snr_db": w["snr"], "vectors_per_step_per_gpu": w["vectors"], "global_batch": w["vectors"] * world,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (no flush)"}


def main():
    args = parse()
    w = workload_of(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and "RANK" not in os.environ:
        raise SystemExit("for --gpus > 1 launch under torch.distributed.run")

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")
        run_reference(args, w, rank, world)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2002_09561_gb300 import mdx

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    if w.get("mixed"):
        main_mixed(args, w, rank, world, local, dev, dist, torch, mdx)
        return

    from paper_2002_09561_gb300 import replicas

    B, n, qam = w["vectors"], w["n"], w["qam"]
    start, _ = replicas.shard(rank, world, B)
    data = generate(w, args.seed, B, start=start)
    H = torch.from_numpy(data["H"]).to(dev)
    y = torch.from_numpy(data["y"]).to(dev)
    nv = torch.from_numpy(data["noise_var"]).to(dev)
    truth = torch.from_numpy(data["sym"]).to(dev)
    ctx = mdx.Context(local, max_batch=B, max_n_rx=n, max_n_tx=n)
    probe = mdx.measure_peaks(local)
    learned = bool(w.get("learned"))
    model_meta = None
    if learned:
        from paper_2002_09561_gb300 import train

        model_meta = train.load_model(ctx, n, qam)
    flags = 0
    if learned:
        # the ordering head exists for models with full features (detect_sd)
        flags = mdx.MDX_LEARNED_RADIUS | (mdx.MDX_LEARNED_ORDER if w["detector"] == "sd" else 0)
    base_flags = 0
    if w.get("complex"):
        base_flags |= mdx.MDX_COMPLEX_TREE
    if w.get("natural"):
        base_flags |= mdx.MDX_ORDER_NATURAL
    if w.get("mmse"):
        base_flags |= mdx.MDX_LINEAR_MMSE
    flags |= base_flags
    params = mdx.make_params(n, n, qam, radius=w["radius"], K=max(w["K"], 1), depth=w["depth"], flags=flags)
    algo = w["detector"]
    out = mdx._outputs(B, n, dev, True)
    stream = torch.cuda.current_stream(dev)
    arm = Arm(torch, mdx, replicas, ctx, algo, H, y, nv, truth, qam, stream, dist, dev, local)

    ms, (qr_ms, search_ms, calls), errs, sampler = arm.time(params, out, args.steps, args.warmup)
    value = B * world * args.steps / (ms / 1e3)
    host = lambda o: (o[0].cpu().numpy(), o[2].cpu().numpy(), o[3].cpu().numpy())  # noqa: E731
    main_host = host(out)
    bits_vec = 2 * n * int(round(math.log2(int(round(qam ** 0.5)))))
    plain = babai = None
    plain_qr = None
    if learned and not args.no_plain:
        pparams = mdx.make_params(n, n, qam, radius=w["radius"], K=max(w["K"], 1), depth=w["depth"],
                                  flags=base_flags)
        pout = mdx._outputs(B, n, dev, True)
        pms, pprof, perrs, _ = arm.time(pparams, pout, args.steps, 1)
        plain_qr = pprof
        ph = host(pout)
        plain = {"value": B * world * args.steps / (pms / 1e3), "unit": "vectors/s", "ms_per_step": pms / args.steps,
                 "initial_radius": "r^2 = N M sigma^2", "mean_nodes": float(ph[2][:, 0].mean()),
                 "identical_decisions": bool(torch.equal(pout[0], out[0])),
                 "ber": int(perrs[0]) / (B * bits_vec), "speedup_learned": pms / ms,
                 "search_ms_per_launch": pprof[1] / max(pprof[2], 1), "per_snr": per_snr(w, ph, data["sym"])}
        if algo == "sd" and not w.get("complex"):
            # the Babai-radius control: no initial radius, so the first leaf the
            # Schnorr-Euchner descent reaches (the Babai / ZF-SIC point) sets r^2
            bsteps = max(1, min(args.steps, 5))
            bparams = mdx.make_params(n, n, qam, radius=math.inf, flags=base_flags)
            bout = mdx._outputs(B, n, dev, True)
            bms, bprof, berrs, _ = arm.time(bparams, bout, bsteps, 1)
            bh = host(bout)
            babai = {"value": B * world * bsteps / (bms / 1e3), "unit": "vectors/s", "ms_per_step": bms / bsteps,
                     "steps": bsteps, "initial_radius": "none (the Babai point reached by the first descent sets it)",
                     "mean_nodes": float(bh[2][:, 0].mean()),
                     "identical_decisions": bool(torch.equal(bout[0], out[0])),
                     "ber": int(berrs[0]) / (B * bits_vec), "speedup_learned": (bms / bsteps) / (ms / args.steps),
                     "search_ms_per_launch": bprof[1] / max(bprof[2], 1), "per_snr": per_snr(w, bh, data["sym"])}

    stats = main_host[2]
    vst = main_host[1]
    tot = replicas.sum_counters({"bit_errors": int(errs[0]), "symbol_errors": int(errs[1]),
                                 "budget_exceeded": int((vst == 2).sum()), "radius_doublings": int((vst == 1).sum()),
                                 "nodes": int(stats[:, 0].sum())}, dist, dev)
    bit_err, sym_err = tot["bit_errors"], tot["symbol_errors"]
    bits = B * world * bits_vec

    # dominant kernel: the tree search; algorithmic FP32 flops per launch from the
    # kernel's own count, sum over branched nodes at row i of 2(n-1-i) + 4P
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = search_roofline(args.workload, algo, stats, search_ms, calls, qr_ms, sms, probe, B)
    # the FP64 QR (timed in the arm without the network, whose QR interval is
    # the QR kernel and a 4-byte counter reset)
    qprof = plain_qr if plain_qr is not None else ((qr_ms, search_ms, calls) if not learned else None)
    qr_roof = qr_roofline(n, n, B, qprof, sms, probe) if qprof else None

    e2e = None
    if not args.no_e2e:
        # the same metric through the C ABI with host buffers: pinned host inputs
        # copied in and results copied out inside the timed region
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()  # noqa: E731
        hH, hy, hnv = pin(data["H"]), pin(data["y"]), pin(data["noise_var"])
        hsym = torch.empty((B, n), dtype=torch.uint8).pin_memory().numpy()
        hmet = torch.empty(B, dtype=torch.float64).pin_memory().numpy()
        hvst = torch.empty(B, dtype=torch.int32).pin_memory().numpy()
        for _ in range(max(1, args.warmup)):
            mdx.detect_host(algo, ctx, params, hH, hy, hnv, hsym, hmet, hvst, stream=stream)
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            mdx.detect_host(algo, ctx, params, hH, hy, hnv, hsym, hmet, hvst, stream=stream)
        el = replicas.max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": B * world * args.steps / el, "unit": "vectors/s",
               "h2d_bytes_per_step": int(hH.nbytes + hy.nbytes + hnv.nbytes),
               "d2h_bytes_per_step": int(hsym.nbytes + hmet.nbytes + hvst.nbytes)}

    cpu = check = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, d_s, _ = cpu_baseline(w, args.seed)
        ref = oracle_detect(w, d_s, want_gap=True)
        check = oracle_check(w, d_s, ref, main_host[0], out[1].cpu().numpy(), args.seed)

    hybrid = None
    if args.workload == DEFAULT_WORKLOAD and not args.no_hybrid:
        ctx.close()
        ctx = None
        del H, y, nv, truth, out
        torch.cuda.empty_cache()
        hybrid = hybrid_record(args, rank, world, local, dev, dist, torch, mdx, replicas, probe)

    if rank == 0:
        cfg = config_of(args, w, world)
        if learned:
            cfg["initial_radius"] = ("learned (network of the models directory), capped by the distance of the "
                                     "network's top-ranked leaf, doubled on an empty sphere")
            cfg["model"] = {k: model_meta.get(k) for k in ("traces", "snr_db", "epochs", "seed")} if model_meta else None
        line = {"metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 search, f64 QR and re-scoring",
                "data": "synthetic (seeded Rayleigh channels, uniform QAM symbols, AWGN)",
                "config": cfg, "roofline": roof, "qr_roofline": qr_roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_call(algo, learned, n) * args.steps, "clocks": sampler.summary(),
                "measured_peaks": probe, "oracle_check": check, "plain": plain, "babai": babai,
                "quality": {"ber": bit_err / bits, "ser": sym_err / (B * world * n),
                            "budget_exceeded": tot["budget_exceeded"], "radius_doublings": tot["radius_doublings"],
                            "mean_nodes": tot["nodes"] / (B * world), "max_nodes_rank0": int(stats[:, 0].max()),
                            "per_snr_rank0": per_snr(w, main_host, data["sym"])},
                "hybrid_100x100": hybrid}
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def launches_per_call(algo, learned, n):
    """Kernels of one timed step: the QR, the network (features, three GEMMs,
    radius) when learned, the sphere decoder's heaviest-first ordering (three
    kernels) for detect_sd, the search, and the error count."""
    k = 3 + (5 if learned else 0)
    if algo == "sd":
        k += 3
    return k


class Arm:
    """Times one detector configuration: W untimed calls, then K calls (each
    a detection plus the batch's bit/symbol error count) between CUDA events
    on the launching stream, bracketed by barriers and synchronizations; the
    elapsed time is the maximum over ranks.  The library's own events give
    the QR and search kernels' share."""

    def __init__(self, torch, mdx, replicas, ctx, algo, H, y, nv, truth, qam, stream, dist, dev, local):
        self.torch, self.mdx, self.replicas, self.ctx, self.algo = torch, mdx, replicas, ctx, algo
        self.H, self.y, self.nv, self.truth, self.qam = H, y, nv, truth, qam
        self.stream, self.dist, self.dev, self.local = stream, dist, dev, local

    def time(self, prm, outs, steps, warm):
        torch, mdx = self.torch, self.mdx

        def step():
            mdx.detect(self.algo, self.ctx, prm, self.H, self.y, self.nv, stream=self.stream, out=outs)
            return mdx.count_errors(self.ctx, outs[0], self.truth, self.qam, stream=self.stream)

        for _ in range(warm):
            step()
        torch.cuda.synchronize(self.dev)
        if self.dist is not None:
            self.dist.barrier()
        torch.cuda.synchronize(self.dev)
        sampler = ClockSampler(self.local)
        sampler.start()
        self.ctx.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        errs = None
        for _ in range(steps):
            errs = step()
        e1.record(self.stream)
        torch.cuda.synchronize(self.dev)
        if self.dist is not None:
            self.dist.barrier()
        torch.cuda.synchronize(self.dev)
        sampler.stop()
        el = e0.elapsed_time(e1)
        prof = self.ctx.profile_read()
        self.ctx.profile(False)
        el = self.replicas.max_over_ranks(el, self.dist, self.dev)
        return el, prof, errs.cpu().numpy(), sampler


def search_roofline(workload, algo, stats, search_ms, calls, qr_ms, sms, probe, B):
    """FP32 roofline of the search kernel: algorithmic flops (the kernel's own
    count, sum over branched nodes at row i of 2(n-1-i) + 4P) per launch over
    the launch's CUDA-event duration, against the derived FP32 peak (SMs x
    128 lanes x 2 x the maximum SM clock) and beside the probe's measured
    FFMA rate."""
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops = float(stats[:, 4].sum())
    per_launch_s = (search_ms / max(calls, 1)) / 1e3
    achieved = flops / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    tpv, tsrc = traffic_per_vector(workload)
    nodes = float(stats[:, 0].sum())
    # the bound in practice: instruction issue (4 schedulers per SM, one warp
    # instruction per cycle each), at the captured instructions per node
    ipn, isrc = instructions_per_node(workload)
    issue_peak = sms * 4 * sm_max * 1e6
    issue = {"warp_instructions_per_node": ipn, "source": isrc}
    if ipn and per_launch_s > 0:
        rate = ipn * nodes / per_launch_s
        issue.update({"achieved": rate / 1e12, "peak": issue_peak / 1e12, "unit": "T warp instructions/s",
                      "frac": rate / issue_peak,
                      "peak_source": f"derived: {sms} SMs x 4 schedulers x 1 instruction per cycle x {sm_max:.0f} MHz"})
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "measured_fma_peak": probe["fp32_fma_tflops"], "frac_of_measured": achieved / probe["fp32_fma_tflops"],
            "traffic": tpv * B if tpv else None,
            "traffic_unit": "bytes per launch (dram read + write)" if tpv else None,
            "traffic_source": tsrc,
            "kernel": f"{algo} search", "search_ms_per_launch": 1e3 * per_launch_s,
            "qr_ms_per_launch": qr_ms / max(calls, 1),
            "nodes_per_s": nodes / per_launch_s if per_launch_s > 0 else None,
            "nodes_per_s_per_sm": nodes / per_launch_s / sms if per_launch_s > 0 else None,
            "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
            "issue": issue}


def qr_roofline(n_rx, n_tx, B, prof, sms, probe):
    """FP64 roofline of the QR: 8 (N M^2 - M^3 / 3) real flops per complex
    Householder QR of an N x M matrix, over the QR interval's CUDA-event
    duration, against the derived FP64 peak (SMs x 2 FP64 FMA lanes x 2 x the
    maximum SM clock) and the probe's measured FP64 FMA and MMA rates."""
    qr_ms, _, calls = prof
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * 2 * 2 * sm_max * 1e6 / 1e12
    N, M = float(n_rx), float(n_tx)
    flops = 8.0 * (N * M * M - M ** 3 / 3.0) * B
    s = (qr_ms / max(calls, 1)) / 1e3
    achieved = flops / s / 1e12 if s > 0 else 0.0
    meas = max(probe["fp64_fma_tflops"], probe["fp64_mma_tflops"])
    return {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "measured_fp64_peak": meas, "frac_of_measured": achieved / meas, "ms_per_launch": 1e3 * s,
            "flops_per_matrix": flops / B, "matrices": B,
            "peak_source": f"derived: {sms} SMs x 2 FP64 FMA lanes x 2 x {sm_max:.0f} MHz; measured = the larger "
                           "of the FP64 FMA and m8n8k4 MMA probes",
            "interval": "QR kernel and the 4-byte work-counter reset"}


def hybrid_record(args, rank, world, local, dev, dist, torch, mdx, replicas, probe):
    """The metric's second configuration: 100x100 64-QAM hybrid (depth 4,
    K = 32) at 20/24/28/32 dB, 10,000 vectors per step, learned radius
    against the paper radius; each arm's throughput, decisions, BER, nodes,
    per-SNR figures, the search kernel's FP32 fraction, the QR's FP64
    fraction, and the oracle on a fixed sample beside it."""
    from paper_2002_09561_gb300 import train

    w = dict(WORKLOADS["100x100-64qam-hybrid32-learned"])
    B, n, qam = w["vectors"], w["n"], w["qam"]
    start, _ = replicas.shard(rank, world, B)
    data = generate(w, args.seed, B, start=start)
    H = torch.from_numpy(data["H"]).to(dev)
    y = torch.from_numpy(data["y"]).to(dev)
    nv = torch.from_numpy(data["noise_var"]).to(dev)
    truth = torch.from_numpy(data["sym"]).to(dev)
    ctx = mdx.Context(local, max_batch=B, max_n_rx=n, max_n_tx=n)
    meta = train.load_model(ctx, n, qam)
    stream = torch.cuda.current_stream(dev)
    arm = Arm(torch, mdx, replicas, ctx, "hybrid", H, y, nv, truth, qam, stream, dist, dev, local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    bits_vec = 2 * n * int(round(math.log2(int(round(qam ** 0.5)))))
    rec = {"workload": "100x100-64qam-hybrid32", "vectors_per_step_per_gpu": B, "snr_db": w["snr"], "K": w["K"],
           "hybrid_depth": w["depth"], "model": {k: meta.get(k) for k in ("traces", "snr_db", "epochs", "seed")}}
    outs = {}
    for name, fl, warm in (("learned", mdx.MDX_LEARNED_RADIUS, args.warmup), ("plain", 0, 1)):
        prm = mdx.make_params(n, n, qam, radius="paper", K=w["K"], depth=w["depth"], flags=fl)
        o = mdx._outputs(B, n, dev, True)
        ms, prof, errs, sampler = arm.time(prm, o, args.steps, warm)
        hh = (o[0].cpu().numpy(), o[2].cpu().numpy(), o[3].cpu().numpy())
        outs[name] = (o, hh)
        r = {"value": B * world * args.steps / (ms / 1e3), "unit": "vectors/s", "ms_per_step": ms / args.steps,
             "ber": int(errs[0]) / (B * bits_vec), "mean_nodes": float(hh[2][:, 0].mean()),
             "roofline": search_roofline("100x100-64qam-hybrid32-" + name, "hybrid", hh[2], prof[1], prof[2], prof[0],
                                         sms, probe, B),
             "clocks": sampler.summary(), "per_snr": per_snr(w, hh, data["sym"])}
        if name == "plain":
            r["qr_roofline"] = qr_roofline(n, n, B, prof, sms, probe)
        rec[name] = r
    rec["identical_decisions"] = bool(torch.equal(outs["learned"][0][0], outs["plain"][0][0]))
    rec["speedup_learned"] = rec["learned"]["value"] / rec["plain"]["value"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, d_s, ref = cpu_baseline(w, args.seed)
        rec["cpu_baseline"] = cpu
        rec["oracle_check"] = oracle_check(w, d_s, ref, outs["learned"][1][0], outs["learned"][0][1].cpu().numpy(),
                                           args.seed)
    ctx.close()
    return rec


def main_mixed(args, w, rank, world, local, dev, dist, torch, mdx):
    """The uneven batch: autotune once (untimed), then time detect_mixed
    replayed from its captured CUDA graph."""
    from paper_2002_09561_gb300 import replicas

    B = w["vectors"]
    d, reqs = mixed_table(w, args.seed + rank, B)  # each rank its own table (seed + rank)
    H = torch.from_numpy(d["H"]).to(dev)
    y = torch.from_numpy(d["y"]).to(dev)
    nv = torch.from_numpy(d["noise_var"]).to(dev)
    ctx = mdx.Context(local, max_batch=B, max_n_rx=max(w["antennas"]), max_n_tx=max(w["antennas"]))
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        tune = None if args.no_autotune else mdx.autotune_mixed(ctx, reqs, H, y, nv, stream=stream)
        out = mdx.detect_mixed(ctx, reqs, H, y, nv, stream=stream)
    flags = mdx.MDX_GRAPH
    for _ in range(args.warmup):
        mdx.detect_mixed(ctx, reqs, H, y, nv, flags=flags, stream=stream, out=out)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        mdx.detect_mixed(ctx, reqs, H, y, nv, flags=flags, stream=stream, out=out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.stop()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = B * world * args.steps / (ms / 1e3)
    # kernel split from one profiled direct call (events around QR and search)
    ctx.profile(True)
    prof_out = mdx.detect_mixed(ctx, reqs, H, y, nv, stream=stream)
    torch.cuda.synchronize(dev)
    qr_ms, search_ms, calls = ctx.profile_read()
    ctx.profile(False)
    same = all(bool(torch.equal(a, b)) for a, b in zip(prof_out, out))
    sym = out[0].cpu().numpy()
    vst = out[2].cpu().numpy()
    stats = out[3].cpu().numpy()
    # symbol errors per request class
    err = sym[:d["sym"].size] != d["sym"]
    owner = np.repeat(np.arange(B), d["n"])
    req_err = np.bincount(owner, weights=err, minlength=B)
    ser = float(req_err.sum() / d["sym"].size)
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops = float(stats[:, 4].sum())
    per_launch_s = (search_ms / max(calls, 1)) / 1e3
    achieved = flops / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "mixed_kernel (persistent search)",
            "search_ms_per_launch": 1e3 * per_launch_s, "qr_ms_per_launch": qr_ms / max(calls, 1),
            "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz"}
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hH, hy, hnv = pin(d["H"]), pin(d["y"]), pin(d["noise_var"])
        hsym = pin(np.zeros(d["sym"].size, np.uint8))
        hmet = pin(np.zeros(B))
        hvst = pin(np.zeros(B, np.int32))
        for _ in range(max(1, args.warmup)):
            mdx.detect_mixed_host(ctx, reqs, hH, hy, hnv, hsym, hmet, hvst, flags=flags, stream=stream)
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            mdx.detect_mixed_host(ctx, reqs, hH, hy, hnv, hsym, hmet, hvst, flags=flags, stream=stream)
        el = replicas.max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": B * world * args.steps / el, "unit": "requests/s",
               "h2d_bytes_per_step": int(hH.nbytes + hy.nbytes + hnv.nbytes),
               "d2h_bytes_per_step": int(hsym.nbytes + hmet.nbytes + hvst.nbytes)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_mixed(w, args.seed, args.cpu_seconds)
    if rank == 0:
        n_runs = len(np.unique(d["n"]))
        sd = reqs["algo"] == 0
        line = {"metric": METRIC, "value": value, "unit": "requests/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 search, f64 QR and re-scoring",
                "data": "synthetic (seeded Rayleigh channels, uniform QAM symbols, AWGN)",
                "config": config_of(args, w, world), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": (n_runs + 1) * args.steps, "clocks": sampler.summary(), "autotune": tune,
                "graph_matches_direct_call": same,
                "quality": {"ser": ser, "ser_sd": float(req_err[sd].sum() / d["n"][sd].sum()),
                            "ser_kbest": float(req_err[~sd].sum() / d["n"][~sd].sum()),
                            "sd_budget_exceeded": int((vst[sd] == 2).sum()), "sd_requests": int(sd.sum()),
                            "mean_nodes_sd": float(stats[sd, 0].mean()),
                            "mean_nodes_kbest": float(stats[~sd, 0].mean())}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
