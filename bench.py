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
import json
import math
import os
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
    # its low-SNR tail is one warp's: the sweep starts at 12 dB)
    "16x16-16qam-sd-complex-learned": dict(n=16, qam=16, snr=[12.0, 14.0, 16.0, 18.0, 20.0], vectors=100_000,
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
METRIC = "decoded vectors/s at matched BER (16x16 16QAM, 100x100 64QAM), learned vs plain"
# DRAM bytes (read + write) of the dominant kernel per vector, from one ncu
# capture of the same kernel on a smaller run of the same workload (traffic
# grows with the number of vectors); None where no capture of the current
# kernel exists.  Captures: sd_kernel, 20,000 vectors: 154.2 MB read + 4.8 MB
# written; hybrid_kernel, 2,000 vectors: 517.5 MB read + 4.1 MB written.
TRAFFIC_PER_VECTOR = {"16x16-16qam-sd-learned": (154.186752e6 + 4.764160e6) / 20000,
                      "100x100-64qam-hybrid32-learned": (517.457664e6 + 4.140800e6) / 2000}
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (4 sub-partitions x 32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mdx", choices=["mdx", "reference"])
    ap.add_argument("--workload", default="16x16-16qam-sd-learned", choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-radius comparison arm")
    ap.add_argument("--vectors", type=int, default=0, help="override vectors per step (per GPU)")
    ap.add_argument("--snr", type=str, default="", help="comma-separated SNR points (override)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline duration")
    ap.add_argument("--no-autotune", action="store_true", help="uneven batch: keep the default tuning")
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

    cores = oracle.max_threads()
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


def cpu_baseline(w, seed, target_s, start_offset):
    """The FP64 oracle on the host cores over a bounded sample of the same
    workload: vectors taken round-robin over the SNR points, in chunks, until
    target_s seconds have been spent."""
    import oracle

    if w.get("mixed"):
        return cpu_baseline_mixed(w, seed, target_s)
    cores = oracle.max_threads()
    algo = w["detector"] + ("_complex" if w.get("complex") else "")
    if algo == "linear":
        cores = 1  # numpy, one thread
    done = 0
    t0 = time.perf_counter()
    chunk = max(cores, 16)
    pos = start_offset
    while time.perf_counter() - t0 < target_s and done < w["vectors"]:
        d = generate(w, seed, chunk, start=pos)
        if algo == "linear":
            oracle.detect_linear("mmse" if w.get("mmse") else "zf", d["H"], d["y"], d["noise_var"], w["qam"])
        else:
            oracle.detect_batch(algo, d["H"], d["y"], d["noise_var"], w["qam"], radius=w["radius"],
                                K=max(w["K"], 1), depth=w["depth"],
                                order="natural" if w.get("natural") else "se")
        done += chunk
        pos += chunk
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "vectors/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} vectors of the same workload ({w['n']}x{w['n']} {w['qam']}-QAM "
                      f"{algo}, SNR points round-robin) in {dt:.1f} s on {cores} threads"}


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    target = max(2.0, min(args.cpu_seconds, 60.0 / max(1, steps + warm)))
    for _ in range(warm):
        cpu_baseline(w, args.seed, target / 4, 0)
    vals = []
    t0 = time.perf_counter()
    for k in range(steps):
        vals.append(cpu_baseline(w, args.seed, target, 0))
    wall = time.perf_counter() - t0
    value = float(np.mean([v["value"] for v in vals]))
    base = dict(vals[-1])
    base["value"] = value
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
    learned = bool(w.get("learned"))
    model_meta = None
    if learned:
        from paper_2002_09561_gb300 import train

        model_meta = train.load_model(ctx, n, qam)
    flags = 0
    if learned:
        # the ordering head exists for models with full features (detect_sd)
        flags = mdx.MDX_LEARNED_RADIUS | (mdx.MDX_LEARNED_ORDER if w["detector"] == "sd" else 0)
    if w.get("complex"):
        flags |= mdx.MDX_COMPLEX_TREE
    if w.get("natural"):
        flags |= mdx.MDX_ORDER_NATURAL
    if w.get("mmse"):
        flags |= mdx.MDX_LINEAR_MMSE
    params = mdx.make_params(n, n, qam, radius=w["radius"], K=max(w["K"], 1), depth=w["depth"], flags=flags)
    algo = w["detector"]
    out = mdx._outputs(B, n, dev, True)
    stream = torch.cuda.current_stream(dev)

    def timed(prm, outs, steps, warm):
        def step():
            mdx.detect(algo, ctx, prm, H, y, nv, stream=stream, out=outs)
            return mdx.count_errors(ctx, outs[0], truth, qam, stream=stream)

        for _ in range(warm):
            step()
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(local)
        sampler.start()
        ctx.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        errs = None
        for _ in range(steps):
            errs = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        sampler.stop()
        el = e0.elapsed_time(e1)
        prof = ctx.profile_read()
        ctx.profile(False)
        el = replicas.max_over_ranks(el, dist, dev)
        return el, prof, errs, sampler

    ms, (qr_ms, search_ms, calls), errs, sampler = timed(params, out, args.steps, args.warmup)
    value = B * world * args.steps / (ms / 1e3)
    plain = None
    if learned and not args.no_plain:
        pparams = mdx.make_params(n, n, qam, radius=w["radius"], K=max(w["K"], 1), depth=w["depth"],
                                  flags=mdx.MDX_COMPLEX_TREE if w.get("complex") else 0)
        pout = mdx._outputs(B, n, dev, True)
        pms, _, perrs, _ = timed(pparams, pout, args.steps, 1)
        same = bool(torch.equal(pout[0], out[0]))
        pst = pout[3].cpu().numpy()
        plain = {"value": B * world * args.steps / (pms / 1e3), "unit": "vectors/s", "ms_per_step": pms / args.steps,
                 "initial_radius": "r^2 = N M sigma^2", "mean_nodes": float(pst[:, 0].mean()),
                 "identical_decisions": same,
                 "ber": int(perrs[0]) / (B * n * 2 * int(round(math.log2(int(round(qam ** 0.5)))))),
                 "speedup_learned": (B * world * args.steps / (ms / 1e3)) / (B * world * args.steps / (pms / 1e3))}

    stats = out[3].cpu().numpy()
    vst = out[2].cpu().numpy()
    P = int(round(qam ** 0.5))
    # whole-job counters (one sum-reduction over the ranks)
    tot = replicas.sum_counters({"bit_errors": int(errs[0]), "symbol_errors": int(errs[1]),
                                 "budget_exceeded": int((vst == 2).sum()), "radius_doublings": int((vst == 1).sum()),
                                 "nodes": int(stats[:, 0].sum())}, dist, dev)
    bit_err, sym_err = tot["bit_errors"], tot["symbol_errors"]
    bits = B * world * n * 2 * int(round(math.log2(P)))

    # dominant kernel: the tree search; algorithmic FP32 flops per launch from the
    # kernel's own count, sum over branched nodes at row i of 2(n-1-i) + 4P
    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops = float(stats[:, 4].sum())
    per_launch_s = (search_ms / max(calls, 1)) / 1e3
    achieved = flops / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    tpv = TRAFFIC_PER_VECTOR.get(args.workload)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": tpv * B if tpv else None, "traffic_unit": "bytes per launch (ncu capture, scaled by vectors)",
            "kernel": f"{algo} search", "search_ms_per_launch": 1e3 * per_launch_s,
            "qr_ms_per_launch": qr_ms / max(calls, 1),
            "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz"}

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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.seed, args.cpu_seconds, 0)

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
                "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": (8 if learned else 3) * args.steps, "clocks": sampler.summary(), "plain": plain,
                "quality": {"ber": bit_err / bits, "ser": sym_err / (B * world * n),
                            "budget_exceeded": tot["budget_exceeded"], "radius_doublings": tot["radius_doublings"],
                            "mean_nodes": tot["nodes"] / (B * world), "max_nodes_rank0": int(stats[:, 0].max())}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


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
