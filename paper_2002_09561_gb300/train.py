"""Train the learned-radius network on traces of the exact sphere decoder.

The traces are synthetic received vectors (Rayleigh channels, uniform QAM
symbols, SNR uniform in a range) whose ML point and ML metric the GPU sphere
decoder computes; the network is trained on them with the library's own
tensor-core forward/backward kernels (mdx_mlp_train_step) and evaluated on
held-out vectors against the paper's fixed radius: visited nodes,
vectors/s, radius-doubling rate, and identical decisions.

    python -m paper_2002_09561_gb300.train --out DIR [--traces 1000000]
writes DIR/mlp_<n>x<n>_<qam>qam.npy (FP32 parameter vector) and a .json
with the training configuration and the evaluation.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import mdx
from . import workload as wl

MODEL_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "models")


def model_path(n_tx: int, qam: int, directory: str = MODEL_DIR) -> str:
    return os.path.join(directory, f"mlp_{n_tx}x{n_tx}_{qam}qam.npy")


def load_model(ctx, n_tx: int, qam: int, directory: str = MODEL_DIR, max_train_batch: int = 0):
    """Create the context's network and load trained parameters; returns the metadata."""
    mdx.mlp_init(ctx, n_tx, qam, max_train_batch, seed=0)
    p = np.load(model_path(n_tx, qam, directory))
    mdx.mlp_set_params(ctx, p)
    meta = model_path(n_tx, qam, directory).replace(".npy", ".json")
    return json.load(open(meta)) if os.path.exists(meta) else {}


def _device_batch(torch, w, dev):
    return [torch.from_numpy(w[k]).to(dev) for k in ("H", "y", "noise_var")]


def generate_traces(torch, ctx, n_tx, qam, count, snr, seed, chunk, dev):
    """H, y, noise_var and the exact SD's ML indices / metric, on the device."""
    rng = np.random.default_rng(seed)
    snr_all = snr[0] + (snr[1] - snr[0]) * rng.random(count)
    Hs, ys, nvs, syms, mets = [], [], [], [], []
    p = mdx.make_params(n_tx, n_tx, qam, radius="paper")
    nodes = 0.0
    for s in range(0, count, chunk):
        c = min(chunk, count - s)
        w = wl.generate(seed, c, n_tx, n_tx, qam, snr_all[s:s + c], start=s)
        H, y, nv = _device_batch(torch, w, dev)
        sym, met, vst, st = mdx.detect("sd", ctx, p, H, y, nv)
        nodes += st[:, 0].double().sum().item()
        Hs.append(H)
        ys.append(y)
        nvs.append(nv)
        syms.append(sym)
        mets.append(met)
    torch.cuda.synchronize()
    return (torch.cat(Hs), torch.cat(ys), torch.cat(nvs), torch.cat(syms), torch.cat(mets)), nodes / count


def evaluate(torch, ctx, n_tx, qam, data, flags=0):
    """Plain (paper radius) vs learned radius on the same vectors."""
    H, y, nv = data
    out = {}
    for name, f in (("plain", 0), ("learned", mdx.MDX_LEARNED_RADIUS)):
        p = mdx.make_params(n_tx, n_tx, qam, radius="paper", flags=flags | f)
        res = mdx.detect("sd", ctx, p, H, y, nv)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        res = mdx.detect("sd", ctx, p, H, y, nv, out=res)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        nodes = res[3][:, 0].double().cpu().numpy()
        out[name] = {"vectors_per_s": H.shape[0] / (ms / 1e3), "ms": ms, "mean_nodes": float(nodes.mean()),
                     "p99_nodes": float(np.percentile(nodes, 99)),
                     "radius_doubling_rate": float((res[2] == 1).double().mean().item()),
                     "sym": res[0].cpu().numpy()}
    out["identical_decisions"] = bool((out["plain"]["sym"] == out["learned"]["sym"]).all())
    for k in ("plain", "learned"):
        del out[k]["sym"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-tx", type=int, default=16)
    ap.add_argument("--qam", type=int, default=16)
    ap.add_argument("--traces", type=int, default=1_000_000)
    ap.add_argument("--snr", type=str, default="8,20")
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--eval-vectors", type=int, default=100_000)
    ap.add_argument("--eval-seed", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--chunk", type=int, default=100_000)
    ap.add_argument("--out", type=str, default=MODEL_DIR)
    a = ap.parse_args()
    import torch

    dev = torch.device("cuda:0")
    n, qam = a.n_tx, a.qam
    snr = tuple(float(s) for s in a.snr.split(","))
    ctx = mdx.Context(0, max_batch=max(a.chunk, a.eval_vectors, a.batch), max_n_rx=n, max_n_tx=n)
    mdx.mlp_init(ctx, n, qam, a.batch, seed=a.seed)
    t0 = time.time()
    (H, y, nv, sym, met), trace_nodes = generate_traces(torch, ctx, n, qam, a.traces, snr, a.seed, a.chunk, dev)
    t_traces = time.time() - t0
    print(f"traces: {a.traces} in {t_traces:.1f} s (mean nodes {trace_nodes:.0f})", flush=True)
    params = mdx.make_params(n, n, qam)
    g = torch.Generator(device=dev)
    g.manual_seed(a.seed)
    steps = a.traces // a.batch
    total = steps * a.epochs
    t1 = time.time()
    hist = []
    k = 0
    for ep in range(a.epochs):
        perm = torch.randperm(a.traces, device=dev, generator=g)
        acc = torch.zeros(2, device=dev)
        for s in range(steps):
            idx = perm[s * a.batch:(s + 1) * a.batch]
            lr = a.lr * 0.5 * (1.0 + math.cos(math.pi * k / total))  # cosine decay
            loss, _ = mdx.mlp_train_step(ctx, params, H[idx].contiguous(), y[idx].contiguous(), nv[idx].contiguous(),
                                         sym[idx].contiguous(), met[idx].contiguous(), lr=lr)
            acc += loss
            k += 1
        acc = (acc / steps).cpu().numpy()
        hist.append([float(acc[0]), float(acc[1])])
        print(f"epoch {ep}: pinball {acc[0]:.4f} cross-entropy {acc[1]:.4f}", flush=True)
    t_train = time.time() - t1
    err = mdx.mlp_error(ctx)
    del H, y, nv, sym, met
    rng = np.random.default_rng(a.eval_seed)
    snr_e = snr[0] + (snr[1] - snr[0]) * rng.random(a.eval_vectors)
    w = wl.generate(a.eval_seed, a.eval_vectors, n, n, qam, snr_e)
    ev = evaluate(torch, ctx, n, qam, _device_batch(torch, w, dev))
    print(json.dumps(ev), flush=True)
    os.makedirs(a.out, exist_ok=True)
    np.save(model_path(n, qam, a.out), mdx.mlp_get_params(ctx, n, qam))
    meta = {"n_tx": n, "qam": qam, "traces": a.traces, "snr_db": list(snr), "seed": a.seed, "epochs": a.epochs,
            "batch": a.batch, "lr": a.lr, "trace_mean_nodes": trace_nodes, "seconds_traces": t_traces,
            "seconds_training": t_train, "loss_history": hist, "kernel_error_word": err,
            "evaluation": {"vectors": a.eval_vectors, "seed": a.eval_seed, **ev}}
    with open(model_path(n, qam, a.out).replace(".npy", ".json"), "w") as f:
        json.dump(meta, f, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
