"""Train the learned-radius network on traces of the exact sphere decoder.

The traces are synthetic received vectors (Rayleigh channels, uniform QAM
symbols, SNR uniform in a range) whose ML point and ML metric the GPU sphere
decoder computes; the network is trained on them with the library's own
tensor-core forward/backward kernels (mdx_mlp_train_step) and evaluated on
held-out vectors against the paper's fixed radius: visited nodes,
vectors/s, radius-doubling rate, and identical decisions.

    python -m paper_2002_09561_gb300.train --out DIR [--traces 1000000]
writes DIR/mlp_<n>x<n>_<qam>qam.npy (FP32 parameter vector) and a .json
with the training configuration and the evaluation.  With --detector hybrid
(large systems, e.g. --n-tx 100 --qam 64 --snr 20,32) the model has summary
features and a radius head trained on the plain hybrid's answer metrics.
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


def device_workload(torch, gen, count, n, qam, snr, dev):
    """Rayleigh channels, uniform QAM symbols and AWGN drawn on the device with
    torch's seeded generator (training traces for large systems, where the
    host generator would dominate): the distributions of workload.generate."""
    P = int(round(qam ** 0.5))
    alpha = math.sqrt(3.0 / (2.0 * (qam - 1)))
    H = torch.randn((count, n, n, 2), generator=gen, device=dev, dtype=torch.float64) * math.sqrt(0.5)
    q = torch.randint(0, qam, (count, n), generator=gen, device=dev)
    s = torch.stack([(2 * (q // P) - (P - 1)) * alpha, (2 * (q % P) - (P - 1)) * alpha], dim=-1).double()
    Hc = torch.complex(H[..., 0], H[..., 1])
    sc = torch.complex(s[..., 0], s[..., 1])
    yc = torch.einsum("bnm,bm->bn", Hc, sc)
    nv = torch.as_tensor(wl.noise_var_from_snr(snr), device=dev, dtype=torch.float64)
    w = torch.randn((count, n, 2), generator=gen, device=dev, dtype=torch.float64) * torch.sqrt(nv / 2.0)[:, None, None]
    y = torch.stack([yc.real, yc.imag], dim=-1) + w
    return H.contiguous(), y.contiguous(), nv.contiguous(), q.to(torch.uint8)


def main_hybrid(a):
    """Radius model for the hybrid detector of a large system (summary
    features, radius head): targets are the plain hybrid's own answer metric,
    so with the radius-doubling fallback the learned hybrid returns the same
    decisions."""
    import torch

    dev = torch.device("cuda:0")
    n, qam, K, depth = a.n_tx, a.qam, a.K, a.depth
    snr = tuple(float(x) for x in a.snr.split(","))
    cap = max(a.chunk, a.batch, a.eval_vectors)
    ctx = mdx.Context(0, max_batch=cap, max_n_rx=n, max_n_tx=n)
    mdx.mlp_init(ctx, n, qam, a.batch, seed=a.seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(a.seed)
    p_plain = mdx.make_params(n, n, qam, radius="paper", K=K, depth=depth)
    t0 = time.time()
    Hs, ys, nvs, mets = [], [], [], []
    rng = np.random.default_rng(a.seed)
    for s0 in range(0, a.traces, a.chunk):
        c = min(a.chunk, a.traces - s0)
        H, y, nv, _ = device_workload(torch, gen, c, n, qam, snr[0] + (snr[1] - snr[0]) * rng.random(c), dev)
        sym, met, vst, st = mdx.detect("hybrid", ctx, p_plain, H, y, nv)
        Hs.append(H)
        ys.append(y)
        nvs.append(nv)
        mets.append(met)
    torch.cuda.synchronize()
    H, y, nv, met = torch.cat(Hs), torch.cat(ys), torch.cat(nvs), torch.cat(mets)
    del Hs, ys, nvs, mets
    t_traces = time.time() - t0
    print(f"traces: {a.traces} hybrid answers in {t_traces:.1f} s", flush=True)
    params = mdx.make_params(n, n, qam)
    steps = a.traces // a.batch
    total = steps * a.epochs
    t1 = time.time()
    hist = []
    k = 0
    for ep in range(a.epochs):
        perm = torch.randperm(a.traces, device=dev, generator=gen)
        acc = torch.zeros(2, device=dev)
        for s in range(steps):
            idx = perm[s * a.batch:(s + 1) * a.batch]
            lr = a.lr * 0.5 * (1.0 + math.cos(math.pi * k / total))
            loss, _ = mdx.mlp_train_step(ctx, params, H[idx].contiguous(), y[idx].contiguous(), nv[idx].contiguous(),
                                         None, met[idx].contiguous(), lr=lr)
            acc += loss
            k += 1
        acc = (acc / steps).cpu().numpy()
        hist.append(float(acc[0]))
        print(f"epoch {ep}: pinball {acc[0]:.4f}", flush=True)
    t_train = time.time() - t1
    err = mdx.mlp_error(ctx)
    del H, y, nv, met
    # held-out: the workload generator's vectors, plain vs learned hybrid
    snr_e = snr[0] + (snr[1] - snr[0]) * np.random.default_rng(a.eval_seed).random(a.eval_vectors)
    w = wl.generate(a.eval_seed, a.eval_vectors, n, n, qam, snr_e)
    He, ye, nve = _device_batch(torch, w, dev)
    ev = {}
    for name, f in (("plain", 0), ("learned", mdx.MDX_LEARNED_RADIUS)):
        p = mdx.make_params(n, n, qam, radius="paper", K=K, depth=depth, flags=f)
        res = mdx.detect("hybrid", ctx, p, He, ye, nve)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        res = mdx.detect("hybrid", ctx, p, He, ye, nve, out=res)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        nodes = res[3][:, 0].double().cpu().numpy()
        ev[name] = {"vectors_per_s": a.eval_vectors / (ms / 1e3), "ms": ms, "mean_nodes": float(nodes.mean()),
                    "radius_doubling_rate": float((res[2] == 1).double().mean().item()), "sym": res[0].cpu().numpy()}
    ev["identical_decisions"] = bool((ev["plain"]["sym"] == ev["learned"]["sym"]).all())
    for name in ("plain", "learned"):
        del ev[name]["sym"]
    print(json.dumps(ev), flush=True)
    os.makedirs(a.out, exist_ok=True)
    np.save(model_path(n, qam, a.out), mdx.mlp_get_params(ctx, n, qam))
    meta = {"n_tx": n, "qam": qam, "detector": "hybrid", "K": K, "depth": depth, "traces": a.traces,
            "snr_db": list(snr), "seed": a.seed, "epochs": a.epochs, "batch": a.batch, "lr": a.lr,
            "features": "summary (log diag R, Babai distance, ybar energy, SNR)",
            "trace_generator": "torch device RNG (workload distributions)", "seconds_traces": t_traces,
            "seconds_training": t_train, "loss_history": hist, "kernel_error_word": err,
            "evaluation": {"vectors": a.eval_vectors, "seed": a.eval_seed, **ev}}
    with open(model_path(n, qam, a.out).replace(".npy", ".json"), "w") as f:
        json.dump(meta, f, indent=1)
    ctx.close()


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
    ap.add_argument("--detector", choices=["sd", "hybrid"], default="sd")
    ap.add_argument("--K", type=int, default=32, help="hybrid: K-best survivors")
    ap.add_argument("--depth", type=int, default=4, help="hybrid: SD master depth")
    a = ap.parse_args()
    if a.detector == "hybrid":
        main_hybrid(a)
        return
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
