"""The learned-radius network on the GPU (tensor-core forward/backward)
against the FP64 reference, and its effect on the exact sphere decoder."""

import math

import numpy as np
import pytest

import oracle
from oracle import mlp_ref
from paper_2002_09561_gb300 import workload as wl

pytestmark = pytest.mark.gpu

N_TX, QAM, P = 16, 16, 4


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2002_09561_gb300 import mdx

    ctx = mdx.Context(0, max_batch=32768, max_n_rx=N_TX, max_n_tx=N_TX)
    mdx.mlp_init(ctx, N_TX, QAM, max_train_batch=4096, seed=7)
    yield torch, mdx, ctx
    ctx.close()


def _dev(torch, w):
    return [torch.from_numpy(w[k]).cuda() for k in ("H", "y", "noise_var")]


def _reference_inputs(mdx, ctx, feat):
    d_in, d_out = mdx.mlp_dims(N_TX, QAM)
    p = mdx.mlp_get_params(ctx, N_TX, QAM).astype(np.float64)
    W1, b1, W2, b2, W3, b3 = mlp_ref.unpack(p, d_in, d_out)
    pr = mlp_ref.pack(mlp_ref.bf16(W1), b1, mlp_ref.bf16(W2), b2, mlp_ref.bf16(W3), b3)
    return pr, mlp_ref.bf16(feat), d_in, d_out


def test_forward_matches_reference(env):
    torch, mdx, ctx = env
    w = wl.generate(11, 512, N_TX, N_TX, QAM, 12.0)
    H, y, nv = _dev(torch, w)
    params = mdx.make_params(N_TX, N_TX, QAM)
    out, feat = mdx.mlp_predict(ctx, params, H, y, nv, want_features=True)
    torch.cuda.synchronize()
    assert mdx.mlp_error(ctx) == 0
    pr, X, d_in, d_out = _reference_inputs(mdx, ctx, feat.cpu().numpy().astype(np.float64))
    ref, _ = mlp_ref.forward(pr, X, d_in, d_out, round_hidden=mlp_ref.bf16)
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    assert err.max() <= 1e-2 * np.abs(ref).max() + 1e-3, err.max()
    # features: the QR's R (column-packed), ybar and SNR/30 of the oracle's QR
    Ro, ybo = oracle.qr_batch(w["H"][:4], w["y"][:4])
    n = 2 * N_TX
    f = feat.cpu().numpy()
    for b in range(4):
        colpacked = np.concatenate([Ro[b][: c + 1, c] for c in range(n)])
        np.testing.assert_allclose(f[b, : n * (n + 1) // 2], colpacked, atol=1e-5 * np.abs(colpacked).max())
        np.testing.assert_allclose(f[b, n * (n + 1) // 2: n * (n + 1) // 2 + n], ybo[b], atol=1e-5 * np.abs(ybo).max())
        assert f[b, n * (n + 1) // 2 + n] == pytest.approx(12.0 / 30.0, rel=1e-5)


def _targets(torch, mdx, ctx, H, y, nv):
    p = mdx.make_params(N_TX, N_TX, QAM, radius="paper")
    sym, met, vst, _ = mdx.detect("sd", ctx, p, H, y, nv)
    torch.cuda.synchronize()
    return sym, met


def test_gradient_matches_reference(env):
    torch, mdx, ctx = env
    B = 1024
    w = wl.generate(12, B, N_TX, N_TX, QAM, 14.0)
    H, y, nv = _dev(torch, w)
    sym, met = _targets(torch, mdx, ctx, H, y, nv)
    params = mdx.make_params(N_TX, N_TX, QAM)
    _, feat = mdx.mlp_predict(ctx, params, H, y, nv, want_features=True)
    loss, grad = mdx.mlp_train_step(ctx, params, H, y, nv, sym, met, update=False, want_grad=True)
    torch.cuda.synchronize()
    assert mdx.mlp_error(ctx) == 0
    pr, X, d_in, d_out = _reference_inputs(mdx, ctx, feat.cpu().numpy().astype(np.float64))
    t = np.log(met.cpu().numpy() / w["noise_var"])
    krow = mlp_ref.targets_to_rows(sym.cpu().numpy(), 2 * N_TX, P)
    lp, lc, gref = mlp_ref.loss_and_grad(pr, X, t, krow, d_in, d_out, 2 * N_TX, P, round_hidden=mlp_ref.bf16)
    g = grad.cpu().numpy().astype(np.float64)
    cos = g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref))
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    print(f"GRADCHECK cosine {cos:.6f} rel-L2 {rel:.4e}")
    assert cos > 0.999 and rel < 2e-2
    lg = loss.cpu().numpy()
    assert lg[0] == pytest.approx(lp, rel=2e-2)
    assert lg[1] == pytest.approx(lc, rel=2e-2)


def test_learned_radius_keeps_the_ml_point(env):
    torch, mdx, ctx = env
    w = wl.generate(13, 2000, N_TX, N_TX, QAM, 12.0)
    H, y, nv = _dev(torch, w)
    plain = mdx.detect("sd", ctx, mdx.make_params(N_TX, N_TX, QAM, radius="paper"), H, y, nv)
    learned = mdx.detect("sd", ctx, mdx.make_params(N_TX, N_TX, QAM, radius="paper", flags=mdx.MDX_LEARNED_RADIUS),
                         H, y, nv)
    torch.cuda.synchronize()
    assert torch.equal(plain[0], learned[0])
    rel = ((plain[1] - learned[1]).abs() / plain[1]).max().item()
    assert rel < 1e-12


def test_learned_order_keeps_the_ml_point(env):
    """The top-ranked leaf of the ordering head caps the radius; with or
    without the learned radius, and from no radius at all, the decisions and
    metrics are those of the plain search."""
    torch, mdx, ctx = env
    w = wl.generate(14, 2000, N_TX, N_TX, QAM, 10.0)
    H, y, nv = _dev(torch, w)
    plain = mdx.detect("sd", ctx, mdx.make_params(N_TX, N_TX, QAM, radius="paper"), H, y, nv)
    for radius, f in (("paper", mdx.MDX_LEARNED_ORDER), ("paper", mdx.MDX_LEARNED_ORDER | mdx.MDX_LEARNED_RADIUS),
                      (math.inf, mdx.MDX_LEARNED_ORDER)):
        got = mdx.detect("sd", ctx, mdx.make_params(N_TX, N_TX, QAM, radius=radius, flags=f), H, y, nv)
        torch.cuda.synchronize()
        assert torch.equal(plain[0], got[0]), (radius, f)
        assert ((plain[1] - got[1]).abs() / plain[1]).max().item() < 1e-12
        # the capped radius always contains the ML point: no radius doubling from no radius
        if radius == math.inf:
            assert (got[2] != 1).all()


def test_learned_order_needs_a_matching_model(env):
    torch, mdx, ctx = env
    w = wl.generate(15, 8, 8, 8, QAM, 10.0)
    H, y, nv = _dev(torch, w)
    with pytest.raises(mdx.MdxError):
        mdx.detect("sd", ctx, mdx.make_params(8, 8, QAM, radius="paper", flags=mdx.MDX_LEARNED_ORDER), H, y, nv)
    w = wl.generate(15, 8, N_TX, N_TX, QAM, 10.0)
    H, y, nv = _dev(torch, w)
    with pytest.raises(mdx.MdxError):
        mdx.detect("kbest", ctx, mdx.make_params(N_TX, N_TX, QAM, K=16, flags=mdx.MDX_LEARNED_ORDER), H, y, nv)


def test_training_reduces_nodes(env):
    """A short training on exact-SD traces (SNR uniform in 8..20 dB): the loss
    falls, and on held-out vectors the learned radius visits fewer nodes than
    the paper's radius with identical decisions."""
    torch, mdx, ctx = env
    rng = np.random.default_rng(0)
    B, steps_per_epoch, epochs = 2048, 12, 8
    Ntr = B * steps_per_epoch
    snr = 8.0 + 12.0 * rng.random(Ntr)
    w = wl.generate(100, Ntr, N_TX, N_TX, QAM, snr)
    H, y, nv = _dev(torch, w)
    sym, met = _targets(torch, mdx, ctx, H, y, nv)
    params = mdx.make_params(N_TX, N_TX, QAM)
    first = last = None
    for ep in range(epochs):
        tot = 0.0
        for s in range(steps_per_epoch):
            sl = slice(s * B, (s + 1) * B)
            loss, _ = mdx.mlp_train_step(ctx, params, H[sl], y[sl], nv[sl], sym[sl], met[sl], lr=2e-3)
            tot += float(loss[0]) + 0.2 * float(loss[1])
        tot /= steps_per_epoch
        first = tot if first is None else first
        last = tot
    assert mdx.mlp_error(ctx) == 0
    print(f"TRAIN loss {first:.4f} -> {last:.4f}")
    assert last < 0.8 * first
    wt = wl.generate(200, 8000, N_TX, N_TX, QAM, 12.0)
    Ht, yt, nvt = _dev(torch, wt)
    seq = mdx.MDX_SEQUENTIAL_SEARCH
    plain = mdx.detect("sd", ctx, mdx.make_params(N_TX, N_TX, QAM, radius="paper", flags=seq), Ht, yt, nvt)
    learned = mdx.detect("sd", ctx, mdx.make_params(N_TX, N_TX, QAM, radius="paper",
                                                    flags=seq | mdx.MDX_LEARNED_RADIUS), Ht, yt, nvt)
    torch.cuda.synchronize()
    assert torch.equal(plain[0], learned[0])
    both = mdx.detect("sd", ctx, mdx.make_params(N_TX, N_TX, QAM, radius="paper",
                                                 flags=seq | mdx.MDX_LEARNED_RADIUS | mdx.MDX_LEARNED_ORDER),
                      Ht, yt, nvt)
    torch.cuda.synchronize()
    assert torch.equal(plain[0], both[0])
    n_plain = plain[3][:, 0].double().sum().item()
    n_learned = learned[3][:, 0].double().sum().item()
    n_both = both[3][:, 0].double().sum().item()
    fallback = (learned[2] == 1).double().mean().item()
    print(f"GAIN nodes plain {n_plain:.0f} learned {n_learned:.0f} ratio {n_learned / n_plain:.3f} "
          f"fallback {fallback:.3f}; learned radius + order {n_both:.0f}")
    assert n_learned < n_plain
    assert n_both <= n_learned * 1.02


# ----------------------------------------------------------- summary-feature models (n_tx > 32)


@pytest.fixture(scope="module")
def big_env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2002_09561_gb300 import mdx

    ctx = mdx.Context(0, max_batch=2048, max_n_rx=100, max_n_tx=100)
    yield torch, mdx, ctx
    ctx.close()


def test_summary_features_match_reference(big_env):
    torch, mdx, ctx = big_env
    n_tx, qam = 40, 16
    mdx.mlp_init(ctx, n_tx, qam, max_train_batch=256, seed=3)
    w = wl.generate(21, 64, n_tx, n_tx, qam, 14.0)
    H, y, nv = _dev(torch, w)
    params = mdx.make_params(n_tx, n_tx, qam)
    out, feat = mdx.mlp_predict(ctx, params, H, y, nv, want_features=True)
    torch.cuda.synchronize()
    d_in, d_out = mdx.mlp_dims(n_tx, qam)
    assert (d_in, d_out) == (128, 128)
    Ro, ybo = oracle.qr_batch(w["H"], w["y"])
    f = feat.cpu().numpy()
    bad = 0
    for b in range(64):
        ref = mlp_ref.reduced_features(Ro[b], ybo[b], w["noise_var"][b], qam, d_in)
        np.testing.assert_allclose(f[b, :2 * n_tx], ref[:2 * n_tx], atol=1e-5)
        np.testing.assert_allclose(f[b, 2 * n_tx + 1:], ref[2 * n_tx + 1:], atol=1e-5)
        # the Babai distance: FP32 rounding may flip a decision on a near-tie
        bad += abs(f[b, 2 * n_tx] - ref[2 * n_tx]) > 1e-4
    assert bad <= 2


def test_summary_model_gradient_matches_reference(big_env):
    torch, mdx, ctx = big_env
    n_tx, qam, B = 40, 16, 512
    mdx.mlp_init(ctx, n_tx, qam, max_train_batch=B, seed=4)
    w = wl.generate(22, B, n_tx, n_tx, qam, 16.0)
    H, y, nv = _dev(torch, w)
    met = torch.from_numpy(w["noise_var"] * (2 * n_tx) * (1.0 + np.random.default_rng(1).random(B))).cuda()
    params = mdx.make_params(n_tx, n_tx, qam)
    _, feat = mdx.mlp_predict(ctx, params, H, y, nv, want_features=True)
    loss, grad = mdx.mlp_train_step(ctx, params, H, y, nv, None, met, update=False, want_grad=True)
    torch.cuda.synchronize()
    assert mdx.mlp_error(ctx) == 0
    d_in, d_out = mdx.mlp_dims(n_tx, qam)
    p = mdx.mlp_get_params(ctx, n_tx, qam).astype(np.float64)
    W1, b1, W2, b2, W3, b3 = mlp_ref.unpack(p, d_in, d_out)
    pr = mlp_ref.pack(mlp_ref.bf16(W1), b1, mlp_ref.bf16(W2), b2, mlp_ref.bf16(W3), b3)
    X = mlp_ref.bf16(feat.cpu().numpy().astype(np.float64))
    t = np.log(met.cpu().numpy() / w["noise_var"])
    lp, lc, gref = mlp_ref.loss_and_grad(pr, X, t, np.zeros((B, 0), dtype=np.int64), d_in, d_out, 0, 4,
                                         round_hidden=mlp_ref.bf16)
    g = grad.cpu().numpy().astype(np.float64)
    cos = g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref))
    print(f"GRADCHECK summary model: cosine {cos:.6f}")
    assert cos > 0.999 and lc == 0.0
    assert float(loss[0]) == pytest.approx(lp, rel=2e-2)


def test_learned_hybrid_keeps_the_answer(big_env):
    """The trained 100x100 64-QAM model: the hybrid from the learned radius
    (doubled on an empty sphere) returns the plain hybrid's decisions and
    visits fewer nodes."""
    torch, mdx, ctx = big_env
    from paper_2002_09561_gb300 import train

    meta = train.load_model(ctx, 100, 64)
    assert meta.get("detector") == "hybrid"
    w = wl.generate(23, 300, 100, 100, 64, 24.0)
    H, y, nv = _dev(torch, w)
    plain = mdx.detect("hybrid", ctx, mdx.make_params(100, 100, 64, radius="paper", K=32, depth=4), H, y, nv)
    learned = mdx.detect("hybrid", ctx, mdx.make_params(100, 100, 64, radius="paper", K=32, depth=4,
                                                        flags=mdx.MDX_LEARNED_RADIUS), H, y, nv)
    torch.cuda.synchronize()
    assert torch.equal(plain[0], learned[0])
    npl, nle = plain[3][:, 0].double().sum().item(), learned[3][:, 0].double().sum().item()
    print(f"HYBRID learned radius: nodes {npl:.0f} -> {nle:.0f}")
    assert nle < npl
    with pytest.raises(mdx.MdxError):  # no ordering head in a summary model
        mdx.detect("sd", ctx, mdx.make_params(100, 100, 64, radius="paper", budget=100,
                                             flags=mdx.MDX_LEARNED_ORDER), H, y, nv)
