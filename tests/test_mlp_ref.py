"""Pins of the FP64 network reference: its backward pass against central
finite differences of its own loss (an independent derivative), and its BF16
rounding against the format's definition."""

import numpy as np
import pytest

from oracle import mlp_ref


def _small_problem(seed=0, B=6, n=4, P=2, d_in=24, d_out=16):
    rng = np.random.default_rng(seed)
    H = mlp_ref.HIDDEN
    count = H * d_in + H + H * H + H + d_out * H + d_out
    p = rng.standard_normal(count) * 0.05
    X = rng.standard_normal((B, d_in))
    t = rng.standard_normal(B) + 2.0
    k = rng.integers(0, P, size=(B, n))
    return p, X, t, k, d_in, d_out, n, P


def test_gradient_matches_finite_differences():
    p, X, t, k, d_in, d_out, n, P = _small_problem()
    lp, lc, g = mlp_ref.loss_and_grad(p, X, t, k, d_in, d_out, n, P)
    rng = np.random.default_rng(1)
    idx = rng.choice(p.size, size=60, replace=False)
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp1, lc1, _ = mlp_ref.loss_and_grad(q, X, t, k, d_in, d_out, n, P)
        q[i] -= 2 * h
        lp2, lc2, _ = mlp_ref.loss_and_grad(q, X, t, k, d_in, d_out, n, P)
        fd = ((lp1 + mlp_ref.LAMBDA * lc1) - (lp2 + mlp_ref.LAMBDA * lc2)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_pinball_quantile():
    """Minimising the pinball loss over a constant output gives the 0.9
    quantile of the targets."""
    rng = np.random.default_rng(2)
    t = rng.standard_normal(2001)
    grid = np.linspace(-3, 3, 6001)
    loss = [np.mean(np.where(t - c >= 0, mlp_ref.TAU * (t - c), (mlp_ref.TAU - 1) * (t - c))) for c in grid]
    assert abs(grid[int(np.argmin(loss))] - np.quantile(t, 0.9)) < 2e-2


def test_bf16_rounding():
    # exactly representable values are unchanged; 1 + 2^-8 is a tie that rounds to even (1.0);
    # 1 + 3 * 2^-9 rounds up to 1 + 2^-7
    vals = np.array([1.0, -2.5, 0.15625, 1 + 2 ** -8, 1 + 3 * 2 ** -9])
    out = mlp_ref.bf16(vals)
    np.testing.assert_array_equal(out, [1.0, -2.5, 0.15625, 1.0, 1 + 2 ** -7])
    rng = np.random.default_rng(3)
    x = rng.standard_normal(1000)
    assert np.max(np.abs(mlp_ref.bf16(x) - x) / np.abs(x)) <= 2 ** -8


def test_targets_to_rows():
    sym = np.array([[0, 5, 15]])
    k = mlp_ref.targets_to_rows(sym, 6, 4)
    np.testing.assert_array_equal(k, [[0, 0, 1, 1, 3, 3]])


def test_reduced_loss_has_no_ordering_term():
    """With no ordering rows (n = 0) the loss is the pinball term alone and the
    gradient still matches finite differences."""
    p, X, t, k, d_in, d_out, n, P = _small_problem(seed=5, B=5, d_out=8)
    lp, lc, g = mlp_ref.loss_and_grad(p, X, t, np.zeros((5, 0), dtype=np.int64), d_in, d_out, 0, P)
    assert lc == 0.0
    rng = np.random.default_rng(6)
    for i in rng.choice(p.size, size=30, replace=False):
        q = p.copy()
        q[i] += 1e-6
        a = mlp_ref.loss_and_grad(q, X, t, np.zeros((5, 0), dtype=np.int64), d_in, d_out, 0, P)[0]
        q[i] -= 2e-6
        b = mlp_ref.loss_and_grad(q, X, t, np.zeros((5, 0), dtype=np.int64), d_in, d_out, 0, P)[0]
        assert abs((a - b) / 2e-6 - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_reduced_features_babai_term_is_the_k1_kbest_distance():
    """The Babai distance in the summary features equals the distance of the
    oracle's K-best with K = 1 (an independent implementation of the same
    successive rounding)."""
    import oracle
    from paper_2002_09561_gb300 import workload as wl

    for seed in range(5):
        w = wl.generate(60 + seed, 1, 10, 10, 64, 18.0)
        Hr, yr = oracle.real_decompose(w["H"][0], w["y"][0])
        f = oracle.qr(Hr, yr)
        feat = mlp_ref.reduced_features(f["R"], f["ybar"], w["noise_var"][0], 64, 64)
        r = oracle.kbest(f["R"], f["ybar"], 64, 1)
        assert feat[20] == pytest.approx(np.log(r["d1"] / w["noise_var"][0]) / 10.0, rel=1e-12)
        np.testing.assert_allclose(feat[:20], np.log(np.diag(f["R"])), rtol=1e-14)
