"""Pins of the FP64 network reference: its backward pass against central
finite differences of its own loss (an independent derivative), and its BF16
rounding against the format's definition."""

import numpy as np

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
