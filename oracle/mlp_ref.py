"""FP64 reference of the learned-radius network (forward, loss, backward).

TEST INFRASTRUCTURE ONLY: used by the tests to check the GPU network's
outputs and gradients; never called by the product path.  The paper has no
learned component; this follows the definition in include/mimo_detect.h:

    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3
    loss = mean_b pinball_0.9(t_b - o_b0)
         + 0.2 * mean_b mean_r CE(softmax(o_b[1 + rP : 1 + (r+1)P]), k_br)

with t = log(d_ML / sigma^2) and k_br the ML PAM index of real row r
(row 2j is Re s_j, index q // P; row 2j+1 is Im s_j, index q % P).
Systems with n_tx > 32 use summary features instead (reduced_features):
log R_ii, the Babai point's distance log(d_B / sigma^2) / 10,
log(||ybar||^2 / (n sigma^2)) / 10 and SNR_dB / 30, and the radius head only
(no cross-entropy term, n = 0 rows in loss_and_grad).
Parity pinned: the backward pass is checked against central finite
differences in tests/test_mlp_ref.py.
"""

from __future__ import annotations

import numpy as np

HIDDEN = 256
TAU = 0.9
LAMBDA = 0.2


def unpack(p, d_in, d_out):
    p = np.asarray(p, dtype=np.float64)
    H = HIDDEN
    o = 0
    W1 = p[o:o + H * d_in].reshape(H, d_in); o += H * d_in
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + d_out * H].reshape(d_out, H); o += d_out * H
    b3 = p[o:o + d_out]; o += d_out
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def forward(p, X, d_in, d_out, round_hidden=None):
    """Outputs [B][d_out] and the cache for backward.  round_hidden, if given,
    is applied to h1 and h2 (to model storage of activations in BF16)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, d_in, d_out)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    if round_hidden is not None:
        h1 = round_hidden(h1)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    if round_hidden is not None:
        h2 = round_hidden(h2)
    o = h2 @ W3.T + b3
    return o, (X, h1, h2)


def targets_to_rows(sym, n, P):
    """[B][n_tx] complex indices -> [B][n] PAM indices of the real rows."""
    sym = np.asarray(sym, dtype=np.int64)
    k = np.empty((sym.shape[0], n), dtype=np.int64)
    k[:, 0::2] = sym // P
    k[:, 1::2] = sym % P
    return k


def loss_and_grad(p, X, t, krow, d_in, d_out, n, P, round_hidden=None):
    """(pinball loss, cross-entropy loss, gradient w.r.t. the parameter vector)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, d_in, d_out)
    o, (X, h1, h2) = forward(p, X, d_in, d_out, round_hidden)
    B = X.shape[0]
    e = t - o[:, 0]
    lp = np.mean(np.where(e >= 0.0, TAU * e, (TAU - 1.0) * e))
    do = np.zeros_like(o)
    do[:, 0] = np.where(e > 0.0, -TAU, 1.0 - TAU) / B
    lc = 0.0
    if n > 0:
        lg = o[:, 1:1 + n * P].reshape(B, n, P)
        lg = lg - lg.max(axis=2, keepdims=True)
        pr = np.exp(lg)
        pr /= pr.sum(axis=2, keepdims=True)
        onehot = np.zeros_like(pr)
        np.put_along_axis(onehot, krow[:, :, None], 1.0, axis=2)
        lc = -np.mean(np.sum(onehot * np.log(np.maximum(pr, 1e-300)), axis=2))
        do[:, 1:1 + n * P] = (LAMBDA * (pr - onehot) / (B * n)).reshape(B, n * P)
    dW3 = do.T @ h2
    db3 = do.sum(axis=0)
    dh2 = (do @ W3) * (h2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    dW1 = dh1.T @ X
    db1 = dh1.sum(axis=0)
    return lp, lc, pack(dW1, db1, dW2, db2, dW3, db3)


def bf16(a):
    """Round float64 values to the nearest BF16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def reduced_features(R, ybar, noise_var, qam, d_in):
    """Summary features of one system from its QR (R row-major n x n, ybar):
    [log R_ii (n), log(d_B / sigma^2) / 10, log(||ybar||^2 / (n sigma^2)) / 10,
    SNR_dB / 30], zero-padded to d_in.  d_B is the distance of the Babai
    point: rows from the top, each rounded to the nearest PAM level (clipped)
    given the rows above."""
    R, ybar = np.asarray(R, dtype=np.float64), np.asarray(ybar, dtype=np.float64)
    n = R.shape[0]
    P = int(round(qam ** 0.5))
    alpha = np.sqrt(3.0 / (2.0 * (qam - 1)))
    x = np.zeros(n)
    db = 0.0
    for i in range(n - 1, -1, -1):
        c = ybar[i] - R[i, i + 1:] @ x[i + 1:]
        k = min(max(np.floor(c / (2.0 * alpha * R[i, i]) + 0.5 * (P - 1) + 0.5), 0), P - 1)
        x[i] = (2.0 * k - (P - 1)) * alpha
        db += (c - R[i, i] * x[i]) ** 2
    f = np.zeros(d_in)
    f[:n] = np.log(np.diag(R))
    f[n] = np.log(db / noise_var) / 10.0
    f[n + 1] = np.log(ybar @ ybar / (n * noise_var)) / 10.0
    f[n + 2] = -10.0 * np.log10(noise_var) / 30.0
    return f
