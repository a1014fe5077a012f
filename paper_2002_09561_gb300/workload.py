"""Seeded synthetic MIMO workloads (the system model of Sec. III-A, Eq. 1).

This module only draws inputs: y = H s + n with H i.i.d. CN(0, 1), s uniform
over a unit-energy square QAM alphabet, n ~ CN(0, sigma^2 I) and
sigma^2 = 10^(-SNR/10) per complex receive entry.  It holds none of the
detection arithmetic (no QR, no partial distances, no search) and is the one
piece shared by the CUDA path's tests/benchmarks and the CPU oracle's.

Random numbers come from a counter-based generator so that any slice of a
workload can be regenerated independently and the bytes are identical on
every machine: the i-th 64-bit draw of stream `s` under `seed` is the
SplitMix64 output mix64(base + (i + 1) * 0x9E3779B97F4A7C15) with
base = mix64(seed * 0x9E3779B97F4A7C15 + s) (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014).  Uniforms take the
top 53 bits, normals come from the Box-Muller transform.
"""

from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_H, STREAM_SYM, STREAM_NOISE, STREAM_SNR, STREAM_CLASS = 1, 2, 3, 4, 5


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        b = np.array([np.uint64(seed) * GOLDEN + np.uint64(stream)], dtype=np.uint64)
    return _mix64(b)[0]


def draw_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """64-bit draws start .. start+count-1 of one stream."""
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _base(seed, stream) + idx * GOLDEN
    return _mix64(z)


def draw_uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniforms in (0, 1): ((u >> 11) + 0.5) * 2^-53."""
    u = draw_u64(seed, stream, start, count)
    return ((u >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def draw_normal(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Standard normals; normal j uses uniforms 2*(j//2) and 2*(j//2)+1."""
    first = start - (start % 2)
    pairs = (start + count - first + 1) // 2
    u = draw_uniform(seed, stream, first, 2 * pairs)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    z = np.empty(2 * pairs)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    off = start - first
    return z[off : off + count]


def pam_size(qam: int) -> int:
    p = int(round(qam ** 0.5))
    if p * p != qam or p < 2:
        raise ValueError(f"square QAM expected, got {qam}")
    return p


def qam_symbols(q: np.ndarray, qam: int) -> np.ndarray:
    """Complex unit-energy QAM points of indices q = k_re * P + k_im."""
    p = pam_size(qam)
    alpha = np.sqrt(3.0 / (2.0 * (qam - 1)))
    re = (2.0 * (q // p) - (p - 1)) * alpha
    im = (2.0 * (q % p) - (p - 1)) * alpha
    return re + 1j * im


def noise_var_from_snr(snr_db) -> np.ndarray:
    """Noise variance per complex receive entry for unit-energy symbols."""
    return 10.0 ** (-np.asarray(snr_db, dtype=np.float64) / 10.0)


def generate(seed: int, batch: int, n_rx: int, n_tx: int, qam: int, snr_db, start: int = 0):
    """Vectors start .. start+batch-1 of the workload (seed, n_rx, n_tx, qam).

    snr_db is a scalar or an array of `batch` values.  Returns a dict of
    numpy arrays: H [B][N][M][2], y [B][N][2] (float64, (re, im) pairs),
    noise_var [B] and sym [B][M] (uint8 complex indices).
    """
    B, N, M = int(batch), int(n_rx), int(n_tx)
    if N < M or M < 1:
        raise ValueError("need n_rx >= n_tx >= 1")
    nh = 2 * N * M
    h = draw_normal(seed, STREAM_H, start * nh, B * nh) * np.sqrt(0.5)
    H = h.reshape(B, N, M, 2)
    q = (draw_u64(seed, STREAM_SYM, start * M, B * M) % np.uint64(qam)).astype(np.uint8)
    q = q.reshape(B, M)
    nv = np.broadcast_to(noise_var_from_snr(snr_db), (B,)).astype(np.float64).copy()
    w = draw_normal(seed, STREAM_NOISE, start * 2 * N, B * 2 * N).reshape(B, N, 2)
    w *= np.sqrt(nv / 2.0)[:, None, None]
    Hc = H[..., 0] + 1j * H[..., 1]
    s = qam_symbols(q.astype(np.int64), qam)
    yc = np.einsum("bnm,bm->bn", Hc, s)
    y = np.stack([yc.real, yc.imag], axis=-1) + w
    return {"H": np.ascontiguousarray(H), "y": np.ascontiguousarray(y), "noise_var": nv, "sym": q}


def generate_mixed(seed: int, count: int, antennas=(8, 16, 32, 64, 100), qams=(4, 16, 64),
                   snr_range=(6.0, 30.0), sd_fraction=0.5):
    """Request descriptors of an uneven mix: per request (n, qam, snr_db, algo)
    with n_tx = n_rx = n drawn uniformly from `antennas`, qam from `qams`,
    SNR uniform in snr_range and algo 0 (exact SD) with probability
    sd_fraction, else 1 (K-best)."""
    u = draw_uniform(seed, STREAM_CLASS, 0, 4 * count).reshape(count, 4)
    ant = np.asarray(antennas)[np.minimum((u[:, 0] * len(antennas)).astype(np.int64), len(antennas) - 1)]
    qm = np.asarray(qams)[np.minimum((u[:, 1] * len(qams)).astype(np.int64), len(qams) - 1)]
    snr = snr_range[0] + (snr_range[1] - snr_range[0]) * u[:, 2]
    algo = (u[:, 3] >= sd_fraction).astype(np.int32)
    return {"n": ant.astype(np.int32), "qam": qm.astype(np.int32), "snr_db": snr, "algo": algo}


def generate_mixed_inputs(seed: int, count: int, antennas=(8, 16, 32, 64, 100), qams=(4, 16, 64),
                          snr_range=(6.0, 30.0), sd_fraction=0.5):
    """The mix of generate_mixed together with its inputs.  Each (n, qam)
    class is one generate() workload under the seed
    seed * 1000003 + 1000 n + qam, whose rows go to the class's requests in
    table order.  Returns the descriptor arrays of generate_mixed plus
    H and y (float64, the requests' [N][M][2] and [N][2] blocks back to back
    in table order), noise_var, sym (uint8, [n_tx] per request, back to back)
    and the offsets h_offset, y_offset, sym_offset of every request."""
    d = generate_mixed(seed, count, antennas, qams, snr_range, sd_fraction)
    n = d["n"].astype(np.int64)
    hsz, ysz = 2 * n * n, 2 * n
    h_off = np.concatenate([[0], np.cumsum(hsz)[:-1]]).astype(np.int64)
    y_off = np.concatenate([[0], np.cumsum(ysz)[:-1]]).astype(np.int64)
    s_off = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    H = np.empty(int(hsz.sum()))
    y = np.empty(int(ysz.sum()))
    sym = np.empty(int(n.sum()), dtype=np.uint8)
    for a in np.unique(n):
        for q in np.unique(d["qam"]):
            idx = np.flatnonzero((n == a) & (d["qam"] == q))
            if idx.size == 0:
                continue
            w = generate(int(seed) * 1000003 + 1000 * int(a) + int(q), idx.size, int(a), int(a), int(q),
                         d["snr_db"][idx])
            Hw, yw = w["H"].reshape(idx.size, -1), w["y"].reshape(idx.size, -1)
            for j, r in enumerate(idx):
                H[h_off[r]:h_off[r] + hsz[r]] = Hw[j]
                y[y_off[r]:y_off[r] + ysz[r]] = yw[j]
                sym[s_off[r]:s_off[r] + a] = w["sym"][j]
    d.update({"H": H, "y": y, "noise_var": noise_var_from_snr(d["snr_db"]), "sym": sym, "h_offset": h_off,
              "y_offset": y_off, "sym_offset": s_off})
    return d
