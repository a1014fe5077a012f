"""FP64 CPU oracle for batched MIMO tree-search detection (arXiv 2002.09561).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
leg of the benchmark load it; the product path (the CUDA library and its
binding) never does, and it shares no code with the CUDA sources.  The
arithmetic lives in oracle.c (plain C, double precision, each function
citing the passage of the paper it writes out); this module only builds
that library and marshals numpy arrays into it.

Every function here has a pin in tests/test_oracle.py or
tests/test_oracle_gaps.py (brute force, closed forms, library routines, the
paper's printed counts, an independent restatement of the K-best gaps).
Parity unpinned (SNR convention): the noise variance sigma^2 = 10^(-SNR/10)
per complex entry, which the input generator applies and the oracle's paper
radius r^2 = N M sigma^2 reads, is the reading of the paper's radius
formula; the paper's ML error-rate curves match it only in shape (a
constant, unexplained 5.5 dB offset), so the convention itself is not
pinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALGO = {"sd": 0, "kbest": 1, "hybrid": 2, "ml": 3, "sd_complex": 4, "kbest_complex": 5}
ORDER = {"se": 0, "natural": 1, "reversed": 2, "random": 3}
V_OK, V_EMPTY_RETRIED, V_BUDGET_EXCEEDED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, -O2)."""
    stale = (not os.path.exists(_SO)) or any(
        os.path.getmtime(p) > os.path.getmtime(_SO) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            d, i, ll, vp = ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
            L.orc_pam_levels.argtypes = [i, vp]
            L.orc_pam_levels.restype = i
            L.orc_real_decompose.argtypes = [i, i, vp, vp, vp, vp]
            L.orc_qr.argtypes = [i, i, vp, vp, vp, vp, vp]
            L.orc_qr.restype = i
            L.orc_metric.argtypes = [i, vp, vp, vp, vp]
            L.orc_metric.restype = d
            L.orc_ml_bruteforce.argtypes = [i, i, i, vp, vp, vp, vp, vp]
            L.orc_sd.argtypes = [i, i, vp, vp, vp, d, ll, i, ctypes.c_uint64, i, vp, vp, vp, vp]
            L.orc_sd.restype = i
            L.orc_kbest.argtypes = [i, i, vp, vp, vp, i, d, vp, vp, vp, vp]
            L.orc_kbest.restype = i
            L.orc_sd_complex.argtypes = [i, i, vp, vp, vp, d, ll, i, vp, vp, vp, vp]
            L.orc_sd_complex.restype = i
            L.orc_kbest_complex.argtypes = [i, i, vp, vp, vp, i, d, vp, vp, vp, vp]
            L.orc_kbest_complex.restype = i
            L.orc_hybrid.argtypes = [i, i, vp, vp, vp, i, i, d, i, ctypes.c_uint64, vp, vp, vp, vp]
            L.orc_hybrid.restype = i
            L.orc_detect_batch.argtypes = [i, i, i, i, i, vp, vp, vp, d, i, i, ll, i, i, vp, vp, vp,
                                           vp, vp, i]
            L.orc_detect_batch.restype = i
            L.orc_qr_batch.argtypes = [i, i, i, vp, vp, vp, vp, i]
            L.orc_qr_batch.restype = i
            L.orc_count_errors.argtypes = [i, i, i, vp, vp, vp]
            L.orc_max_threads.restype = i
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Stats(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_longlong), ("peds", ctypes.c_longlong),
                ("restarts", ctypes.c_longlong), ("leaves", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def max_threads() -> int:
    return lib().orc_max_threads()


def pam_levels(qam: int) -> np.ndarray:
    out = np.zeros(16)
    P = lib().orc_pam_levels(qam, _p(out))
    if P < 0:
        raise ValueError(qam)
    return out[:P].copy()


def real_decompose(H: np.ndarray, y: np.ndarray):
    """H [N][M][2], y [N][2] -> Hr [2N][2M], yr [2N]."""
    H, y = _f64(H), _f64(y)
    N, M = H.shape[0], H.shape[1]
    Hr = np.zeros((2 * N, 2 * M))
    yr = np.zeros(2 * N)
    lib().orc_real_decompose(N, M, _p(H), _p(y), _p(Hr), _p(yr))
    return Hr, yr


def qr(A: np.ndarray, y: np.ndarray | None = None, want_q: bool = False):
    A = _f64(A)
    m, n = A.shape
    R = np.zeros((n, n))
    yb = np.zeros(n)
    Q = np.zeros((m, n)) if want_q else None
    yv = None if y is None else _f64(y)
    sing = lib().orc_qr(m, n, _p(A), _p(yv), _p(Q), _p(R), _p(yb))
    return {"Q": Q, "R": R, "ybar": yb, "singular": bool(sing)}


def metric(R, ybar, qam, k) -> float:
    R, ybar = _f64(R), _f64(ybar)
    lev = pam_levels(qam)
    k = np.ascontiguousarray(k, dtype=np.int32)
    return lib().orc_metric(R.shape[0], _p(R), _p(ybar), _p(lev), _p(k))


def ml_bruteforce(H, y, qam):
    H, y = _f64(H), _f64(y)
    N, M = H.shape[0], H.shape[1]
    sym = np.zeros(M, dtype=np.uint8)
    d1 = np.zeros(1)
    d2 = np.zeros(1)
    lib().orc_ml_bruteforce(N, M, qam, _p(H), _p(y), _p(sym), _p(d1), _p(d2))
    return {"sym": sym, "d1": d1[0], "d2": d2[0]}


def sd(R, ybar, qam, r2=np.inf, budget=0, order="se", seed=0, two_best=False):
    R, ybar = _f64(R), _f64(ybar)
    n = R.shape[0]
    lev = pam_levels(qam)
    k = np.zeros(n, dtype=np.int32)
    d1 = np.zeros(1)
    d2 = np.zeros(1)
    st = Stats()
    rc = lib().orc_sd(n, len(lev), _p(R), _p(ybar), _p(lev), float(r2), int(budget), ORDER[order],
                      int(seed), int(two_best), _p(k), _p(d1), _p(d2), ctypes.byref(st))
    if rc < 0:
        raise ValueError("bad arguments")
    return {"k": k, "d1": d1[0], "d2": d2[0], "status": rc, **st.as_dict()}


def kbest(R, ybar, qam, K, r2=np.inf):
    R, ybar = _f64(R), _f64(ybar)
    n = R.shape[0]
    lev = pam_levels(qam)
    k = np.zeros(n, dtype=np.int32)
    d1 = np.zeros(1)
    gap = np.zeros(1)
    st = Stats()
    rc = lib().orc_kbest(n, len(lev), _p(R), _p(ybar), _p(lev), int(K), float(r2), _p(k), _p(d1),
                         _p(gap), ctypes.byref(st))
    if rc < 0:
        raise ValueError("bad arguments")
    return {"k": k, "d1": d1[0], "gap": gap[0], "status": rc, **st.as_dict()}


def sd_complex(R, ybar, qam, r2=np.inf, budget=0, two_best=False):
    """Complex-tree SD (orc_sd_complex): one level per complex antenna."""
    R, ybar = _f64(R), _f64(ybar)
    n = R.shape[0]
    lev = pam_levels(qam)
    k = np.zeros(n, dtype=np.int32)
    d1 = np.zeros(1)
    d2 = np.zeros(1)
    st = Stats()
    rc = lib().orc_sd_complex(n, len(lev), _p(R), _p(ybar), _p(lev), float(r2), int(budget), int(two_best), _p(k),
                              _p(d1), _p(d2), ctypes.byref(st))
    if rc < 0:
        raise ValueError("bad arguments")
    return {"k": k, "d1": d1[0], "d2": d2[0], "status": rc, **st.as_dict()}


def kbest_complex(R, ybar, qam, K, r2=np.inf):
    """Complex-tree K-best (orc_kbest_complex)."""
    R, ybar = _f64(R), _f64(ybar)
    n = R.shape[0]
    lev = pam_levels(qam)
    k = np.zeros(n, dtype=np.int32)
    d1 = np.zeros(1)
    gap = np.zeros(1)
    st = Stats()
    rc = lib().orc_kbest_complex(n, len(lev), _p(R), _p(ybar), _p(lev), int(K), float(r2), _p(k), _p(d1),
                                 _p(gap), ctypes.byref(st))
    if rc < 0:
        raise ValueError("bad arguments")
    return {"k": k, "d1": d1[0], "gap": gap[0], "status": rc, **st.as_dict()}


def hybrid(R, ybar, qam, K, depth, r2=np.inf, order="se", seed=0):
    R, ybar = _f64(R), _f64(ybar)
    n = R.shape[0]
    lev = pam_levels(qam)
    k = np.zeros(n, dtype=np.int32)
    d1 = np.zeros(1)
    gap = np.zeros(1)
    st = Stats()
    rc = lib().orc_hybrid(n, len(lev), _p(R), _p(ybar), _p(lev), int(K), int(depth), float(r2),
                          ORDER[order], int(seed), _p(k), _p(d1), _p(gap), ctypes.byref(st))
    if rc < 0:
        raise ValueError("bad arguments")
    return {"k": k, "d1": d1[0], "gap": gap[0], "status": rc, **st.as_dict()}


def detect_batch(algo, H, y, noise_var, qam, radius=np.inf, K=16, depth=4, budget=0, order="se",
                 want_gap=False, nthreads=0):
    """Detect a batch; radius: float (inf = none) or 'paper' for r^2 = N M sigma^2."""
    H, y, nv = _f64(H), _f64(y), _f64(noise_var)
    B, N, M = H.shape[0], H.shape[1], H.shape[2]
    r = -1.0 if isinstance(radius, str) else float(radius)
    sym = np.zeros((B, M), dtype=np.uint8)
    met = np.zeros(B)
    status = np.zeros(B, dtype=np.int32)
    stats = np.zeros((B, 4), dtype=np.int64)
    gap = np.zeros(B)
    rc = lib().orc_detect_batch(ALGO[algo], B, N, M, int(qam), _p(H), _p(y), _p(nv), r, int(K),
                                int(depth), int(budget), ORDER[order], int(want_gap), _p(sym),
                                _p(met), _p(status), _p(stats), _p(gap), int(nthreads))
    if rc < 0:
        raise ValueError("bad arguments")
    return {"sym": sym, "metric": met, "status": status, "stats": stats, "gap": gap}


def qr_batch(H, y, nthreads=0):
    H, y = _f64(H), _f64(y)
    B, N, M = H.shape[0], H.shape[1], H.shape[2]
    n = 2 * M
    R = np.zeros((B, n, n))
    yb = np.zeros((B, n))
    lib().orc_qr_batch(B, N, M, _p(H), _p(y), _p(R), _p(yb), int(nthreads))
    return R, yb


def count_errors(sym_hat, sym_true, qam):
    a = np.ascontiguousarray(sym_hat, dtype=np.uint8)
    b = np.ascontiguousarray(sym_true, dtype=np.uint8)
    out = np.zeros(2, dtype=np.int64)
    lib().orc_count_errors(a.shape[0], a.shape[1], int(qam), _p(a), _p(b), _p(out))
    return int(out[0]), int(out[1])


def detect_mixed(reqs, H, y, noise_var, want_gap=True, nthreads=0):
    """An uneven batch (request table with the fields of mdx_request: n_rx,
    n_tx, qam, algo (0 = exact SD, 1 = K-best, 2 = complex-tree SD, 3 = natural-order SD), K, init_radius_sq (negative =
    the paper's N M sigma^2), node_budget and the offsets of each request's H,
    y and symbols in the flat arrays) detected request by request with
    detect_batch, grouping requests of equal parameters.  Returns flat symbols
    and per-request metric, status, gap and stats (nodes, evaluations,
    restarts, leaves, as detect_batch)."""
    H, y, nv = _f64(H).ravel(), _f64(y).ravel(), _f64(noise_var).ravel()
    nreq = len(reqs)
    nsym = int(max((int(r["sym_offset"]) + int(r["n_tx"]) for r in reqs), default=0))
    sym = np.zeros(nsym, dtype=np.uint8)
    met, gap = np.zeros(nreq), np.ones(nreq)
    status = np.zeros(nreq, dtype=np.int32)
    stats = np.zeros((nreq, 4), dtype=np.int64)
    groups = {}
    for i, r in enumerate(reqs):
        key = (int(r["n_rx"]), int(r["n_tx"]), int(r["qam"]), int(r["algo"]),
               int(r["K"]) if int(r["algo"]) == 1 else 0, float(r["init_radius_sq"]),
               int(r["node_budget"]) if int(r["algo"]) != 1 else 0)
        groups.setdefault(key, []).append(i)
    for (N, M, qam, algo, K, r0, budget), idx in groups.items():
        Hb = np.stack([H[int(reqs[i]["h_offset"]):int(reqs[i]["h_offset"]) + 2 * N * M] for i in idx])
        yb = np.stack([y[int(reqs[i]["y_offset"]):int(reqs[i]["y_offset"]) + 2 * N] for i in idx])
        radius = "paper" if r0 < 0 else r0
        name = {0: "sd", 1: "kbest", 2: "sd_complex", 3: "sd"}[algo]
        out = detect_batch(name, Hb.reshape(len(idx), N, M, 2), yb.reshape(len(idx), N, 2),
                           nv[idx], qam, radius=radius, K=max(K, 1), budget=budget,
                           order="natural" if algo == 3 else "se", want_gap=want_gap and algo != 1,
                           nthreads=nthreads)
        for j, i in enumerate(idx):
            s0 = int(reqs[i]["sym_offset"])
            sym[s0:s0 + M] = out["sym"][j]
        met[idx] = out["metric"]
        status[idx] = out["status"]
        gap[idx] = out["gap"]
        stats[idx] = out["stats"]
    return {"sym": sym, "metric": met, "status": status, "gap": gap, "stats": stats}


def _slice(x, qam):
    """Nearest PAM index of each real component (clipped to the grid) and the
    relative distance of each component to its decision boundary."""
    P = int(round(qam ** 0.5))
    alpha = np.sqrt(3.0 / (2.0 * (qam - 1)))
    u = (x / alpha + (P - 1)) / 2.0
    k = np.clip(np.floor(u + 0.5), 0, P - 1).astype(np.int64)
    frac = np.abs(u - np.floor(u) - 0.5)  # 0 at a boundary between two levels
    inside = (u > 0.0) & (u < P - 1)
    margin = np.where(inside, frac, 1.0)
    return k, margin


def detect_linear(kind, H, y, noise_var, qam):
    """Linear detection of a batch (the controls of Sec. III-A): ZF, the
    least-squares solution of the real system, or MMSE,
    (Hr^T Hr + sigma^2 I)^-1 Hr^T yr (unit-energy symbols, sigma^2 per
    complex entry), each component sliced to the nearest PAM level.  Returns
    sym [B][M], metric ||ybar - R x^||^2 (oracle QR), and margin [B], the
    smallest distance of a component to a decision boundary (in half PAM
    steps; near 0 means the slicing is a near-tie)."""
    H, y, nv = _f64(H), _f64(y), _f64(noise_var)
    B, N, M = H.shape[0], H.shape[1], H.shape[2]
    P = int(round(qam ** 0.5))
    lev = pam_levels(qam)
    sym = np.zeros((B, M), dtype=np.uint8)
    met, margin = np.zeros(B), np.zeros(B)
    R, yb = qr_batch(H, y)
    for b in range(B):
        Hr, yr = real_decompose(H[b], y[b])
        if kind == "zf":
            x = np.linalg.lstsq(Hr, yr, rcond=None)[0]
        elif kind == "mmse":
            x = np.linalg.solve(Hr.T @ Hr + nv[b] * np.eye(2 * M), Hr.T @ yr)
        else:
            raise ValueError(kind)
        k, mg = _slice(x, qam)
        sym[b] = k[0::2] * P + k[1::2]
        met[b] = float(np.sum((yb[b] - R[b] @ lev[k]) ** 2))
        margin[b] = mg.min()
    return {"sym": sym, "metric": met, "margin": margin}
