"""Thin Python binding of libmdx (include/mimo_detect.h).

Argument marshalling only: every step of detection runs in the CUDA library.
The raw entry points take integer addresses; the helpers below take torch
CUDA tensors (torch is used for device memory and streams) or numpy arrays in
pinned host memory (MDX_HOST_BUFFERS).  There is no CPU fallback: if the
library is missing or no GPU is present, every call raises.
"""

from __future__ import annotations

import ctypes
import math
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdx.so")

MDX_OK, MDX_EINVAL, MDX_EUNSUPPORTED, MDX_ENOMEM, MDX_ECUDA = 0, -1, -2, -3, -4
MDX_V_OK, MDX_V_EMPTY_RETRIED, MDX_V_BUDGET_EXCEEDED, MDX_V_SINGULAR = 0, 1, 2, 3
MDX_HOST_BUFFERS, MDX_NO_RESCORE, MDX_LEARNED_RADIUS, MDX_SEQUENTIAL_SEARCH = 1, 2, 4, 8
MDX_LEARNED_ORDER = 1 << 5
MDX_COMPLEX_TREE = 1 << 6
MDX_ORDER_NATURAL = 1 << 7
MDX_LINEAR_MMSE = 1 << 8
MDX_MAX_TX, MDX_MAX_RX, MDX_MAX_K = 100, 128, 256
MDX_ALGO_SD, MDX_ALGO_KBEST, MDX_ALGO_SD_COMPLEX, MDX_ALGO_SD_NATURAL = 0, 1, 2, 3
MDX_GRAPH = 1 << 4

# Every symbol the header declares; the library must export all of them.
EXPORTS = ["mdx_create", "mdx_destroy", "mdx_strerror", "mdx_last_error", "mdx_workspace_bytes",
           "mdx_qr", "detect_sd", "detect_kbest", "detect_hybrid", "mdx_count_errors",
           "mdx_profile", "mdx_profile_read", "detect_kbest_noalloc", "mdx_mlp_param_count",
           "mdx_mlp_dims", "mdx_mlp_init", "mdx_mlp_set_params", "mdx_mlp_get_params", "mdx_mlp_predict",
           "mdx_mlp_train_step", "mdx_mlp_error", "detect_mixed", "mdx_autotune_mixed", "detect_linear",
           "mdx_measure_peaks"]
NOALLOC_SCRATCH_BYTES = 16 << 20
STATS = 5  # per-vector stats: nodes, peds, restarts, rescored, algorithmic FP32 flops


class MdxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n_rx", ctypes.c_int), ("n_tx", ctypes.c_int), ("qam", ctypes.c_int),
                ("init_radius_sq", ctypes.c_double), ("K", ctypes.c_int),
                ("hybrid_depth", ctypes.c_int), ("node_budget", ctypes.c_longlong),
                ("flags", ctypes.c_int)]


def make_params(n_rx, n_tx, qam, radius=math.inf, K=16, depth=4, budget=0, flags=0) -> Params:
    """radius: float r^2 (inf = none) or 'paper' for r^2 = N M sigma^2."""
    r = -1.0 if isinstance(radius, str) else float(radius)
    return Params(int(n_rx), int(n_tx), int(qam), r, int(K), int(depth), int(budget), int(flags))


# mdx_request as a numpy structured type (64 bytes, the C layout)
def request_dtype():
    import numpy as np

    return np.dtype([("n_rx", "<i4"), ("n_tx", "<i4"), ("qam", "<i4"), ("algo", "<i4"), ("K", "<i4"),
                     ("pad", "<i4"), ("init_radius_sq", "<f8"), ("node_budget", "<i8"), ("h_offset", "<i8"),
                     ("y_offset", "<i8"), ("sym_offset", "<i8")])


_lock = threading.Lock()
_lib = None


def lib():
    """Load libmdx.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise MdxError(MDX_ECUDA, f"{LIB_PATH} is missing: run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, i, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
            L.mdx_create.argtypes = [ctypes.POINTER(vp), i, i, i, i]
            L.mdx_create.restype = i
            L.mdx_destroy.argtypes = [vp]
            L.mdx_destroy.restype = i
            L.mdx_strerror.argtypes = [i]
            L.mdx_strerror.restype = ctypes.c_char_p
            L.mdx_last_error.argtypes = [vp]
            L.mdx_last_error.restype = ctypes.c_char_p
            L.mdx_workspace_bytes.argtypes = [vp]
            L.mdx_workspace_bytes.restype = ctypes.c_size_t
            L.mdx_qr.argtypes = [vp, i, i, i, vp, vp, vp, vp, i, vp]
            L.mdx_qr.restype = i
            for name in ("detect_sd", "detect_kbest", "detect_hybrid", "detect_linear"):
                f = getattr(L, name)
                f.argtypes = [vp, ctypes.POINTER(Params), i, vp, vp, vp, vp, vp, vp, vp, vp]
                f.restype = i
            L.mdx_count_errors.argtypes = [vp, i, i, i, vp, vp, vp, i, vp]
            L.mdx_count_errors.restype = i
            L.detect_kbest_noalloc.argtypes = [ctypes.POINTER(Params), i, vp, vp, vp, vp, vp, vp, vp, vp]
            L.detect_kbest_noalloc.restype = i
            L.mdx_mlp_param_count.argtypes = [i, i]
            L.mdx_mlp_param_count.restype = ctypes.c_size_t
            L.mdx_mlp_dims.argtypes = [i, i, vp, vp]
            L.mdx_mlp_dims.restype = i
            L.mdx_mlp_init.argtypes = [vp, i, i, i, ctypes.c_ulonglong]
            L.mdx_mlp_init.restype = i
            L.mdx_mlp_set_params.argtypes = [vp, vp, ctypes.c_size_t]
            L.mdx_mlp_set_params.restype = i
            L.mdx_mlp_get_params.argtypes = [vp, vp, ctypes.c_size_t]
            L.mdx_mlp_get_params.restype = i
            L.mdx_mlp_predict.argtypes = [vp, ctypes.POINTER(Params), i, vp, vp, vp, vp, vp, vp]
            L.mdx_mlp_predict.restype = i
            L.mdx_mlp_train_step.argtypes = [vp, ctypes.POINTER(Params), i, vp, vp, vp, vp, vp, ctypes.c_float, i,
                                             vp, vp, vp]
            L.mdx_mlp_train_step.restype = i
            L.mdx_mlp_error.argtypes = [vp, vp]
            L.mdx_mlp_error.restype = i
            L.detect_mixed.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp, vp, i, vp]
            L.detect_mixed.restype = i
            L.mdx_autotune_mixed.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.mdx_autotune_mixed.restype = i
            L.mdx_profile.argtypes = [vp, i]
            L.mdx_profile.restype = i
            L.mdx_profile_read.argtypes = [vp, vp]
            L.mdx_profile_read.restype = i
            L.mdx_measure_peaks.argtypes = [i, vp, vp]
            L.mdx_measure_peaks.restype = i
            _lib = L
    return _lib


class Context:
    """Owns an mdx_ctx (device workspace for up to max_batch vectors)."""

    def __init__(self, device: int = 0, max_batch: int = 1024, max_n_rx: int = 16, max_n_tx: int = 16):
        self._h = ctypes.c_void_p()
        st = lib().mdx_create(ctypes.byref(self._h), device, max_batch, max_n_rx, max_n_tx)
        if st != MDX_OK:
            raise MdxError(st, f"mdx_create: {lib().mdx_strerror(st).decode()}")
        self.device, self.max_batch, self.max_n_rx, self.max_n_tx = device, max_batch, max_n_rx, max_n_tx

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        return int(lib().mdx_workspace_bytes(self._h))

    def check(self, st: int, what: str):
        if st != MDX_OK:
            msg = lib().mdx_last_error(self._h).decode(errors="replace")
            raise MdxError(st, f"{what}: {lib().mdx_strerror(st).decode()}: {msg}")

    def profile(self, enable: bool = True):
        """Record CUDA events around the QR and search kernels of each call."""
        self.check(lib().mdx_profile(self._h, int(enable)), "mdx_profile")

    def profile_read(self):
        """(QR ms, search ms, calls) summed since the last read; the error word
        of the last sphere-decoder launch is kept in self.last_sd_error."""
        import numpy as np

        out = np.zeros(8)
        self.check(lib().mdx_profile_read(self._h, ctypes.c_void_p(out.ctypes.data)), "mdx_profile_read")
        self.last_sd_error = int(out[3])
        self.last_sd_split = {"checks": int(out[4]), "splits": int(out[5]), "donated": int(out[6]),
                              "no_level": int(out[7])}
        return float(out[0]), float(out[1]), int(out[2])

    def close(self):
        if self._h:
            lib().mdx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _call_detect(name, ctx, params, batch, H, y, noise_var, sym, metric, vstatus, stats, stream):
    f = getattr(lib(), name)
    st = f(ctx.handle, ctypes.byref(params), int(batch), _ptr(H), _ptr(y), _ptr(noise_var), _ptr(sym),
           _ptr(metric), _ptr(vstatus), _ptr(stats), _stream(stream))
    ctx.check(st, name)


def _outputs(batch, n_tx, device, want_stats):
    import torch

    sym = torch.empty((batch, n_tx), dtype=torch.uint8, device=device)
    met = torch.empty(batch, dtype=torch.float64, device=device)
    vst = torch.empty(batch, dtype=torch.int32, device=device)
    stats = torch.empty((batch, STATS), dtype=torch.int64, device=device) if want_stats else None
    return sym, met, vst, stats


def detect(algo: str, ctx: Context, params: Params, H, y, noise_var, stream=None, want_stats=True,
           out=None):
    """Run detect_<algo> on torch CUDA tensors H [B][N][M][2], y [B][N][2],
    noise_var [B] (float64).  Returns (sym, metric, vstatus, stats) tensors."""
    B = int(H.shape[0])
    if out is None:
        out = _outputs(B, params.n_tx, H.device, want_stats)
    sym, met, vst, stats = out
    _call_detect(f"detect_{algo}", ctx, params, B, H, y, noise_var, sym, met, vst, stats, stream)
    return sym, met, vst, stats


def detect_sd(ctx, params, H, y, noise_var, **kw):
    return detect("sd", ctx, params, H, y, noise_var, **kw)


def detect_kbest(ctx, params, H, y, noise_var, **kw):
    return detect("kbest", ctx, params, H, y, noise_var, **kw)


def detect_hybrid(ctx, params, H, y, noise_var, **kw):
    return detect("hybrid", ctx, params, H, y, noise_var, **kw)


def detect_host(algo: str, ctx: Context, params: Params, H, y, noise_var, sym, metric, vstatus,
                stats=None, stream=None):
    """detect_<algo> on numpy host arrays (outputs preallocated); the library
    stages them through its device buffers (MDX_HOST_BUFFERS) and returns
    when the results are in host memory."""
    p = Params(params.n_rx, params.n_tx, params.qam, params.init_radius_sq, params.K,
               params.hybrid_depth, params.node_budget, params.flags | MDX_HOST_BUFFERS)
    _call_detect(f"detect_{algo}", ctx, p, H.shape[0], H, y, noise_var, sym, metric, vstatus, stats,
                 stream)


def qr(ctx: Context, H, y, stream=None):
    """Dense R [B][n][n] and ybar [B][n] (float64 torch tensors) of H, y."""
    import torch

    B, N, M = int(H.shape[0]), int(H.shape[1]), int(H.shape[2])
    R = torch.empty((B, 2 * M, 2 * M), dtype=torch.float64, device=H.device)
    yb = torch.empty((B, 2 * M), dtype=torch.float64, device=H.device)
    st = lib().mdx_qr(ctx.handle, B, N, M, _ptr(H), _ptr(y), _ptr(R), _ptr(yb), 0, _stream(stream))
    ctx.check(st, "mdx_qr")
    return R, yb


def count_errors(ctx: Context, sym_hat, sym_true, qam: int, stream=None):
    """(bit errors, symbol errors) of uint8 CUDA tensors [B][M] (Gray map)."""
    import torch

    out = torch.zeros(2, dtype=torch.int64, device=sym_hat.device)
    B, M = int(sym_hat.shape[0]), int(sym_hat.shape[1])
    st = lib().mdx_count_errors(ctx.handle, B, M, int(qam), _ptr(sym_hat), _ptr(sym_true), _ptr(out), 0,
                                _stream(stream))
    ctx.check(st, "mdx_count_errors")
    return out


# ----------------------------------------------------------------------------- uneven batches


def make_requests(n_rx, n_tx, qam, algo, K=64, radius=None, budget=0, h_offset=None, y_offset=None,
                  sym_offset=None):
    """A request table (numpy, request_dtype) from per-request arrays.
    radius: per-request r^2 (inf = none, negative = the paper's N M sigma^2);
    default: the paper's radius for exact SD, none for K-best.  Offsets
    default to the requests packed back to back in table order."""
    import numpy as np

    n_rx = np.asarray(n_rx, dtype=np.int64)
    cnt = n_rx.size
    t = np.zeros(cnt, dtype=request_dtype())
    t["n_rx"] = n_rx
    t["n_tx"] = np.broadcast_to(np.asarray(n_tx), (cnt,))
    t["qam"] = np.broadcast_to(np.asarray(qam), (cnt,))
    t["algo"] = np.broadcast_to(np.asarray(algo), (cnt,))
    t["K"] = np.broadcast_to(np.asarray(K), (cnt,))
    if radius is None:
        radius = np.where(t["algo"] == MDX_ALGO_SD, -1.0, math.inf)
    t["init_radius_sq"] = np.broadcast_to(np.asarray(radius, dtype=np.float64), (cnt,))
    t["node_budget"] = np.broadcast_to(np.asarray(budget), (cnt,))
    hsz = 2 * t["n_rx"].astype(np.int64) * t["n_tx"]
    ysz = 2 * t["n_rx"].astype(np.int64)
    t["h_offset"] = np.concatenate([[0], np.cumsum(hsz)[:-1]]) if h_offset is None else h_offset
    t["y_offset"] = np.concatenate([[0], np.cumsum(ysz)[:-1]]) if y_offset is None else y_offset
    t["sym_offset"] = (np.concatenate([[0], np.cumsum(t["n_tx"].astype(np.int64))[:-1]])
                       if sym_offset is None else sym_offset)
    return t


def _table(reqs):
    import numpy as np

    reqs = np.ascontiguousarray(reqs, dtype=request_dtype())
    return reqs, ctypes.c_void_p(reqs.ctypes.data) if reqs.size else None


def detect_mixed(ctx: Context, reqs, H, y, noise_var, flags=0, stream=None, want_stats=True, out=None):
    """detect_mixed over a request table (see make_requests) and flat float64
    CUDA tensors H, y, noise_var [nreq].  Returns (sym (flat uint8, indexed by
    sym_offset), metric [nreq], vstatus [nreq], stats [nreq][STATS])."""
    import torch

    reqs, tp = _table(reqs)
    nreq = int(reqs.size)
    if out is None:
        nsym = int((reqs["sym_offset"] + reqs["n_tx"]).max()) if nreq else 0
        dev = H.device
        out = (torch.zeros(max(nsym, 1), dtype=torch.uint8, device=dev),
               torch.empty(max(nreq, 1), dtype=torch.float64, device=dev),
               torch.empty(max(nreq, 1), dtype=torch.int32, device=dev),
               torch.empty((max(nreq, 1), STATS), dtype=torch.int64, device=dev) if want_stats else None)
    sym, met, vst, stats = out
    st = lib().detect_mixed(ctx.handle, nreq, tp, _ptr(H), _ptr(y), _ptr(noise_var), _ptr(sym), _ptr(met),
                            _ptr(vst), _ptr(stats), int(flags), _stream(stream))
    ctx.check(st, "detect_mixed")
    return sym, met, vst, stats


def detect_mixed_host(ctx: Context, reqs, H, y, noise_var, sym, metric, vstatus, stats=None, flags=0,
                      stream=None):
    """detect_mixed on numpy host arrays (outputs preallocated), staged through
    the context's device buffers (MDX_HOST_BUFFERS); returns when the results
    are in host memory."""
    reqs, tp = _table(reqs)
    st = lib().detect_mixed(ctx.handle, int(reqs.size), tp, _ptr(H), _ptr(y), _ptr(noise_var), _ptr(sym),
                            _ptr(metric), _ptr(vstatus), _ptr(stats), int(flags) | MDX_HOST_BUFFERS,
                            _stream(stream))
    ctx.check(st, "detect_mixed")


def autotune_mixed(ctx: Context, reqs, H, y, noise_var, stream=None):
    """Tune the uneven-batch kernel for this table (outputs are scratch);
    returns {"warps_per_cta", "slice_bytes", "ms"}."""
    import numpy as np
    import torch

    reqs, tp = _table(reqs)
    sym, met, vst, _ = detect_mixed(ctx, reqs, H, y, noise_var, stream=stream, want_stats=False)
    res = np.zeros(3)
    st = lib().mdx_autotune_mixed(ctx.handle, int(reqs.size), tp, _ptr(H), _ptr(y), _ptr(noise_var), _ptr(sym),
                                  _ptr(met), _ptr(vst), ctypes.c_void_p(res.ctypes.data), _stream(stream))
    ctx.check(st, "mdx_autotune_mixed")
    torch.cuda.synchronize()
    return {"warps_per_cta": int(res[0]), "slice_bytes": int(res[1]), "ms": float(res[2])}


# ----------------------------------------------------------------------------- learned radius


def mlp_dims(n_tx: int, qam: int):
    a, b = ctypes.c_int(), ctypes.c_int()
    st = lib().mdx_mlp_dims(n_tx, qam, ctypes.byref(a), ctypes.byref(b))
    if st != MDX_OK:
        raise MdxError(st, "mdx_mlp_dims")
    return a.value, b.value


def mlp_param_count(n_tx: int, qam: int) -> int:
    return int(lib().mdx_mlp_param_count(n_tx, qam))


def mlp_init(ctx: Context, n_tx: int, qam: int, max_train_batch: int, seed: int = 0):
    ctx.check(lib().mdx_mlp_init(ctx.handle, n_tx, qam, max_train_batch, seed), "mdx_mlp_init")


def mlp_get_params(ctx: Context, n_tx: int, qam: int):
    import numpy as np

    out = np.zeros(mlp_param_count(n_tx, qam), dtype=np.float32)
    ctx.check(lib().mdx_mlp_get_params(ctx.handle, ctypes.c_void_p(out.ctypes.data), out.size), "get_params")
    return out


def mlp_set_params(ctx: Context, params):
    import numpy as np

    p = np.ascontiguousarray(params, dtype=np.float32)
    ctx.check(lib().mdx_mlp_set_params(ctx.handle, ctypes.c_void_p(p.ctypes.data), p.size), "set_params")


def mlp_predict(ctx: Context, params: Params, H, y, noise_var, want_features=False, stream=None):
    """Network outputs [B][d_out] (and features [B][d_in]) as torch tensors."""
    import torch

    B = int(H.shape[0])
    d_in, d_out = mlp_dims(params.n_tx, params.qam)
    out = torch.empty((B, d_out), dtype=torch.float32, device=H.device)
    feat = torch.empty((B, d_in), dtype=torch.float32, device=H.device) if want_features else None
    st = lib().mdx_mlp_predict(ctx.handle, ctypes.byref(params), B, _ptr(H), _ptr(y), _ptr(noise_var), _ptr(out),
                               _ptr(feat), _stream(stream))
    ctx.check(st, "mdx_mlp_predict")
    return (out, feat) if want_features else out


def mlp_train_step(ctx: Context, params: Params, H, y, noise_var, ml_sym, ml_metric, lr=1e-3, update=True,
                   want_grad=False, stream=None):
    """One step; returns (loss tensor [2], grad tensor or None)."""
    import torch

    B = int(H.shape[0])
    loss = torch.zeros(2, dtype=torch.float32, device=H.device)
    grad = (torch.empty(mlp_param_count(params.n_tx, params.qam), dtype=torch.float32, device=H.device)
            if want_grad else None)
    st = lib().mdx_mlp_train_step(ctx.handle, ctypes.byref(params), B, _ptr(H), _ptr(y), _ptr(noise_var),
                                  _ptr(ml_sym), _ptr(ml_metric), float(lr), int(update), _ptr(grad), _ptr(loss),
                                  _stream(stream))
    ctx.check(st, "mdx_mlp_train_step")
    return loss, grad


def mlp_error(ctx: Context) -> int:
    e = ctypes.c_int()
    ctx.check(lib().mdx_mlp_error(ctx.handle, ctypes.byref(e)), "mdx_mlp_error")
    return e.value


def measure_peaks(device: int = 0, stream=None):
    """FP32 FMA, FP64 FMA and FP64 m8n8k4 MMA throughput of `device`
    (TFLOP/s, mdx_measure_peaks)."""
    import numpy as np

    out = np.zeros(4)
    st = lib().mdx_measure_peaks(int(device), ctypes.c_void_p(out.ctypes.data), _stream(stream))
    if st != MDX_OK:
        raise MdxError(st, "mdx_measure_peaks")
    return {"fp32_fma_tflops": float(out[0]), "fp64_fma_tflops": float(out[1]),
            "fp64_mma_tflops": float(out[2]), "probe_ms": float(out[3])}
