"""detect_kbest_noalloc: the K-best entry point for callers that may not
allocate device memory (for example a receiver that fixes its memory at
start-up and forbids allocation on its data path).  It takes no context and
keeps its scratch in a static device array inside the library, so it must
give exactly what detect_kbest gives, call after call, even though every call
reuses the scratch the previous one left behind.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""

import ctypes
import math

import pytest

from paper_2002_09561_gb300 import workload as wl

pytestmark = pytest.mark.gpu

MET_RTOL = 1e-5  # the metric tolerance of the other parity tests


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2002_09561_gb300 import mdx

    torch.cuda.set_device(0)
    ctx = mdx.Context(0, max_batch=2048, max_n_rx=16, max_n_tx=16)
    yield torch, mdx, ctx
    ctx.close()


def _inputs(torch, seed, B, N, M, qam, snr):
    w = wl.generate(seed, B, N, M, qam, snr)
    dev = torch.device("cuda:0")
    return [torch.from_numpy(w[k]).to(dev) for k in ("H", "y", "noise_var")]


def _noalloc(torch, mdx, params, H, y, nv):
    B = int(H.shape[0])
    sym, met, vst, stats = mdx._outputs(B, params.n_tx, H.device, True)
    p = mdx._ptr
    st = mdx.lib().detect_kbest_noalloc(ctypes.byref(params), B, p(H), p(y), p(nv), p(sym), p(met), p(vst),
                                        p(stats), mdx._stream(None))
    return st, (sym, met, vst, stats)


def _same(torch, a, b):
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]), "detected indices differ"
    assert torch.equal(a[2], b[2]), "per-vector status differs"
    rel = ((a[1] - b[1]).abs() / b[1].abs().clamp_min(1e-300)).max().item()
    assert rel < MET_RTOL, rel
    assert torch.equal(a[3], b[3]), "statistics differ"


def test_noalloc_matches_detect_kbest_on_consecutive_calls(env):
    torch, mdx, ctx = env
    # two calls in a row with different sizes and data: the second must not
    # see anything the first left in the shared scratch
    cases = [(101, 1500, 16, 16, 16, 10.0, 64, math.inf),
             (102, 333, 12, 10, 64, 20.0, 16, "paper")]
    for seed, B, N, M, qam, snr, K, radius in cases:
        H, y, nv = _inputs(torch, seed, B, N, M, qam, snr)
        params = mdx.make_params(N, M, qam, radius=radius, K=K)
        st, got = _noalloc(torch, mdx, params, H, y, nv)
        assert st == mdx.MDX_OK, st
        ref = mdx.detect("kbest", ctx, params, H, y, nv)
        _same(torch, got, ref)


def test_noalloc_matches_detect_kbest_blocked_qr_and_complex_tree(env):
    """The 100x100 systems take the blocked FP64 QR (and its scratch nearly
    fills the array: about 243 KB per vector, so 60 vectors); the complex
    tree takes the K-best kernel's complex level steps.  Two calls in a row
    each, against detect_kbest."""
    torch, mdx, _ = env
    big = mdx.Context(0, max_batch=64, max_n_rx=100, max_n_tx=100)
    try:
        for seed in (111, 112):
            H, y, nv = _inputs(torch, seed, 60, 100, 100, 64, 28.0)
            params = mdx.make_params(100, 100, 64, K=32)
            st, got = _noalloc(torch, mdx, params, H, y, nv)
            assert st == mdx.MDX_OK, st
            _same(torch, got, mdx.detect("kbest", big, params, H, y, nv))
    finally:
        big.close()
    _, _, ctx = env
    for seed in (113, 114):
        H, y, nv = _inputs(torch, seed, 200, 8, 8, 16, 12.0)
        params = mdx.make_params(8, 8, 16, K=16, flags=mdx.MDX_COMPLEX_TREE)
        st, got = _noalloc(torch, mdx, params, H, y, nv)
        assert st == mdx.MDX_OK, st
        _same(torch, got, mdx.detect("kbest", ctx, params, H, y, nv))


def test_noalloc_rejects_batches_beyond_its_scratch(env):
    torch, mdx, ctx = env
    per_vector = 8 * (528 + 32) + 4 * (528 + 32) + 4  # 16x16: R and ybar in FP64 and FP32, flag
    B = mdx.NOALLOC_SCRATCH_BYTES // per_vector + 10
    H = torch.zeros((B, 16, 16, 2), dtype=torch.float64, device="cuda")
    y = torch.zeros((B, 16, 2), dtype=torch.float64, device="cuda")
    nv = torch.ones(B, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(torch, mdx, mdx.make_params(16, 16, 16, K=16), H, y, nv)
    assert st == mdx.MDX_EUNSUPPORTED
    # and still works afterwards
    H, y, nv = _inputs(torch, 7, 64, 16, 16, 16, 14.0)
    params = mdx.make_params(16, 16, 16, K=16)
    st, got = _noalloc(torch, mdx, params, H, y, nv)
    assert st == mdx.MDX_OK
    _same(torch, got, mdx.detect("kbest", ctx, params, H, y, nv))


def test_noalloc_rejects_host_buffers_and_the_flags_detect_kbest_rejects(env):
    torch, mdx, ctx = env
    H, y, nv = _inputs(torch, 8, 4, 4, 4, 4, 10.0)
    for flag in (mdx.MDX_HOST_BUFFERS, mdx.MDX_LEARNED_RADIUS, mdx.MDX_LEARNED_ORDER, mdx.MDX_ORDER_NATURAL):
        params = mdx.make_params(4, 4, 4, K=4, flags=flag)
        st, _ = _noalloc(torch, mdx, params, H, y, nv)
        assert st == mdx.MDX_EUNSUPPORTED, flag
        if flag != mdx.MDX_HOST_BUFFERS:
            with pytest.raises(mdx.MdxError) as e:
                mdx.detect("kbest", ctx, params, H, y, nv)
            assert e.value.status == mdx.MDX_EUNSUPPORTED
    # a size whose shared memory detect_kbest refuses (complex tree at 100x100
    # 64-QAM, K = 256: 16,384 keys of 8 bytes beside R and the paths) is
    # refused here too, before any launch
    H, y, nv = _inputs(torch, 9, 4, 100, 100, 64, 20.0)
    params = mdx.make_params(100, 100, 64, K=256, flags=mdx.MDX_COMPLEX_TREE)
    st, _ = _noalloc(torch, mdx, params, H, y, nv)
    assert st == mdx.MDX_EUNSUPPORTED
