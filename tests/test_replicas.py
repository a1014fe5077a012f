"""The multi-GPU path's host logic with two gloo ranks on the CPU: disjoint
shards covering the stream, the max-reduction of the elapsed time, and the
sum-reduction of the error counters equal to one process over all vectors."""

import os
import socket

import numpy as np
import pytest

import oracle
from paper_2002_09561_gb300 import replicas
from paper_2002_09561_gb300 import workload as wl

N_TX, QAM, PER_RANK, SEED = 4, 16, 24, 77


def _counts(start, count):
    w = wl.generate(SEED, count, N_TX, N_TX, QAM, 8.0, start=start)
    out = oracle.detect_linear("zf", w["H"], w["y"], w["noise_var"], QAM)
    bits, syms = oracle.count_errors(out["sym"], w["sym"], QAM)
    return {"bit_errors": bits, "symbol_errors": syms, "symbols": count * N_TX}


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, count = replicas.shard(rank, world, PER_RANK)
        tot = replicas.sum_counters(_counts(start, count), dist)
        slowest = replicas.max_over_ranks(1.0 + rank, dist)
        q.put((rank, start, count, tot, slowest))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_replicas_reduce_to_the_single_process_result():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, c0, t0, m0), (r1, s1, c1, t1, m1) = res
    assert (s0, c0, s1, c1) == (0, PER_RANK, PER_RANK, PER_RANK)  # disjoint, contiguous
    assert t0 == t1 == _counts(0, 2 * PER_RANK)  # the same as one process over both shards
    assert m0 == m1 == 2.0


def test_single_process_helpers():
    assert replicas.shard(0, 1, 5) == (0, 5)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.sum_counters({"b": 2, "a": 1}) == {"a": 1, "b": 2}
    with pytest.raises(ValueError):
        replicas.shard(2, 2, 5)
