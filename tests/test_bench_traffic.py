"""The benchmark's stored DRAM-traffic and instructions-per-node figures are
tied to the code they were captured on: code_hash ignores comments and
spacing but not code, and a figure whose kernel sources hash differently is
not reported."""

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_code_hash_ignores_comments_not_code(tmp_path):
    b = _bench()
    (tmp_path / "k.cu").write_text("// a\nint f(int x) { return x + 1; } /* b */\n")
    h0 = b.code_hash(["k.cu"], csrc=str(tmp_path))
    (tmp_path / "k.cu").write_text("/* other\n comment */ int f(int x)  {\n  return x + 1;  // c\n}\n")
    assert b.code_hash(["k.cu"], csrc=str(tmp_path)) == h0
    (tmp_path / "k.cu").write_text("int f(int x) { return x + 2; }\n")
    assert b.code_hash(["k.cu"], csrc=str(tmp_path)) != h0


def test_traffic_reported_only_for_the_captured_code():
    b = _bench()
    for workload, (value, source, h) in b.TRAFFIC_PER_VECTOR.items():
        got, why = b.traffic_per_vector(workload)
        if b.code_hash(b.KERNEL_SOURCES[workload]) == h:
            assert got == value and why == source
        else:
            assert got is None and "changed since its capture" in why
    b.TRAFFIC_PER_VECTOR["16x16-16qam-sd-learned"] = (1.0, "x", "0" * 16)
    assert b.traffic_per_vector("16x16-16qam-sd-learned")[0] is None
    assert b.traffic_per_vector("no such workload") == (None, "no capture of the current kernel")


def test_instructions_per_node_reported_only_for_the_captured_code():
    b = _bench()
    for workload, (value, source, h) in b.INSTRUCTIONS_PER_NODE.items():
        got, why = b.instructions_per_node(workload)
        if b.code_hash(b.KERNEL_SOURCES[workload]) == h:
            assert got == value and why == source
        else:
            assert got is None and "changed since its capture" in why
    b.INSTRUCTIONS_PER_NODE["16x16-16qam-sd-learned"] = (1.0, "x", "0" * 16)
    assert b.instructions_per_node("16x16-16qam-sd-learned")[0] is None
    assert b.instructions_per_node("no such workload") == (None, "no capture of the current kernel")


def test_issue_rate_in_the_search_roofline():
    import numpy as np

    b = _bench()
    stats = np.zeros((2, 5), dtype=np.int64)
    stats[:, 0] = 1000  # nodes
    stats[:, 4] = 40000  # flops
    r = b.search_roofline("16x16-16qam-sd-learned", "sd", stats, 2.0, 1, 0.5, 152,
                          {"fp32_fma_tflops": 77.0}, 2)
    ipn, _ = b.instructions_per_node("16x16-16qam-sd-learned")
    assert r["issue"]["warp_instructions_per_node"] == ipn
    if ipn:
        # 2,000 nodes in 2 ms at ipn instructions each
        assert abs(r["issue"]["achieved"] - ipn * 2000 / 2e-3 / 1e12) < 1e-12
        assert abs(r["issue"]["frac"] - r["issue"]["achieved"] / r["issue"]["peak"]) < 1e-12
