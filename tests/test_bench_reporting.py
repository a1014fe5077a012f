"""The benchmark's reporting helpers, on the CPU: the Gray-coded bit-error
count against the oracle's (itself pinned on adjacent-level errors), the
per-SNR breakdown and the oracle check on small hand-built cases, the QR's
algorithmic flop count against its closed form, and the launch count per
step."""

import importlib.util
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("qam", [4, 16, 64])
def test_gray_bit_errors_equal_the_oracle_count(qam):
    b = _bench()
    rng = np.random.default_rng(qam)
    truth = rng.integers(0, qam, size=(300, 8)).astype(np.uint8)
    hat = truth.copy()
    flip = rng.random(truth.shape) < 0.2
    hat[flip] = rng.integers(0, qam, size=int(flip.sum())).astype(np.uint8)
    bits = b.gray_bit_errors(hat, truth, qam)
    assert bits.shape == (300,)
    assert int(bits.sum()) == oracle.count_errors(hat, truth, qam)[0]
    assert (bits[(hat == truth).all(axis=1)] == 0).all()


def test_per_snr_breakdown_by_hand():
    b = _bench()
    w = {"snr": [4.0, 20.0], "qam": 4, "n": 2}  # QPSK: 2 bits per symbol, 4 per vector
    truth = np.zeros((4, 2), dtype=np.uint8)
    sym = truth.copy()
    sym[0, 0] = 3  # vector 0 (4 dB): both bits of one symbol wrong
    sym[2, 1] = 1  # vector 2 (4 dB): one bit wrong
    vst = np.array([1, 0, 0, 2], dtype=np.int32)  # a radius doubling at 4 dB, a budget stop at 20 dB
    st = np.zeros((4, 5), dtype=np.int64)
    st[:, 0] = [10, 20, 30, 40]
    rows = b.per_snr(w, (sym, vst, st), truth)
    lo, hi = rows
    assert lo["snr_db"] == 4.0 and lo["vectors"] == 2 and hi["vectors"] == 2
    assert lo["ber"] == pytest.approx(3 / 8) and hi["ber"] == 0.0
    assert lo["ser"] == pytest.approx(2 / 4) and hi["ser"] == 0.0
    assert lo["mean_nodes"] == 20.0 and hi["mean_nodes"] == 30.0
    assert lo["p99_nodes"] == pytest.approx(np.percentile([10, 30], 99))
    assert lo["radius_doubling_rate"] == 0.5 and hi["radius_doubling_rate"] == 0.0
    assert lo["budget_rate"] == 0.0 and hi["budget_rate"] == 0.5


def test_oracle_check_counts_mismatches_and_near_ties():
    b = _bench()
    w = {"snr": [10.0], "qam": 16, "n": 2, "detector": "sd"}
    truth = np.array([[1, 2], [3, 4], [5, 6], [7, 8]], dtype=np.uint8)
    ref = {"sym": truth.copy(), "metric": np.array([1.0, 2.0, 3.0, 4.0]),
           "gap": np.array([0.5, 0.5, 1e-9, 0.5])}
    gpu_sym = truth.copy()
    gpu_sym[1, 0] = 9  # a mismatch with a clear gap: counted
    gpu_sym[2, 1] = 9  # a mismatch on a near-tie: allowed
    gpu_met = ref["metric"] * np.array([1.0 + 1e-12, 1.0, 1.0, 1.0 - 2e-12])
    d = {"noise_var": np.ones(4), "sym": truth}
    r = b.oracle_check(w, d, ref, gpu_sym, gpu_met, seed=7)
    assert r["vectors"] == 4 and r["identical"] == 2
    assert r["mismatches_outside_near_ties"] == 1 and r["differing_near_ties"] == 1
    assert r["near_tie_fraction"] == 0.25
    assert r["max_rel_metric_error"] == pytest.approx(2e-12, rel=1e-3)
    assert r["ber_per_snr"][0]["oracle"] == 0.0 and r["ber_per_snr"][0]["gpu"] > 0.0


def test_qr_roofline_flops_are_the_householder_count():
    b = _bench()
    probe = {"fp64_fma_tflops": 1.0, "fp64_mma_tflops": 1.1}
    r = b.qr_roofline(16, 16, 1000, (2.0, None, 1), 152, probe)
    # 8 (N M^2 - M^3 / 3) real flops per complex 16 x 16 Householder QR
    assert r["flops_per_matrix"] == pytest.approx(8 * (16 * 256 - 4096 / 3))
    assert r["achieved"] == pytest.approx(r["flops_per_matrix"] * 1000 / 2e-3 / 1e12)
    assert r["frac_of_measured"] == pytest.approx(r["achieved"] / 1.1)


def test_launches_per_step():
    b = _bench()
    # QR, search, error count; the network's five kernels; the SD's three ordering kernels
    assert b.launches_per_call("sd", True, 32) == 11
    assert b.launches_per_call("sd", False, 32) == 6
    assert b.launches_per_call("kbest", False, 32) == 3
    assert b.launches_per_call("hybrid", True, 200) == 8
