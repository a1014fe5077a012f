"""Pins of the oracle's near-tie gaps (the numbers that decide which vectors
the GPU parity tests exempt).

The K-best of Sec. VI keeps, at every row, the K candidates with the least
partial distance; two candidates on either side of that cut whose distances
agree to FP32 precision may legitimately change places on the GPU, and so
may the two best final leaves.  orc_kbest, orc_kbest_complex and orc_hybrid
therefore report the smallest relative gap (hi - lo) / hi over every K / K+1
cut and every final best / second-best pair they met.  A bug that shrinks
those gaps would silently widen the parity exemption, so they are recomputed
here by an independent restatement: candidates' partial distances evaluated
directly as sum over rows r >= i of (ybar_r - sum_{j >= r} R_rj a_{x_j})^2
(Eq. 4 written out, not the incremental Eq. inc the oracle accumulates),
every level's full candidate list kept and sorted by numpy's lexsort on
(distance, parent rank, child), the hybrid's master as an explicit
depth-first recursion in increasing partial distance (Best-FS, Sec. IV-A).
Tiny systems only; the gaps must agree to 1e-12 and the answers exactly.
"""

import numpy as np
import pytest

import oracle
from paper_2002_09561_gb300 import workload as wl


def _system(seed, M, qam, snr):
    w = wl.generate(seed, 1, M, M, qam, snr)
    Hr, yr = oracle.real_decompose(w["H"][0], w["y"][0])
    f = oracle.qr(Hr, yr)
    return f["R"], f["ybar"], float(w["noise_var"][0])


def _ped(R, yb, lev, x, i):
    """Partial distance of the rows i..n-1 fixed in x (Eq. 4, directly)."""
    res = yb[i:] - R[i:, i:] @ lev[x[i:]]
    return float(res @ res)


def _rel_gap(lo, hi):
    if hi > 0.0:
        return (hi - lo) / hi
    return 0.0 if hi == lo else 1.0


class _Kbest:
    """K-best over rows top..0 from one node (prefix fixed above `top`)."""

    def __init__(self, R, yb, lev, K):
        self.R, self.yb, self.lev, self.K = R, yb, lev, K
        self.n, self.P = R.shape[0], len(lev)

    def run(self, r2, top, prefix, gaps):
        surv = [prefix.copy()]
        for i in range(top, -1, -1):
            peds, ranks, kids, paths = [], [], [], []
            for rank, x in enumerate(surv):
                for k in range(self.P):
                    z = x.copy()
                    z[i] = k
                    d = _ped(self.R, self.yb, self.lev, z, i)
                    if d < r2:
                        peds.append(d)
                        ranks.append(rank)
                        kids.append(k)
                        paths.append(z)
            if not peds:
                return None, None
            order = np.lexsort((np.array(kids), np.array(ranks), np.array(peds)))
            srt = [peds[t] for t in order]
            if len(srt) > self.K:
                gaps.append(_rel_gap(srt[self.K - 1], srt[self.K]))
            surv = [paths[t] for t in order[:self.K]]
            last = srt[:self.K]
        if len(surv) > 1:
            gaps.append(_rel_gap(last[0], last[1]))
        return surv[0], last[0]


def np_kbest(R, yb, lev, K, r2):
    kb = _Kbest(R, yb, lev, K)
    while True:
        gaps = []
        x, d = kb.run(r2, kb.n - 1, np.zeros(kb.n, dtype=int), gaps)
        if x is not None:
            return x, d, min(gaps, default=1.0)
        r2 *= 2.0


def np_kbest_complex(R, yb, lev, K, r2):
    n, P = R.shape[0], len(lev)
    while True:
        gaps = []
        surv, last = [np.zeros(n, dtype=int)], None
        for j in range(n // 2 - 1, -1, -1):
            peds, ranks, kids, paths = [], [], [], []
            for rank, x in enumerate(surv):
                for q in range(P * P):
                    z = x.copy()
                    z[2 * j], z[2 * j + 1] = q // P, q % P
                    d = _ped(R, yb, lev, z, 2 * j)
                    if d < r2:
                        peds.append(d)
                        ranks.append(rank)
                        kids.append(q)
                        paths.append(z)
            if not peds:
                surv = None
                break
            order = np.lexsort((np.array(kids), np.array(ranks), np.array(peds)))
            srt = [peds[t] for t in order]
            if len(srt) > K:
                gaps.append(_rel_gap(srt[K - 1], srt[K]))
            surv = [paths[t] for t in order[:K]]
            last = srt[:K]
        if surv is not None:
            if len(surv) > 1:
                gaps.append(_rel_gap(last[0], last[1]))
            return surv[0], last[0], min(gaps, default=1.0)
        r2 *= 2.0


def np_hybrid(R, yb, lev, K, d, r2):
    """Best-FS master over the top d rows; every node reached at depth d
    inside the current sphere is finished by K-best with the current radius,
    and a better leaf shrinks the radius (Sec. VI)."""
    n, P = R.shape[0], len(lev)
    kb = _Kbest(R, yb, lev, K)
    while True:
        st = {"r2": r2, "best": None, "gaps": []}

        def visit(i, x):
            peds = []
            for k in range(P):
                z = x.copy()
                z[i] = k
                peds.append(_ped(R, yb, lev, z, i))
            for k in np.argsort(np.array(peds), kind="stable"):
                if not peds[k] < st["r2"]:
                    continue
                z = x.copy()
                z[i] = k
                if i == n - d:
                    leaf, lp = kb.run(st["r2"], i - 1, z, st["gaps"])
                    if leaf is not None and lp < st["r2"]:
                        st["r2"], st["best"] = lp, leaf
                else:
                    visit(i - 1, z)

        visit(n - 1, np.zeros(n, dtype=int))
        if st["best"] is not None:
            return st["best"], st["r2"], min(st["gaps"], default=1.0)
        r2 *= 2.0


CASES_KB = [(3, 16, 4, "inf", 6.0), (4, 4, 3, "inf", 2.0), (3, 64, 5, "paper", 14.0), (2, 16, 2, "paper", 0.0),
            (3, 4, 1, "inf", 4.0)]


@pytest.mark.parametrize("M,qam,K,radius,snr", CASES_KB)
def test_kbest_gap_recomputed_independently(M, qam, K, radius, snr):
    lev = oracle.pam_levels(qam)
    seen_cut = False
    for seed in range(8):
        R, yb, nv = _system(900 + 17 * seed + M, M, qam, snr)
        r2 = np.inf if radius == "inf" else M * M * nv  # r^2 = N M sigma^2 (Sec. III-B), N = M
        got = oracle.kbest(R, yb, qam, K, r2)
        x, d, g = np_kbest(R, yb, lev, K, r2)
        np.testing.assert_array_equal(got["k"], x)
        assert got["d1"] == pytest.approx(d, rel=1e-12)
        assert abs(got["gap"] - g) < 1e-12, (seed, got["gap"], g)
        seen_cut |= g < 1.0
    assert seen_cut


@pytest.mark.parametrize("M,qam,K,radius,snr", [(3, 16, 4, "inf", 6.0), (2, 64, 6, "inf", 10.0),
                                                (3, 4, 2, "paper", 3.0)])
def test_kbest_complex_gap_recomputed_independently(M, qam, K, radius, snr):
    lev = oracle.pam_levels(qam)
    for seed in range(6):
        R, yb, nv = _system(950 + 13 * seed + M, M, qam, snr)
        r2 = np.inf if radius == "inf" else M * M * nv
        got = oracle.kbest_complex(R, yb, qam, K, r2)
        x, d, g = np_kbest_complex(R, yb, lev, K, r2)
        np.testing.assert_array_equal(got["k"], x)
        assert got["d1"] == pytest.approx(d, rel=1e-12)
        assert abs(got["gap"] - g) < 1e-12, (seed, got["gap"], g)


@pytest.mark.parametrize("M,qam,K,d,radius,snr", [(3, 16, 3, 2, "paper", 8.0), (4, 4, 2, 3, "inf", 2.0),
                                                  (3, 64, 4, 1, "paper", 16.0), (3, 16, 2, 4, "inf", 4.0)])
def test_hybrid_gap_recomputed_independently(M, qam, K, d, radius, snr):
    lev = oracle.pam_levels(qam)
    for seed in range(6):
        R, yb, nv = _system(990 + 11 * seed + M + d, M, qam, snr)
        r2 = np.inf if radius == "inf" else M * M * nv
        got = oracle.hybrid(R, yb, qam, K, d, r2)
        x, dist, g = np_hybrid(R, yb, lev, K, d, r2)
        np.testing.assert_array_equal(got["k"], x)
        assert got["d1"] == pytest.approx(dist, rel=1e-12)
        assert abs(got["gap"] - g) < 1e-12, (seed, got["gap"], g)


def test_detect_batch_reports_the_same_gaps():
    """The batch driver (what the parity tests call) passes the same gaps
    through, for K-best and the hybrid, from the channel matrices."""
    qam, K, M = 16, 3, 3
    lev = oracle.pam_levels(qam)
    w = wl.generate(4242, 12, M, M, qam, 6.0)
    kb = oracle.detect_batch("kbest", w["H"], w["y"], w["noise_var"], qam, K=K)
    hy = oracle.detect_batch("hybrid", w["H"], w["y"], w["noise_var"], qam, K=K, depth=2, radius="paper")
    for b in range(12):
        Hr, yr = oracle.real_decompose(w["H"][b], w["y"][b])
        f = oracle.qr(Hr, yr)
        _, _, g = np_kbest(f["R"], f["ybar"], lev, K, np.inf)
        assert abs(kb["gap"][b] - g) < 1e-12
        _, _, g = np_hybrid(f["R"], f["ybar"], lev, K, 2, M * M * w["noise_var"][b])
        assert abs(hy["gap"][b] - g) < 1e-12
