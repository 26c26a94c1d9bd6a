"""Pins of the oracle's Poisson-aware matching (Secs. 4.2-4.3) against facts
that do not come from the oracle: scipy's Poisson log-likelihood and
chi-square test, the worked Anscombe example (tests/golden), the closed-form
Pearson moments, hand-derived small-count moments, the common high-count
limit, brute-force Binomial sums written here with scipy's pmf, the
standardized null moments by full enumeration, and an independent numpy
ranking of one reference's candidates.

Each test names the passage it pins.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
METRICS = ("poisson_deviance", "pearson", "anscombe_ssd")


def np_phi(metric, r, c):
    """Eq. (varphi) written out with numpy (FP64)."""
    r = np.asarray(r, np.float64)
    c = np.asarray(c, np.float64)
    n = r + c
    with np.errstate(divide="ignore", invalid="ignore"):
        if metric == "poisson_deviance":
            a = np.where(r > 0, r * np.log(np.where(r > 0, 2 * r, 1.0) / np.where(n > 0, n, 1.0)), 0.0)
            b = np.where(c > 0, c * np.log(np.where(c > 0, 2 * c, 1.0) / np.where(n > 0, n, 1.0)), 0.0)
            return np.where(n > 0, 2 * (a + b), 0.0)
        if metric == "pearson":
            return np.where(n > 0, (r - c) ** 2 / np.where(n > 0, n, 1.0), 0.0)
        A = lambda x: 2 * np.sqrt(x + 0.375)
        return 0.5 * (A(c) - A(r)) ** 2


def brute_moments(metric, n):
    """Prop. "Universal finite-count moments" with scipy's Binomial(n, 1/2) pmf."""
    x = np.arange(n + 1)
    w = stats.binom.pmf(x, n, 0.5)
    f = np_phi(metric, x, n - x)
    mu = float(np.sum(w * f))
    return mu, float(np.sum(w * f * f) - mu * mu)


# ---------------------------------------------------------------------------
# metrics (Sec. 4.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("r,c", [(0, 0), (0, 3), (1, 0), (2, 2), (5, 1), (7, 19), (40, 55), (300, 250)])
def test_deviance_is_likelihood_ratio(oracle, r, c):
    """Prop. "Poisson deviance as symmetric likelihood-ratio distance": the
    per-entry deviance is 2 (l(separate rates) - l(pooled rate)), here from
    scipy's Poisson log-pmf."""
    if r + c == 0:
        assert oracle.phi("poisson_deviance", r, c) == 0.0
        return
    m = (r + c) / 2
    lr = 2 * (stats.poisson.logpmf(r, r) + stats.poisson.logpmf(c, c)
              - stats.poisson.logpmf(r, m) - stats.poisson.logpmf(c, m))
    assert oracle.phi("poisson_deviance", r, c) == pytest.approx(lr, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("r,c", [(1, 0), (2, 2), (5, 1), (7, 19), (40, 55), (0.5, 2.25)])
def test_pearson_is_chi_square(oracle, r, c):
    """Remark "Pearson statistic as classical chi-square test for two Poisson
    counts": equals scipy's chi-square statistic against the equal split."""
    ref = stats.chisquare([r, c]).statistic
    assert oracle.phi("pearson", r, c) == pytest.approx(ref, rel=1e-12)
    assert oracle.phi("pearson", 0, 0) == 0.0


def test_anscombe_worked_example(oracle):
    """Example "Breakdown of Anscombe approximation for small counts": the
    moments of A(K) for K ~ Poi(1) printed in the paper."""
    g = json.load(open(os.path.join(GOLDEN, "anscombe_small_count_example.json")))
    k = np.arange(0, 60)
    w = stats.poisson.pmf(k, g["poisson_mean"])
    a = np.array([oracle.anscombe(float(x)) for x in k])
    e1, e2 = float(np.sum(w * a)), float(np.sum(w * a * a))
    assert e2 == pytest.approx(g["E_A2"], abs=1e-12)
    assert e1 == pytest.approx(g["E_A"], abs=g["printed_digits_tolerance"])
    assert e2 - e1 * e1 == pytest.approx(g["Var_A"], abs=g["printed_digits_tolerance"])
    # Def. "Anscombe-SSD matching statistic": half the squared difference
    assert oracle.phi("anscombe_ssd", 3, 7) == pytest.approx(0.5 * (oracle.anscombe(7) - oracle.anscombe(3)) ** 2)


def test_common_high_count_limit(oracle):
    """Thm. "Common high-count limit": near equal large counts all three
    contributions agree to leading order, 2 m delta^2 for r, c = m (1 +- delta)."""
    m, d = 1e6, 1e-3
    r, c = m * (1 + d), m * (1 - d)
    for metric in METRICS:
        assert oracle.phi(metric, r, c) == pytest.approx(2 * m * d * d, rel=2e-3)


@pytest.mark.parametrize("metric", METRICS)
def test_phi_matches_numpy_definition(oracle, metric):
    """Eq. (varphi) on random real-valued raw counts, zero counts included."""
    rng = np.random.default_rng(7)
    r = np.concatenate([rng.gamma(0.7, 3.0, 200), [0, 0, 1, 0.25]])
    c = np.concatenate([rng.gamma(0.7, 3.0, 200), [0, 2, 0, 0.25]])
    got = np.array([oracle.phi(metric, a, b) for a, b in zip(r, c)])
    np.testing.assert_allclose(got, np_phi(metric, r, c), rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------
# finite-count moments (Sec. 4.3)
# ---------------------------------------------------------------------------

def test_pearson_moments_closed_form(oracle):
    """Prop. "Exact Pearson moments": mu = 1, v = 2 - 2/n for n >= 1; 0 at n = 0."""
    assert oracle.moments("pearson", 0) == (0.0, 0.0)
    for n in list(range(1, 120)) + [500, 2048, 4096]:
        mu, v = oracle.moments("pearson", n)
        # (log-gamma weights carry ~1e-12 relative error at n in the thousands)
        assert mu == pytest.approx(1.0, abs=1e-10)
        assert v == pytest.approx(2 - 2 / n, abs=1e-9)


def test_small_count_moments_by_hand(oracle):
    """Prop. "Universal finite-count moments" at n = 1, 2 by hand: the
    allocations (1,0), (0,1) give 2 log 2 (deviance) and
    2 (sqrt(11/8) - sqrt(3/8))^2 (Anscombe) with zero variance; n = 2 gives the
    deviance 4 log 2 with probability 1/2 and 0 otherwise."""
    l2 = math.log(2)
    assert oracle.moments("poisson_deviance", 1) == (pytest.approx(2 * l2, rel=1e-15), 0.0)
    a1 = 2 * (math.sqrt(11 / 8) - math.sqrt(3 / 8)) ** 2
    assert oracle.moments("anscombe_ssd", 1) == (pytest.approx(a1, rel=1e-15), 0.0)
    mu, v = oracle.moments("poisson_deviance", 2)
    assert mu == pytest.approx(2 * l2, rel=1e-14)
    assert v == pytest.approx(4 * l2 * l2, rel=1e-13)
    for metric in METRICS:
        assert oracle.moments(metric, 0) == (0.0, 0.0)


@pytest.mark.parametrize("metric", METRICS)
def test_moments_brute_force(oracle, metric):
    """Prop. "Universal finite-count moments" against a Binomial(n, 1/2) sum
    written here with scipy's pmf and the numpy contributions."""
    for n in list(range(2, 61)) + [150, 400]:
        mu, v = oracle.moments(metric, n)
        bm, bv = brute_moments(metric, n)
        assert mu == pytest.approx(bm, rel=1e-11, abs=1e-13)
        assert v == pytest.approx(bv, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("metric", METRICS)
def test_moments_high_count_limit(oracle, metric):
    """Thm. "Common high-count limit": the null contribution tends to chi^2_1
    (mean 1, variance 2)."""
    mu, v = oracle.moments(metric, 4000)
    assert mu == pytest.approx(1.0, abs=2e-3)
    assert v == pytest.approx(2.0, abs=5e-3)


@pytest.mark.parametrize("metric", METRICS)
def test_standardized_null_moments_by_enumeration(oracle, metric):
    """Cor. "Standardized null moments": with pooled counts n = (3, 5, 2) fixed,
    Z_m over every allocation (x_i ~ Bin(n_i, 1/2), independent) has mean 0 and
    variance 1; Z_m built from Def. "Candidate-standardized distance"."""
    n = (3, 5, 2)
    mom = [oracle.moments(metric, k) for k in n]
    smu = sum(m for m, _ in mom)
    ssd = math.sqrt(sum(v for _, v in mom))
    e1 = e2 = 0.0
    for xs in itertools.product(*[range(k + 1) for k in n]):
        w = math.prod(stats.binom.pmf(x, k, 0.5) for x, k in zip(xs, n))
        z = (sum(oracle.phi(metric, x, k - x) for x, k in zip(xs, n)) - smu) / ssd
        e1 += w * z
        e2 += w * z * z
    assert e1 == pytest.approx(0.0, abs=1e-12)
    assert e2 == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("metric", METRICS)
def test_float_tables_round_fp64_moments(oracle, metric):
    """The float32 tables the decisions read are the FP64 moments rounded."""
    mu, v = oracle.moment_table_f32(metric, 300)
    for n in (0, 1, 2, 3, 17, 299):
        m, s = oracle.moments(metric, n)
        assert mu[n] == np.float32(m) and v[n] == np.float32(s)


def _np_threshold(metric, policy, pref, P, t, beta, kappa, tau=None):
    if policy == "fixed":
        return P * (tau if tau else 1 + t * math.sqrt(2 / P))
    if policy == "candidate_standardized":
        return t
    mom = [brute_moments(metric, int(round(2 * r))) for r in pref]
    rbar = float(np.mean(pref))
    return sum(m for m, _ in mom) + t * math.sqrt(sum(v for _, v in mom)) + beta * P * rbar ** kappa


def _np_score(metric, policy, pref, q):
    acc = float(np.sum(np_phi(metric, pref, q)))
    if policy != "candidate_standardized":
        return acc
    mom = [brute_moments(metric, int(round(a + b))) for a, b in zip(pref, q)]
    sv = sum(v for _, v in mom)
    return (acc - sum(m for m, _ in mom)) / math.sqrt(sv) if sv > 0 else 0.0


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("policy", ["fixed", "reference_finite_count", "candidate_standardized"])
def test_match_ref_against_numpy_ranking(oracle, metric, policy):
    """Sec. 4.3 acceptance (Def. "Reference finite-count threshold", Def.
    "Candidate-standardized distance", the fixed high-count rule) and App. A
    group rules, against an independent FP64 ranking: the oracle's members are
    the accepted candidates in ascending score (at most M - 1 after the
    reference), except where two FP64 scores or a score and the threshold lie
    within float rounding of each other."""
    rng = np.random.default_rng(11)
    lam = 6.0
    x = 1.0 + 0.8 * np.sin(np.arange(96) / 5.0)
    k = rng.poisson(lam * x)
    s_p = 1.0 / lam
    y = (k * s_p).astype(np.float32).astype(np.float64)
    patch, search, M = 8, 31, 8
    p = oracle.params((96,), (patch,), (2,), (search,), noise=("poisson", s_p), group_size=(M, M),
                      match_metric=metric, match_policy=policy, match_t=1.0)
    checked = 0
    for ref in (20, 41, 60):
        mem, _ = oracle.match_ref(p, y, 1, ref)
        counts = np.maximum(y / s_p, 0)
        pref = counts[ref:ref + patch]
        T = _np_threshold(metric, policy, pref, patch, 1.0, 0.1, 1.0)
        lo, hi = max(ref - search // 2, 0), min(ref + search // 2, 96 - patch)
        cand = [(c, _np_score(metric, policy, pref, counts[c:c + patch])) for c in range(lo, hi + 1) if c != ref]
        cand.sort(key=lambda t: (t[1], t[0]))
        scale = max(abs(T), 1.0)
        if any(abs(s - T) < 1e-4 * scale for _, s in cand):
            continue
        acc = [c for c, s in cand if s < T]
        take = min(len(acc), M - 1)
        if 1 + take < 2:
            take = 1
        count = 1 + take
        pw = 1
        while pw * 2 <= count:
            pw *= 2
        assert mem[0] == ref and len(mem) == pw, (ref, list(mem), acc)
        scores = dict(cand)
        want = [c for c, _ in cand[: pw - 1]]
        for a, b in zip(mem[1:], want):
            if a != b:
                assert abs(scores[a] - scores[b]) < 1e-5 * max(abs(scores[b]), 1.0)
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("metric", METRICS)
def test_contributions_symmetric_nonnegative(oracle, metric):
    """Eqs. (deviance), (pearson), (anscombe-distance): each contribution is
    symmetric in (r, c), non-negative, and zero exactly when r = c."""
    rng = np.random.default_rng(9)
    for r, c in zip(rng.gamma(0.8, 5.0, 200), rng.gamma(0.8, 5.0, 200)):
        a, b = oracle.phi(metric, r, c), oracle.phi(metric, c, r)
        assert a == pytest.approx(b, rel=1e-12, abs=1e-15)
        assert a > 0.0
        assert oracle.phi(metric, r, r) == pytest.approx(0.0, abs=1e-12)


def test_exact_sum_is_fsum(oracle):
    """The oracle's summation of Poisson contributions equals Python's
    math.fsum (Shewchuk's exact summation rounded once) on sums that a
    sequential double sum gets wrong, and does not depend on term order."""
    rng = np.random.default_rng(4)
    for k in range(100):
        x = rng.standard_normal(int(rng.integers(1, 70))) * 10.0 ** int(rng.integers(-12, 12))
        x = np.concatenate([x, [1e16, 1.0, -1e16], x[:2] * 1e-20])
        assert oracle.exact_sum(x) == math.fsum(x)
        assert oracle.exact_sum(x[rng.permutation(len(x))]) == oracle.exact_sum(x)
    assert oracle.exact_sum([1e16, 1.0, -1e16]) == 1.0


@pytest.mark.parametrize("metric,a,b", [
    ("ssd", (29, 3, 2, 2, 4, 13, 24, 19), (2, 13, 2, 4, 3, 24, 19, 29)),
    ("poisson_deviance", (9, 8, 27, 24, 25, 5, 12, 11), (12, 9, 27, 25, 11, 8, 5, 24)),
    ("pearson", (0, 28, 17, 6, 23, 17, 2, 20), (0, 20, 28, 17, 2, 17, 23, 6)),
    ("anscombe_ssd", (21, 19, 18, 6, 28, 11, 15, 9), (18, 21, 19, 11, 28, 15, 9, 6))])
def test_permuted_patches_tie_exactly(oracle, metric, a, b):
    """Two candidates whose per-entry terms are a permutation of each other
    tie in real arithmetic; their scores must be equal, so that the smaller
    index ranks first (App. A group order).  Guide: the reference counts 7 on
    all 8 entries at origin 0, a candidate at origin 8 and a permutation of it
    at origin 16, s_P = 0.1 (raw counts not exact in binary).  SSD: gamma = 0
    (Eq. ssd); the Poisson distances: standardized policy, every candidate
    accepted.  The pairs are chosen so that a sequential double-precision
    sum splits the tie (checked here)."""
    s_p = 0.1
    P = 8
    ref = np.full(P, 7.0)
    a, b = np.array(a, float), np.array(b, float)
    g = (np.concatenate([ref, a, b]) * s_p).astype(np.float32).astype(np.float64)
    counts = g / s_p

    def seqsum(v):
        t = 0.0
        for x in v:
            t += x
        return t

    if metric == "ssd":
        seq = [seqsum((g[o:o + P] - g[:P]) ** 2) for o in (P, 2 * P)]
        p = oracle.params(g.shape, (P,), (1,), (33,), ("poisson", s_p), (32, 32), gamma_ht=0.0, tau_ht=1e9,
                          group_transform="dct")
    else:
        seq = [seqsum([oracle.phi(metric, r, c) for r, c in zip(counts[:P], counts[o:o + P])]) for o in (P, 2 * P)]
        p = oracle.params(g.shape, (P,), (1,), (33,), ("poisson", s_p), (32, 32), group_transform="dct", match_metric=metric,
                          match_policy="candidate_standardized", match_t=1e9)
    assert seq[0] != seq[1]
    mem, sc = oracle.match_ref(p, g, 1, 0)
    scores = dict(zip(mem[1:], sc[1:]))
    assert P in scores and 2 * P in scores
    assert scores[P] == scores[2 * P]
    assert list(mem).index(P) < list(mem).index(2 * P)


def test_raw_counts_recover_integers(oracle):
    """Eq. (raw-counts) recovers the counts K of y = s_P K stored in float32
    (relative rounding 2^-24) for the scales the workloads use; values off
    an integer by more than a relative 2^-20 are kept."""
    for s_p in (0.1, 1 / 50.0, 0.2, 1 / 30.0, 1 / 7.3):
        p = oracle.params((8,), (2,), (1,), (3,), ("poisson", s_p))
        for k in (0, 1, 2, 3, 17, 49, 50, 123, 4095, 8191):
            y = float(np.float32(k * s_p))
            assert oracle.raw_count(p, y) == k
        y = float(np.float32(3.3 * s_p))
        assert abs(oracle.raw_count(p, y) - 3.3) < 1e-6
        assert oracle.raw_count(p, -y) == 0.0
