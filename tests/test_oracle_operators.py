"""Pins of the oracle's reproduction operators and objectives (Appendix B and
the DTLZ definitions): invariants, degenerate cases that reduce to identity,
closed-form distributions (KS tests) and hand-worked objective values.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


def _params(orc, **kw):
    base = dict(m=3, d=64, N=210, H=19, problem=orc.DTLZ2, t_max=100, seed=7)
    base.update(kw)
    return orc.make_params(**base)


def _parents(p, seed=0):
    rng = np.random.default_rng(seed)
    P = (p.N + 1) // 2
    return rng.uniform(0.05, 0.95, (P, p.d)), rng.uniform(0.05, 0.95, (P, p.d))


def test_sbx_mean_preserved(orc):
    p = _params(orc)
    X1, X2 = _parents(p)
    Xc = orc.sbx(p, 3, X1, X2)
    P = X1.shape[0]
    lhs = Xc[:P] + Xc[P:]
    assert np.allclose(lhs, X1 + X2, rtol=0, atol=4 * np.finfo(float).eps * 2)


def test_sbx_no_crossover_is_identity(orc):
    p = _params(orc, p_c=0.0)
    X1, X2 = _parents(p, 1)
    Xc = orc.sbx(p, 5, X1, X2)
    P = X1.shape[0]
    assert np.array_equal(Xc[:P], X1) and np.array_equal(Xc[P:], X2)


def _beta_cdf(b, eta):
    b = np.asarray(b)
    return np.where(b <= 1.0, 0.5 * b ** (eta + 1), 1.0 - 0.5 * b ** (-(eta + 1)))


@pytest.mark.parametrize("eta", [20.0, 2.0])
def test_sbx_spread_distribution(orc, eta):
    p = _params(orc, d=256, N=400, eta_c=eta)
    X1, X2 = _parents(p, 2)
    Xc = orc.sbx(p, 11, X1, X2)
    P = X1.shape[0]
    B = (Xc[:P] - Xc[P:]) / (X1 - X2)       # recovers B per site
    kept = np.isclose(B, 1.0, rtol=0, atol=1e-9)
    frac_keep = kept.mean()
    n = kept.size
    assert abs(frac_keep - 0.5) < 5 * math.sqrt(0.25 / n)
    Bs = B[~kept]
    frac_neg = (Bs < 0).mean()
    assert abs(frac_neg - 0.5) < 5 * math.sqrt(0.25 / Bs.size)
    beta = np.abs(Bs)
    res = stats.kstest(beta, lambda b: _beta_cdf(b, eta))
    assert res.pvalue > 1e-3, res


def test_sbx_pair_gate_rate(orc):
    p = _params(orc, d=8, N=4000, p_c=0.3)
    X1, X2 = _parents(p, 3)
    Xc = orc.sbx(p, 2, X1, X2)
    P = X1.shape[0]
    crossed = np.any(Xc[:P] != X1, axis=1)
    # a crossed pair keeps every variable with prob 2^-8 only
    assert abs(crossed.mean() - 0.3) < 5 * math.sqrt(0.3 * 0.7 / P)


def test_mutation_rate_zero_identity(orc):
    p = _params(orc, p_m=0.0)
    rng = np.random.default_rng(4)
    Xc = rng.uniform(0, 1, (p.N, p.d))
    Xm, mask = orc.mutation(p, 3, Xc)
    assert mask.sum() == 0
    assert np.array_equal(Xm, Xc)


def test_mutation_clips_into_box(orc):
    p = _params(orc, p_m=float(64))   # every site
    rng = np.random.default_rng(5)
    Xc = rng.uniform(-0.5, 1.5, (p.N, p.d))
    Xm, mask = orc.mutation(p, 3, Xc)
    assert mask.all()
    assert Xm.min() >= 0.0 and Xm.max() <= 1.0


def test_mutation_site_frequency(orc):
    p = _params(orc, d=50, N=2000)
    Xc = np.full((p.N, p.d), 0.5)
    _, mask = orc.mutation(p, 9, Xc)
    n = mask.size
    q = math.ceil((1 << 24) / 50) / (1 << 24)     # R4 < 1/d on the 24-bit grid
    k = int(mask.sum())
    assert stats.binomtest(k, n, q).pvalue > 1e-3
    assert abs(q - 1 / 50) < 1e-7


def _q24(p_m, d):
    """Per-site mutation probability p_m/d on the 24-bit grid."""
    return math.ceil((1 << 24) * p_m / d) / (1 << 24)


def test_mutation_subset_law(orc):
    """Appendix B draws one uniform per site, so the sites of a row are
    independent Bernoulli(q) events.  The oracle draws the count and then a
    uniform subset; on d = 4 every one of the 16 masks must appear with
    probability q^|S| (1-q)^(4-|S|)."""
    p = _params(orc, d=4, N=20000, p_m=1.6)
    _, mask = orc.mutation(p, 6, np.full((p.N, p.d), 0.5))
    q = _q24(1.6, 4)
    code = mask.astype(np.int64) @ (1 << np.arange(4))
    obs = np.bincount(code, minlength=16)
    size = np.array([bin(s).count("1") for s in range(16)])
    exp = p.N * q ** size * (1 - q) ** (4 - size)
    res = stats.chisquare(obs, exp)
    assert res.pvalue > 1e-3, (obs, exp)


def test_mutation_count_law(orc):
    """Row site counts follow Binomial(d, q)."""
    d, p_m = 300, 1.0
    p = _params(orc, d=d, N=20000, p_m=p_m)
    _, mask = orc.mutation(p, 8, np.full((p.N, p.d), 0.5))
    q = _q24(p_m, d)
    k = mask.sum(axis=1)
    obs = np.array([(k == i).sum() for i in range(5)] + [(k >= 5).sum()])
    pmf = stats.binom.pmf(np.arange(5), d, q)
    exp = p.N * np.append(pmf, 1 - pmf.sum())
    res = stats.chisquare(obs, exp)
    assert res.pvalue > 1e-3, (obs, exp)


def test_mutation_positions_uniform(orc):
    """Every position is equally likely to be a site (the subset step's draw
    ranges); a skew towards the last positions would show here."""
    d = 40
    p = _params(orc, d=d, N=20000, p_m=3.0)
    _, mask = orc.mutation(p, 2, np.full((p.N, p.d), 0.5))
    obs = mask.sum(axis=0)
    res = stats.chisquare(obs)
    assert res.pvalue > 1e-3, obs
    assert abs(obs.sum() / mask.size - _q24(3.0, d)) < 5 * math.sqrt(_q24(3.0, d) / mask.size)


def _pm_cdf(q, x, eta):
    """CDF of the mutation step (x' - x)/(U-L) of Deb's polynomial mutation
    at an interior x with U-L = 1, derived from the Appendix B formula with
    M uniform on [0, 1)."""
    q = np.asarray(q, dtype=np.float64)
    a = (1 - x) ** (eta + 1)      # (1 - delta1)^(eta+1), delta1 = x
    b = x ** (eta + 1)            # (1 - delta2)^(eta+1), delta2 = 1 - x
    neg = ((1 + q) ** (eta + 1) - a) / (2 * (1 - a))
    pos = 0.5 + (1 - (1 - q) ** (eta + 1)) / (2 * (1 - b))
    return np.clip(np.where(q < 0, neg, pos), 0, 1)


@pytest.mark.parametrize("x", [0.3, 0.85])
def test_mutation_step_distribution(orc, x):
    eta = 20.0
    p = _params(orc, d=100, N=400, p_m=100.0, eta_m=eta)
    Xc = np.full((p.N, p.d), x)
    Xm, mask = orc.mutation(p, 4, Xc)
    assert mask.all()
    steps = (Xm - x).ravel()
    res = stats.kstest(steps, lambda q: _pm_cdf(q, x, eta))
    assert res.pvalue > 1e-3, res
    assert steps.min() >= -x - 1e-12 and steps.max() <= 1 - x + 1e-12


def _hand_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "dtlz_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, b = line.split(";")
            a = a.split()
            prob, m, d = int(a[0]), int(a[1]), int(a[2])
            x = [float(v) for v in a[3:]]
            fx = [float(v) for v in b.split()]
            rows.append((prob, m, d, x, fx))
    return rows


def test_dtlz_hand_worked(orc):
    rows = _hand_rows()
    assert len(rows) == 7
    for prob, m, d, x, fx in rows:
        p = orc.make_params(m=m, d=d, N=1, H=0, problem=prob)
        F = orc.evaluate(p, np.array([x]))
        assert np.allclose(F[0], fx, rtol=1e-13, atol=1e-13), (prob, F[0], fx)


@pytest.mark.parametrize("m,d", [(2, 12), (3, 12), (5, 30), (3, 5000)])
def test_dtlz_fronts(orc, m, d):
    rng = np.random.default_rng(m * 1000 + d)
    X = np.full((64, d), 0.5)
    X[:, : m - 1] = rng.uniform(0, 1, (64, m - 1))     # g = 0: on the front
    F2 = orc.evaluate(orc.make_params(m=m, d=d, N=64, H=0, problem=orc.DTLZ2), X)
    assert np.allclose(np.linalg.norm(F2, axis=1), 1.0, rtol=0, atol=1e-15)
    F1 = orc.evaluate(orc.make_params(m=m, d=d, N=64, H=0, problem=orc.DTLZ1), X)
    # DTLZ1's g sums k terms of (0 - cos 0) = -1 on top of k: exact zero
    assert np.allclose(F1.sum(1), 0.5, rtol=0, atol=1e-12)
    # off the front, g > 0 raises every objective
    X2 = X.copy()
    X2[:, m - 1:] = 0.3
    assert (orc.evaluate(orc.make_params(m=m, d=d, N=64, H=0, problem=orc.DTLZ2), X2)
            >= F2 - 1e-15).all()


@pytest.mark.parametrize("m,d", [(2, 12), (3, 12), (5, 30), (3, 5000)])
def test_dtlz3_dtlz4_against_dtlz1_dtlz2(orc, m, d):
    """DTLZ3 is DTLZ2's unit-norm shape scaled by DTLZ1's 1 + g (DTLZ1's
    objectives sum to (1 + g)/2); DTLZ4 is DTLZ2 of x with the position
    variables raised to the 100th power; both fronts (x_m.. = 1/2) are the
    unit sphere."""
    rng = np.random.default_rng(m * 7919 + d)
    X = rng.uniform(0, 1, (64, d))
    X[:8, : m - 1] = rng.uniform(0.9, 1.0, (8, m - 1))   # where the 100th power is not tiny

    def ev(prob, x):
        return orc.evaluate(orc.make_params(m=m, d=d, N=64, H=0, problem=prob), x)
    F1, F2, F3, F4 = (ev(pr, X) for pr in (orc.DTLZ1, orc.DTLZ2, orc.DTLZ3, orc.DTLZ4))
    shape = F2 / np.linalg.norm(F2, axis=1, keepdims=True)
    assert np.allclose(F3, 2.0 * F1.sum(1, keepdims=True) * shape, rtol=1e-12, atol=0)
    Xp = X.copy()
    Xp[:, : m - 1] = X[:, : m - 1] ** 100
    assert np.allclose(F4, ev(orc.DTLZ2, Xp), rtol=1e-12, atol=1e-300)
    Xf = X.copy()
    Xf[:, m - 1:] = 0.5
    for prob in (orc.DTLZ3, orc.DTLZ4):
        assert np.allclose(np.linalg.norm(ev(prob, Xf), axis=1), 1.0, rtol=0, atol=1e-12)


def test_init_population(orc):
    p = _params(orc, d=13, N=105, H=13, seed=123)
    X = orc.init_population(p)
    assert X.min() >= 0.0 and X.max() < 1.0
    # 24-bit grid: exactly representable in float32
    assert np.array_equal(X.astype(np.float32).astype(np.float64), X)
    assert stats.kstest(X.ravel(), "uniform").pvalue > 1e-3
    # first word of individual 0 comes from counter (0, 0, 0, INIT)
    w = orc.philox([0, 0, 0, orc.TAG_INIT], [123, 0])
    assert X[0, 0] == (w[0] >> 8) / 2 ** 24 and X[0, 3] == (w[3] >> 8) / 2 ** 24


def test_mating_uniform_over_valid(orc):
    p = _params(orc, N=20000)
    vlist = np.array([2, 5, 6, 11], dtype=np.int32)
    par = orc.mating(p, 7, vlist)
    assert set(np.unique(par)) <= set(vlist.tolist())
    counts = np.array([(par == v).sum() for v in vlist])
    assert stats.chisquare(counts).pvalue > 1e-3
    # draw e uses word e % 4 of counter (e/4, 0, t, MATE) and (w*K) >> 32
    w = orc.philox([1, 0, 7, orc.TAG_MATE], [7, 0])
    assert par[5] == vlist[(w[1] * 4) >> 32]


def test_igd(orc):
    """IGD (Appendix C): zero when the population contains every reference
    point; a closed form for one reference point; invalid members ignored;
    a pure-Python brute force on a small random case."""
    R = np.array([[1.0, 0.0], [0.0, 1.0], [0.6, 0.8]])
    assert orc.igd(R, np.ones(3, np.uint8), R) == 0.0
    P = np.array([[3.0, 4.0], [100.0, 100.0]])
    assert orc.igd(P, np.array([1, 0], np.uint8), np.zeros((1, 2))) == 5.0
    assert orc.igd(P, np.array([1, 1], np.uint8), np.array([[97.0, 96.0]])) == 5.0
    with pytest.raises(ValueError):
        orc.igd(P, np.zeros(2, np.uint8), R)
    rng = np.random.default_rng(3)
    F = rng.uniform(0, 2, (7, 3))
    v = np.array([1, 0, 1, 1, 0, 1, 1], np.uint8)
    Rr = rng.uniform(0, 1, (5, 3))
    total = 0.0
    for r in Rr.tolist():
        best = None
        for f, ok in zip(F.tolist(), v.tolist()):
            if not ok:
                continue
            dist = sum((a - b) ** 2 for a, b in zip(r, f)) ** 0.5
            best = dist if best is None else min(best, dist)
        total += best
    assert abs(orc.igd(F, v, Rr) - total / len(Rr)) < 1e-14


def _hv_grid(points, ref):
    """Brute force on integer coordinates: the unit cells [a, a + 1) below
    ref that some point weakly dominates (p <= a in every objective)."""
    import itertools
    count = 0
    for a in itertools.product(*[range(int(r)) for r in ref]):
        if any(all(pk <= ak for pk, ak in zip(p, a)) for p in points):
            count += 1
    return count


def test_hypervolume(orc):
    """HV (Appendix C): one box; two boxes by inclusion-exclusion; members
    that do not dominate the reference point, or are invalid, add nothing;
    integer point sets against a brute-force count of unit cells (m = 2, 3)."""
    one = np.ones(1, np.uint8)
    assert orc.hypervolume(np.array([[1.0, 2.0, 0.5]]), one, [3.0, 3.0, 1.0]) == 2.0 * 1.0 * 0.5
    a, b, r = np.array([1.0, 3.0]), np.array([2.0, 1.0]), np.array([4.0, 4.0])
    inter = np.prod(r - np.maximum(a, b))
    assert abs(orc.hypervolume(np.stack([a, b]), np.ones(2, np.uint8), r)
               - (np.prod(r - a) + np.prod(r - b) - inter)) < 1e-15
    F = np.array([[1.0, 1.0], [5.0, 0.5], [0.5, 0.5]])
    assert orc.hypervolume(F, np.array([1, 1, 0], np.uint8), [4.0, 4.0]) == 9.0
    rng = np.random.default_rng(11)
    for m, ref in ((2, (7, 7)), (3, (5, 5, 5)), (3, (6, 4, 5))):
        for _ in range(6):
            n = int(rng.integers(1, 9))
            P = rng.integers(0, 6, (n, m)).astype(np.float64)
            v = rng.integers(0, 2, n).astype(np.uint8)
            v[0] = 1
            pts = [p for p, ok in zip(P.tolist(), v.tolist()) if ok]
            assert orc.hypervolume(P, v, ref) == _hv_grid(pts, ref), (P, v, ref)
