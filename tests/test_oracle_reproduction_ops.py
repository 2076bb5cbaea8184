"""Pins of the oracle's alternative reproduction operators (the extensibility
experiment, Sec. 4.4 / Appendix C): random reproduction, DE/rand/1/bin, CSO and PSO.
Each pin checks a property the published operator fixes, independently of
the oracle's own arithmetic."""
import itertools

import numpy as np
import pytest


def _p(orc, **kw):
    base = dict(m=3, d=6, N=8, H=0, problem=orc.DTLZ2, t_max=100, seed=3)
    base.update(kw)
    return orc.make_params(**base)


def test_random_offspring(orc):
    """Uniform on the box, on the 24-bit grid, a different draw per
    generation, the same on a repeat."""
    p = _p(orc, N=500, d=40)
    X = orc.random_offspring(p, 5)
    assert X.shape == (500, 40) and X.min() >= 0.0 and X.max() < 1.0
    assert np.array_equal(X * 2**24, np.floor(X * 2**24))
    n = X.size
    assert abs(X.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(X.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    assert np.array_equal(X, orc.random_offspring(p, 5))
    assert not np.array_equal(X, orc.random_offspring(p, 6))
    pb = _p(orc, N=50, d=10, L=-1.0, U=1.0)
    Xb = orc.random_offspring(pb, 1)
    assert Xb.min() >= -1.0 and Xb.max() < 1.0


def test_de_picks_distinct_and_uniform(orc):
    """r1, r2, r3 are distinct and differ from the target; as an ordered
    triple over the other K - 1 positions they are uniform (chi-square over
    the 24 triples of K = 5); j_rand is uniform over the d variables."""
    p = _p(orc, d=7)
    K, n = 5, 24000
    counts = {}
    jr = np.zeros(7)
    for o in range(n):
        tpos, a, b, c, j = orc.de_picks(p, 2, K, o)
        assert tpos == o % K
        assert len({tpos, a, b, c}) == 4 and all(0 <= q < K for q in (a, b, c))
        others = [q for q in range(K) if q != tpos]
        key = (others.index(a), others.index(b), others.index(c))
        counts[key] = counts.get(key, 0) + 1
        jr[j] += 1
    assert len(counts) == 24
    e = n / 24
    chi2 = sum((v - e) ** 2 / e for v in counts.values())
    assert chi2 < 80, chi2          # 23 degrees of freedom; p ~ 1e-7 at 80
    e7 = n / 7
    assert sum((v - e7) ** 2 / e7 for v in jr) < 45   # 6 degrees of freedom
    # fewer than four valid members: with replacement, in range
    for o in range(200):
        tpos, a, b, c, _ = orc.de_picks(p, 2, 3, o)
        assert all(0 <= q < 3 for q in (tpos, a, b, c))


def test_de_offspring_special_cases(orc):
    """F = 0, CR = 1: every offspring is its base vector x_r1.  CR = 0: only
    variable j_rand leaves the target.  Invalid members (absent from the
    valid list) are never used.  The CR coin fires at rate CR."""
    rng = np.random.default_rng(7)
    p = _p(orc, N=12, d=9)
    X = rng.uniform(0, 1, (12, 9))
    vlist = np.array([0, 2, 3, 5, 7, 8, 11])
    U0 = orc.de_offspring(p, 4, X, vlist, F=0.0, CR=1.0)
    for o in range(12):
        _, a, _, _, _ = orc.de_picks(p, 4, len(vlist), o)
        assert np.array_equal(U0[o], X[vlist[a]])
    valid_rows = {tuple(X[v]) for v in vlist}
    assert all(tuple(u) in valid_rows for u in U0)
    Uc = orc.de_offspring(p, 4, X, vlist, F=0.5, CR=0.0)
    for o in range(12):
        tpos, a, b, c, j = orc.de_picks(p, 4, len(vlist), o)
        xt = X[vlist[tpos]]
        keep = np.arange(9) != j
        assert np.array_equal(Uc[o][keep], xt[keep])
        v = X[vlist[a], j] + 0.5 * (X[vlist[b], j] - X[vlist[c], j])
        assert Uc[o, j] == min(max(v, 0.0), 1.0)
    pw = _p(orc, N=40, d=400)
    Xw2 = rng.uniform(0.25, 0.75, (40, 400))   # inside the box: only taken variables change
    U = orc.de_offspring(pw, 1, Xw2, np.arange(40), F=0.5, CR=0.3)
    taken = 0
    total = 0
    for o in range(40):
        tpos, a, b, c, j = orc.de_picks(pw, 1, 40, o)
        diff = U[o] != Xw2[tpos]
        diff[j] = False
        taken += diff.sum()
        total += 399
    rate = taken / total
    assert abs(rate - 0.3) < 5 * np.sqrt(0.3 * 0.7 / total), rate


def test_de_offspring_brute_force(orc):
    """CR = 1: every offspring is clip(x_a + F (x_b - x_c)) for an ordered
    triple of distinct members other than its target (o mod K), found by
    trying all of them."""
    rng = np.random.default_rng(9)
    N, d, F = 6, 5, 0.7
    p = _p(orc, N=N, d=d)
    X = rng.uniform(0, 1, (N, d))
    U = orc.de_offspring(p, 3, X, np.arange(N), F=F, CR=1.0)
    for o in range(N):
        t = o % N
        cands = [q for q in range(N) if q != t]
        ok = any(np.array_equal(U[o], np.clip(X[a] + F * (X[b] - X[c]), 0.0, 1.0))
                 for a, b, c in itertools.permutations(cands, 3))
        assert ok, o


@pytest.mark.parametrize("K", [1, 2])
def test_de_offspring_tiny_valid_lists(orc, K):
    """With fewer than four valid members the draws repeat members; with one,
    every offspring is that member."""
    p = _p(orc, N=5, d=4)
    X = np.random.default_rng(1).uniform(0, 1, (5, 4))
    vlist = np.arange(K) + 1
    U = orc.de_offspring(p, 1, X, vlist, F=0.5, CR=0.9)
    assert np.isfinite(U).all() and U.min() >= 0 and U.max() <= 1
    if K == 1:
        assert (U == X[1]).all()


@pytest.mark.parametrize("op", [1, 2])
def test_generation_uses_the_operator(orc, op):
    """A generation with the DE (op 1) or random (op 2) operator makes its
    offspring with that operator (the same rows as the operator called alone
    on the generation's population and valid list), evaluates them and
    selects as the SBX generation does."""
    p = orc.make_params(m=3, d=9, N=105, H=13, problem=orc.DTLZ1, t_max=20, seed=4, op=op,
                        de_F=0.7, de_CR=0.6)
    V0, st = orc.initial_state(p)
    st.valid[[3, 17, 40]] = 0
    X, vlist = st.X.copy(), np.nonzero(st.valid)[0]
    t = st.t
    out = orc.generation(p, V0, st)
    want = orc.de_offspring(p, t, X, vlist, 0.7, 0.6) if op == 1 else orc.random_offspring(p, t)
    assert np.array_equal(out["Xchild"], want)
    assert np.array_equal(out["Fchild"], orc.evaluate(p, want, t))
    assert (out["parents"] == -1).all()
    assert (out["survivor"] >= -1).all() and (np.bincount(out["survivor"][out["survivor"] >= 0]) <= 1).all()


# ---- the competitive swarm optimizer (CSO; Cheng and Jin 2015) -----------

def test_cso_picks_distinct_and_uniform(orc):
    """Two distinct positions of the valid list, every ordered pair about
    equally often; a one-member list meets itself."""
    p = _p(orc)
    K, n = 5, 20000
    counts = np.zeros((K, K), dtype=int)
    for o in range(n):
        a, b = orc.cso_picks(p, 3, K, o)
        assert 0 <= a < K and 0 <= b < K and a != b
        counts[a, b] += 1
    off = counts[~np.eye(K, dtype=bool)]
    exp = n / (K * (K - 1))
    assert ((off - exp) ** 2 / exp).sum() < 60   # chi-square, 19 dof
    assert orc.cso_picks(p, 3, 1, 7) == (0, 0)


def _competition(orc, p, t, o, vlist, apd):
    a, b = orc.cso_picks(p, t, len(vlist), o)
    ia, ib = vlist[a], vlist[b]
    w = ia if (apd[ia] < apd[ib] or (apd[ia] == apd[ib] and ia <= ib)) else ib
    return w, (ib if w == ia else ia)


def test_cso_loser_moves_towards_winner(orc):
    """With zero velocities and phi = 0 (a first generation), the loser's new
    position lies on the segment to the winner, coordinate by coordinate, its
    velocity is the displacement, and across many variables it covers the
    segment uniformly (mean 1/2 of the way)."""
    p = _p(orc, N=40, d=500, cso_phi=0.0)
    rng = np.random.default_rng(1)
    X = rng.uniform(size=(40, 500))
    apd = rng.uniform(size=40)
    vlist = np.arange(40)
    Xo, Vo = orc.cso_offspring(p, 2, X, np.zeros_like(X), apd, vlist, X.mean(0))
    fr = []
    for o in range(40):
        w, l = _competition(orc, p, 2, o, vlist, apd)
        lo, hi = np.minimum(X[w], X[l]), np.maximum(X[w], X[l])
        assert (Xo[o] >= lo - 1e-15).all() and (Xo[o] <= hi + 1e-15).all()
        assert np.allclose(Vo[o], Xo[o] - X[l], atol=1e-15)
        span = X[w] - X[l]
        ok = np.abs(span) > 1e-3
        fr.append(((Xo[o] - X[l])[ok] / span[ok]))
    fr = np.concatenate(fr)
    assert abs(fr.mean() - 0.5) < 5 * np.sqrt(1 / 12 / fr.size)
    assert fr.min() >= 0.0 and fr.max() < 1.0


def test_cso_winner_rule_and_velocity_term(orc):
    """The smaller APD wins, ties to the smaller index (all +inf before any
    selection); with the positions equal, the update is r1 v alone: every
    coordinate of the new velocity is a fraction in [0, 1) of the old one,
    of mean 1/2."""
    p = _p(orc, N=64, d=300, cso_phi=0.0)
    X = np.full((64, 300), 0.5)
    Vel = np.random.default_rng(2).uniform(-0.2, 0.2, size=(64, 300))
    apd = np.full(64, np.inf)
    vlist = np.arange(64)
    Xo, Vo = orc.cso_offspring(p, 5, X, Vel, apd, vlist, X.mean(0))
    ratios = []
    for o in range(64):
        w, l = _competition(orc, p, 5, o, vlist, apd)
        a, b = orc.cso_picks(p, 5, 64, o)
        assert l == max(a, b)          # ties: the smaller index wins
        r = Vo[o] / Vel[l]
        assert (r >= 0).all() and (r < 1).all()
        assert np.allclose(Xo[o], np.clip(0.5 + Vo[o], 0, 1), atol=1e-15)
        ratios.append(r)
    r = np.concatenate(ratios)
    assert abs(r.mean() - 0.5) < 5 * np.sqrt(1 / 12 / r.size)


def test_cso_centre_term_and_clip(orc):
    """phi pulls the loser towards the swarm centre: with winner = loser (one
    member) and zero velocity, x' = x + phi r3 (xbar - x), clipped to the
    box."""
    p = _p(orc, N=1, d=400, cso_phi=0.3, L=0.0, U=1.0)
    X = np.random.default_rng(3).uniform(size=(1, 400))
    xbar = np.full(400, 0.9)
    Xo, Vo = orc.cso_offspring(p, 1, X, np.zeros_like(X), np.zeros(1), np.array([0]), xbar)
    frac = Vo[0] / (0.3 * (xbar - X[0]))
    assert (frac >= 0).all() and (frac < 1).all()
    assert abs(frac.mean() - 0.5) < 5 * np.sqrt(1 / 12 / 400)
    assert np.array_equal(Xo[0], np.clip(X[0] + Vo[0], 0.0, 1.0))


def test_generation_with_cso_keeps_the_swarm_state(orc):
    """A CSO generation makes its offspring with the operator (from the
    population, its velocities, the kept APDs and the swarm centre), and the
    survivors carry their velocities and the APD that kept them."""
    p = orc.make_params(m=3, d=9, N=105, H=13, problem=orc.DTLZ1, t_max=20, seed=4,
                        op=orc.OP_CSO, cso_phi=0.2)
    V0, st = orc.initial_state(p)
    orc.generation(p, V0, st)               # every member gets an APD
    st.valid[[3, 17, 40]] = 0
    X, Vel, apd, vlist = st.X.copy(), st.vel.copy(), st.apd.copy(), np.nonzero(st.valid)[0]
    t = st.t
    F_old, valid_old, V_t, g_t = st.F.copy(), st.valid.copy(), st.V.copy(), st.gamma.copy()
    out = orc.generation(p, V0, st)
    want_x, want_v = orc.cso_offspring(p, t, X, Vel, apd, vlist, X[vlist].mean(0))
    assert np.allclose(out["Xchild"], want_x, rtol=0, atol=1e-12)
    assert (out["parents"] == -1).all()
    # the APDs the survivors were kept with: the selection's, recomputed
    sel = orc.select(np.concatenate([np.nan_to_num(F_old), out["Fchild"]]),
                     np.concatenate([valid_old, np.ones(p.N, np.uint8)]), V_t, g_t, t,
                     p.t_max, p.alpha)
    for j in range(p.N):
        i = out["survivor"][j]
        if i < 0:
            assert not st.valid[j] and np.isinf(st.apd[j])
            continue
        src_v = Vel[i] if i < p.N else want_v[i - p.N]
        assert np.allclose(st.vel[j], src_v, rtol=0, atol=1e-12)
        assert st.apd[j] == sel["apd"][i]


# ---- PSO (inertia-weight particle swarm with MOPSO personal bests) ---------

def _leader(orc, p, t, o, vlist, apd):
    _, a, b = orc.pso_picks(p, t, len(vlist), o)
    ia, ib = vlist[a], vlist[b]
    return ia if (apd[ia] < apd[ib] or (apd[ia] == apd[ib] and ia <= ib)) else ib


def test_pso_picks(orc):
    """The particle of offspring o is position o mod K; the two leader
    candidates are distinct and, as an ordered pair, uniform (chi-square over
    the 20 pairs of K = 5); with K = 1 the member is its own leader."""
    p = _p(orc)
    K, n = 5, 20000
    counts = np.zeros((K, K))
    for o in range(n):
        q, a, b = orc.pso_picks(p, 2, K, o)
        assert q == o % K and a != b and 0 <= a < K and 0 <= b < K
        counts[a, b] += 1
    off = counts[~np.eye(K, dtype=bool)]
    exp = n / (K * (K - 1))
    assert ((off - exp) ** 2 / exp).sum() < 60   # chi-square, 19 dof
    assert orc.pso_picks(p, 3, 1, 7) == (0, 0, 0)


def test_pso_inertia_and_still_swarm(orc):
    """With c1 = c2 = 0 the velocity is w v exactly and the position x + w v
    clipped; with w = 0 as well the particle stays where it is."""
    rng = np.random.default_rng(4)
    X = rng.uniform(size=(30, 200))
    Vel = rng.uniform(-0.3, 0.3, size=(30, 200))
    Pb = rng.uniform(size=(30, 200))
    apd = rng.uniform(size=30)
    vlist = np.arange(30)
    p = _p(orc, N=30, d=200, pso_w=0.6, pso_c1=0.0, pso_c2=0.0)
    Xo, Vo = orc.pso_offspring(p, 3, X, Vel, Pb, apd, vlist)
    for o in range(30):
        assert np.array_equal(Vo[o], 0.6 * Vel[o])
        assert np.array_equal(Xo[o], np.clip(X[o] + 0.6 * Vel[o], 0.0, 1.0))
    p0 = _p(orc, N=30, d=200, pso_w=0.0, pso_c1=0.0, pso_c2=0.0)
    Xo, Vo = orc.pso_offspring(p0, 3, X, Vel, Pb, apd, vlist)
    assert np.array_equal(Xo, X) and not Vo.any()


@pytest.mark.parametrize("term", ["cognitive", "social"])
def test_pso_attraction_terms(orc, term):
    """One attraction at a time, from rest: the particle moves towards its
    personal best (c1) or its leader (c2), the winner of the APD tournament,
    by c r (target - x) with r uniform in [0, 1), mean 1/2, per variable."""
    c1, c2 = (1.3, 0.0) if term == "cognitive" else (0.0, 1.3)
    p = _p(orc, N=40, d=400, pso_w=0.0, pso_c1=c1, pso_c2=c2, L=-10.0, U=10.0)
    rng = np.random.default_rng(5)
    X = rng.uniform(size=(40, 400))
    Pb = rng.uniform(size=(40, 400))
    apd = rng.uniform(size=40)
    vlist = np.arange(40)
    Xo, Vo = orc.pso_offspring(p, 6, X, np.zeros_like(X), Pb, apd, vlist)
    fr = []
    for o in range(40):
        tgt = Pb[o] if term == "cognitive" else X[_leader(orc, p, 6, o, vlist, apd)]
        span = 1.3 * (tgt - X[o])
        assert np.allclose(Vo[o], Xo[o] - X[o], atol=1e-15)
        ok = np.abs(span) > 1e-3
        r = (Xo[o] - X[o])[ok] / span[ok]
        assert (r >= -1e-12).all() and (r < 1.0).all()
        fr.append(r)
    fr = np.concatenate(fr)
    assert abs(fr.mean() - 0.5) < 5 * np.sqrt(1 / 12 / fr.size)


def test_pso_personal_best_rule(orc):
    """The offspring's personal best is its new position unless the
    particle's old best dominates it: dominated -> the old best (with its
    objectives); dominating, incomparable or equal -> the new position."""
    p = _p(orc, m=2, N=4, d=3)
    vlist = np.arange(4)
    Pb = np.arange(12, dtype=float).reshape(4, 3)
    Xc = -np.arange(12, dtype=float).reshape(4, 3)
    FPb = np.array([[1.0, 1.0], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0]])
    Fc = np.array([[2.0, 1.0],     # dominated by the old best
                   [0.5, 1.0],     # dominates it
                   [0.5, 2.0],     # incomparable
                   [1.0, 1.0]])    # equal
    Po, FPo = orc.pso_pbest(p, 1, vlist, Pb, FPb, Xc, Fc)
    assert np.array_equal(Po[0], Pb[0]) and np.array_equal(FPo[0], FPb[0])
    for o in (1, 2, 3):
        assert np.array_equal(Po[o], Xc[o]) and np.array_equal(FPo[o], Fc[o])


def test_generation_with_pso_keeps_the_swarm_state(orc):
    """A PSO generation makes its offspring with the operator (from the
    population, velocities, personal bests and kept APDs), and the survivors
    carry their velocities, personal bests (with objectives) and APDs."""
    p = orc.make_params(m=3, d=9, N=105, H=13, problem=orc.DTLZ1, t_max=20, seed=4,
                        op=orc.OP_PSO)
    V0, st = orc.initial_state(p)
    assert np.array_equal(st.pbest, st.X) and np.array_equal(st.fpbest, st.F)
    orc.generation(p, V0, st)
    st.valid[[3, 17, 40]] = 0
    X, Vel, Pb, FPb, apd = st.X.copy(), st.vel.copy(), st.pbest.copy(), st.fpbest.copy(), st.apd.copy()
    vlist = np.nonzero(st.valid)[0]
    t = st.t
    out = orc.generation(p, V0, st)
    want_x, want_v = orc.pso_offspring(p, t, X, Vel, Pb, apd, vlist)
    assert np.allclose(out["Xchild"], want_x, rtol=0, atol=1e-12)
    want_p, want_fp = orc.pso_pbest(p, t, vlist, Pb, FPb, want_x, out["Fchild"])
    for j in range(p.N):
        i = out["survivor"][j]
        if i < 0:
            continue
        if i < p.N:
            assert np.array_equal(st.vel[j], Vel[i]) and np.array_equal(st.pbest[j], Pb[i])
            assert np.array_equal(st.fpbest[j], FPb[i])
        else:
            c = i - p.N
            assert np.allclose(st.vel[j], want_v[c], atol=1e-12)
            assert np.allclose(st.pbest[j], want_p[c], atol=1e-12)
            assert np.allclose(st.fpbest[j], want_fp[c], atol=1e-12)


def test_cso_draws_are_distinct_per_term(orc):
    """r1, r2 and r3 of the same offspring and variable are different
    uniforms: each is read off its term alone (one member: the velocity term;
    two members a unit apart with zero velocity: the winner term; the centre
    term with phi), and the three are pairwise uncorrelated."""
    d, t, o_n = 400, 3, 8
    # r1: one member (winner = loser), unit velocity, phi = 0 -> v' = r1
    p1 = _p(orc, N=o_n, d=d, cso_phi=0.0, L=-10.0, U=10.0)
    X1 = np.zeros((1, d))
    _, V1 = orc.cso_offspring(p1, t, X1, np.ones((1, d)), np.zeros(1), np.array([0]), X1[0])
    # r2: two members a unit apart, zero velocity -> |v'| = r2
    p2 = _p(orc, N=o_n, d=d, cso_phi=0.0, L=-10.0, U=10.0)
    X2 = np.stack([np.zeros(d), np.ones(d)])
    _, V2 = orc.cso_offspring(p2, t, X2, np.zeros((2, d)), np.array([1.0, 2.0]),
                              np.array([0, 1]), X2.mean(0))
    # r3: one member, zero velocity, centre a unit away, phi = 1 -> v' = r3
    p3 = _p(orc, N=o_n, d=d, cso_phi=1.0, L=-10.0, U=10.0)
    _, V3 = orc.cso_offspring(p3, t, X1, np.zeros((1, d)), np.zeros(1), np.array([0]),
                              np.ones(d))
    r1, r2, r3 = V1.ravel(), np.abs(V2).ravel(), V3.ravel()
    for r in (r1, r2, r3):
        assert r.min() >= 0.0 and r.max() < 1.0
        assert abs(r.mean() - 0.5) < 5 * np.sqrt(1 / 12 / r.size)
    bound = 5 / np.sqrt(r1.size)
    for a, b in ((r1, r2), (r1, r3), (r2, r3)):
        assert not np.array_equal(a, b)
        assert abs(np.corrcoef(a, b)[0, 1]) < bound


def test_pso_draws_are_distinct_per_term(orc):
    """PSO's r1 (personal best) and r2 (leader) of the same offspring and
    variable are different uniforms: each is read off its term alone, and the
    two are uncorrelated."""
    d, t, n = 400, 4, 8
    # r1: w = c2 = 0, zero velocity, personal best a unit away -> v' = r1
    p1 = _p(orc, N=n, d=d, pso_w=0.0, pso_c1=1.0, pso_c2=0.0, L=-10.0, U=10.0)
    X = np.stack([np.ones(d), np.zeros(d)])   # member 0 (apd 1) leads, member 1 follows
    Z = np.zeros((2, d))
    _, V1 = orc.pso_offspring(p1, t, X, Z, X + 1.0, np.array([1.0, 2.0]), np.array([0, 1]))
    # r2: w = c1 = 0, zero velocity; the odd offspring move member 1 towards
    # member 0, a unit away -> v' = r2
    p2 = _p(orc, N=n, d=d, pso_w=0.0, pso_c1=0.0, pso_c2=1.0, L=-10.0, U=10.0)
    _, V2 = orc.pso_offspring(p2, t, X, Z, X, np.array([1.0, 2.0]), np.array([0, 1]))
    assert not V2[0::2].any()                 # member 0 is its own leader
    r1, r2 = V1[1::2].ravel(), V2[1::2].ravel()
    for r in (r1, r2):
        assert r.min() >= 0.0 and r.max() < 1.0
        assert abs(r.mean() - 0.5) < 5 * np.sqrt(1 / 12 / r.size)
    assert not np.array_equal(r1, r2)
    assert abs(np.corrcoef(r1, r2)[0, 1]) < 5 / np.sqrt(r1.size)
