"""Pins of the oracle's environmental selection (Algorithm 1, Eqs. 2-5).

1. Brute force by the set definition on tiny populations, with angles taken
   from atan2(|a x b|, a.b) rather than arccos of a cosine.
2. The paper's masked-tensor formulation written literally in numpy
   (T_part, sgn, -1 -> inf, column argmin).
3. Invariants: one survivor per non-empty vector, survivors associated with
   their own vector, and the limits of the penalty term.
"""
import numpy as np
import pytest


def _angle(a, b):
    """Angle between two vectors of any length m, via a QR-free atan2."""
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 or nb == 0:
        return np.pi / 2
    u, v = a / na, b / nb
    s = np.linalg.norm(u - (u @ v) * v)     # |sin|
    return float(np.arctan2(s, u @ v))


def _brute(F, valid, V, t, t_max, alpha):
    n, m = F.shape
    r = V.shape[0]
    idx = [i for i in range(n) if valid[i]]
    z = F[idx].min(0)
    gam = []
    for j in range(r):
        gam.append(min(_angle(V[i], V[j]) for i in range(r) if i != j))
    subpop = {j: [] for j in range(r)}
    for i in idx:
        fp = F[i] - z
        angs = [_angle(fp, V[j]) for j in range(r)]
        j = int(np.argmin(angs))
        subpop[j].append((i, angs[j], np.linalg.norm(fp)))
    surv = []
    for j in range(r):
        if not subpop[j]:
            surv.append(-1)
            continue
        apd = [(1 + m * (t / t_max) ** alpha * th / gam[j]) * nf for (_, th, nf) in subpop[j]]
        surv.append(subpop[j][int(np.argmin(apd))][0])
    return np.array(surv), np.array(gam)


def _literal_alg1(F, V, gam, t, t_max, alpha):
    """Algorithm 1 as printed, on dense n x r tensors (all rows valid)."""
    n, m = F.shape
    r = V.shape[0]
    z = F.min(0)                                           # line 3
    Fp = F - np.repeat(z[None, :], n, 0)                   # line 4
    nF = np.linalg.norm(Fp, axis=1, keepdims=True)
    nV = np.linalg.norm(V, axis=1, keepdims=True)
    cos = (Fp @ V.T) / (nF * nV.T)                         # line 5
    Theta = np.arccos(np.clip(cos, -1, 1))
    A = np.repeat(np.argmin(Theta, 1)[:, None], r, 1)      # line 6 (Eq. 2)
    Tpart = np.repeat(np.arange(n)[:, None], r, 1)         # line 7
    I = np.repeat(np.arange(r)[None, :], n, 0)             # line 8
    S = np.abs(np.sign(A - I))
    Tpart = (1 - S) * Tpart - S                            # line 9 (Eq. 3)
    TAPD = np.empty((n, r))
    for j in range(r):                                     # lines 11-13 (Eq. 4)
        tp = Tpart[:, j]
        th = Theta[tp, j]
        TAPD[:, j] = (1 + m * (t / t_max) ** alpha * th / gam[j]) * nF[tp, 0]
    TAPD[Tpart == -1] = np.inf                             # line 14
    Inext = np.argmin(TAPD, 0)                             # line 15
    empty = np.isinf(TAPD).all(0)
    Inext[empty] = -1                                      # invalid slots
    return Inext


def _case(seed, n, r, m):
    rng = np.random.default_rng(seed)
    F = rng.uniform(0.0, 3.0, (n, m)) ** 2
    V = np.abs(rng.normal(size=(r, m)))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    return F, V


@pytest.mark.parametrize("seed", range(12))
def test_select_brute_force(orc, seed):
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(2, 5))
    n = int(rng.integers(2, 13))
    r = int(rng.integers(2, 7))
    F, V = _case(seed, n, r, m)
    valid = (rng.uniform(size=n) > 0.2).astype(np.uint8)
    valid[0] = 1
    t, t_max, alpha = int(rng.integers(1, 10)), 10, 2.0
    gam = orc.gamma(V)
    want, gam_bf = _brute(F, valid, V, t, t_max, alpha)
    assert np.allclose(gam, gam_bf, rtol=1e-9)
    got = orc.select(F, valid, V, gam, t, t_max, alpha)
    assert np.array_equal(got["survivor"], want)


@pytest.mark.parametrize("seed", range(8))
def test_select_matches_literal_algorithm(orc, seed):
    F, V = _case(1000 + seed, 40, 9, 3)
    gam = orc.gamma(V)
    for t in (1, 5, 10):
        got = orc.select(F, np.ones(40, np.uint8), V, gam, t, 10, 2.0)
        want = _literal_alg1(F, V, gam, t, 10, 2.0)
        assert np.array_equal(got["survivor"], want)


def test_select_invariants(orc):
    K = orc.lattice(3, 13)
    V = orc.lattice_unit(K)
    gam = orc.gamma(V)
    rng = np.random.default_rng(5)
    F = rng.uniform(0, 1, (210, 3))
    valid = np.ones(210, np.uint8)
    valid[::7] = 0
    out = orc.select(F, valid, V, gam, 30, 100, 2.0)
    surv, assoc = out["survivor"], out["assoc"]
    alive = surv[surv >= 0]
    assert len(set(alive.tolist())) == len(alive)                 # at most one each
    assert all(valid[i] for i in alive)                           # survivors in S
    assert all(assoc[surv[j]] == j for j in range(len(V)) if surv[j] >= 0)
    nonempty = set(assoc[assoc >= 0].tolist())
    assert set(np.nonzero(surv >= 0)[0].tolist()) == nonempty
    assert (assoc[valid == 0] == -1).all()
    assert np.allclose(out["zstar"], F[valid == 1].min(0))


def test_select_zero_penalty_keeps_closest(orc):
    # t/t_max -> 0 (alpha large): APD -> ||f'||, the survivor is the member
    # of each subpopulation nearest to z*
    F, V = _case(77, 60, 7, 3)
    gam = orc.gamma(V)
    out = orc.select(F, None, V, gam, 1, 10, 200.0)
    nf = np.linalg.norm(F - F.min(0), axis=1)
    for j, s in enumerate(out["survivor"]):
        members = np.nonzero(out["assoc"] == j)[0]
        if len(members):
            assert s == members[np.argmin(nf[members])]


def test_select_ideal_point_solution(orc):
    # a solution equal to z*: cosines read as 0, vector 0, theta pi/2, APD 0
    F = np.array([[0.0, 0.0], [1.0, 0.2], [0.3, 2.0]])
    V = np.array([[1.0, 0.0], [0.0, 1.0], [0.7071067811865476, 0.7071067811865476]])
    gam = orc.gamma(V)
    out = orc.select(F, None, V, gam, 3, 10, 2.0)
    assert out["assoc"][0] == 0 and out["apd"][0] == 0.0
    assert np.isclose(out["theta"][0], np.pi / 2)
    assert out["survivor"][0] == 0
