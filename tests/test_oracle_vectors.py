"""Pins of the oracle's reference-vector code: lattice, gamma (Eq. 5) and the
adaptation step of Algorithm 2.

Anchors: the lattice count C(H+m-1, m-1), the simplex constraint, the
closed-form neighbour angles of the m = 2 lattice, angles recomputed with
atan2(|a x b|, a.b) instead of arccos, and the invariances of the rescaling.
"""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("m,H,N", [(3, 13, 105), (3, 139, 9870), (2, 99, 100),
                                   (5, 5, 126), (10, 3, 220), (3, 19, 210), (2, 1, 2)])
def test_lattice_count(orc, m, H, N):
    assert orc.lattice_count(m, H) == N == math.comb(H + m - 1, m - 1)


@pytest.mark.parametrize("m,H", [(3, 13), (2, 99), (5, 5), (10, 3), (4, 7)])
def test_lattice_rows(orc, m, H):
    K = orc.lattice(m, H)
    assert K.shape == (math.comb(H + m - 1, m - 1), m)
    assert (K >= 0).all() and (K.sum(1) == H).all()
    assert len({tuple(r) for r in K}) == len(K)
    # lexicographic order of the leading m-1 coordinates
    lead = [tuple(r[:-1]) for r in K]
    assert lead == sorted(lead)


@pytest.mark.parametrize("m,H", [(3, 13), (3, 139), (2, 99), (10, 3)])
def test_unit_vectors(orc, m, H):
    K = orc.lattice(m, H)
    V = orc.lattice_unit(K)
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, rtol=0, atol=4e-16)
    # direction of k: V * ||k|| == k
    nk = np.sqrt((K.astype(np.float64) ** 2).sum(1, keepdims=True))
    assert np.allclose(V * nk, K, rtol=0, atol=1e-12)


def test_gamma_m2_closed_form(orc):
    H = 99
    V = orc.lattice_unit(orc.lattice(2, H))
    g = orc.gamma(V)
    k = np.arange(H + 1)
    phi = np.arctan2(H - k, k)               # polar angle of (k, H-k)
    gaps = np.abs(np.diff(phi))
    expect = np.empty(H + 1)
    expect[0] = gaps[0]
    expect[-1] = gaps[-1]
    expect[1:-1] = np.minimum(gaps[:-1], gaps[1:])
    # arccos of a cosine near 1 loses ~eps/sin(theta): 1e-10 relative at theta ~ 0.01
    assert np.allclose(g, expect, rtol=1e-10, atol=0)


def _gamma_atan2(V):
    r = len(V)
    out = np.empty(r)
    for j in range(r):
        c = V @ V[j]
        s = np.linalg.norm(np.cross(V, V[j]), axis=1)
        a = np.arctan2(s, c)
        a[j] = np.inf
        out[j] = a.min()
    return out


def test_gamma_m3_atan2(orc):
    V = orc.lattice_unit(orc.lattice(3, 13))
    assert np.allclose(orc.gamma(V), _gamma_atan2(V), rtol=1e-9, atol=0)
    # a rescaled (adapted) set as well
    W = orc.adapt(V, np.array([3.0, 0.5, 1.7]))
    assert np.allclose(orc.gamma(W), _gamma_atan2(W), rtol=1e-9, atol=0)


def test_adapt_identity_and_norm(orc):
    V0 = orc.lattice_unit(orc.lattice(3, 13))
    assert np.allclose(orc.adapt(V0, np.ones(3)), V0, rtol=0, atol=2e-16)
    rng = np.array([2.0, 0.25, 7.0])
    V = orc.adapt(V0, rng)
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, rtol=0, atol=4e-16)
    # V_j parallel to V0_j * range: cross product vanishes
    W = V0 * rng
    assert np.allclose(np.linalg.norm(np.cross(V, W), axis=1), 0, atol=1e-14)
    assert (np.einsum("ij,ij->i", V, W) > 0).all()


def test_adapt_scale_invariant(orc):
    V0 = orc.lattice_unit(orc.lattice(3, 19))
    rng = np.array([2.0, 0.25, 7.0])
    V1 = orc.adapt(V0, rng)
    V2 = orc.adapt(V0, rng * 1024.0)      # power of two: exact scaling
    assert np.array_equal(V1, V2)
    assert np.allclose(orc.gamma(V1), orc.gamma(orc.adapt(V0, rng * 3.3)), rtol=1e-12)


def test_adapt_zero_range_floor(orc):
    V0 = orc.lattice_unit(orc.lattice(3, 13))
    V = orc.adapt(V0, np.array([1.0, 0.0, 1.0]))
    assert np.isfinite(V).all()
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=4e-16)
    # a collapsed axis keeps only a 1e-12 share, unless it is the only non-zero one
    other = (V0[:, 0] > 0) | (V0[:, 2] > 0)
    assert np.abs(V[other, 1]).max() <= 12e-12 * (1 + 1e-9)   # k2 <= 12 vs k1 >= 1
    assert np.allclose(V[~other], [[0.0, 1.0, 0.0]])


def test_objective_range(orc):
    F = np.array([[1.0, 5.0], [3.0, -1.0], [100.0, 100.0]])
    assert np.array_equal(orc.objective_range(F, np.array([1, 1, 0])), [2.0, 6.0])


def test_lattice_for_population_size(orc):
    """A population size n that is not a lattice size maps to the largest
    lattice with at most n points: the paper's sweep sizes n = 2^5 .. 2^14
    (m = 3) and n = 100, pinned by the count formula on both sides of H and
    by hand-counted cases (C(8,2) = 28 <= 32 < 36 = C(9,2), C(14,2) = 91 <=
    100 < 105)."""
    from math import comb
    assert orc.lattice_for(3, 32) == 6 and comb(8, 2) == 28
    assert orc.lattice_for(3, 100) == 12 and comb(14, 2) == 91
    assert orc.lattice_for(3, 105) == 13
    assert orc.lattice_for(2, 100) == 99
    assert orc.lattice_for(3, 2) == -1
    for m in (2, 3, 5):
        for n in [2 ** k for k in range(5, 15)] + [100, 9870, 9871]:
            H = orc.lattice_for(m, n)
            if H < 0:
                assert comb(m, m - 1) > n
                continue
            assert comb(H + m - 1, m - 1) <= n < comb(H + m, m - 1)
