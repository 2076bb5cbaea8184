"""Shared helpers of the GPU parity tests (comparison rules and run set-up).

Tolerances (stated once, used everywhere):
  * rollout objectives (BF16 policy GEMMs): 1e-2 of max(|f|, median |f_k|);
  * random words, masks, mating indices, lattice, initial population: exact;
  * decision variables: |x_gpu - x_orc| <= 1e-5 (U - L)   (float32 SBX/PM);
  * objectives: |f_gpu - f_orc| <= 1e-5 ||f_orc||_2 per row (relative to the
    row's objective vector, so components that vanish on the front are not
    held to a relative bound they cannot carry);
  * gamma (FP64): |g_gpu - g_orc| <= 64 eps / sin(g) + 1e-12 g: arccos of a
    cosine near 1 loses eps / sin(theta) (theta ~ 1e-3 rad at N = 9870);
  * association: exact unless the two vectors' dot products with f' differ
    by less than `tie_rel` ||f'|| = 1e-6 ||f'|| (float32 dots of unit vectors:
    each carries at most ~m 2^-24 ||f'|| of rounding, plus the float32
    rounding of the vector, ~2^-24 per component);
  * survivors: exact unless explained by such an association tie or by two
    APD values within 1e-5 relative.
"""
from __future__ import annotations

import numpy as np

X_ATOL = 1e-5
F_RTOL = 1e-5
APD_RTOL = 1e-5


def params(orc, m, d, N, H, problem, t_max=100, seed=0, alpha=2.0, f_r=0.1, **kw):
    return orc.make_params(m=m, d=d, N=N, H=H, problem=problem, t_max=t_max, alpha=alpha,
                           f_r=f_r, seed=seed, **kw)


def make_run(p):
    from paper_2404_01159_gb300 import Run
    return Run(m=p.m, d=p.d, N=p.N, H=p.H, problem=p.problem, t_max=p.t_max, alpha=p.alpha,
               f_r=p.f_r, eta_c=p.eta_c, eta_m=p.eta_m, p_c=p.p_c, p_m=p.p_m, lower=p.L,
               upper=p.U, seed=p.seed, reproduction=p.op, de_F=p.de_F, de_CR=p.de_CR,
               cso_phi=p.cso_phi, pso_w=p.pso_w, pso_c1=p.pso_c1, pso_c2=p.pso_c2)


def to_np(st):
    out = {}
    for k, v in st.items():
        out[k] = v.cpu().numpy() if hasattr(v, "cpu") else v
    return out


def assert_children(gx, ox, L=0.0, U=1.0):
    err = np.abs(gx.astype(np.float64) - ox)
    bad = err > X_ATOL * (U - L)
    assert not bad.any(), (int(bad.sum()), float(err.max()))


def assert_objectives(gf, of, rtol=F_RTOL):
    gf = gf.astype(np.float64)
    scale = np.linalg.norm(of, axis=1, keepdims=True)
    err = np.abs(gf - of)
    bad = err > rtol * scale + 1e-30
    assert not bad.any(), (int(bad.sum()), float((err / (scale + 1e-300)).max()))


ROLL_RTOL = 1e-2


def assert_rollout_objectives(gf, of, rtol=ROLL_RTOL):
    """Rollout objectives (BF16 policy GEMMs, FP32 accumulate) against the
    FP64 oracle: |f_gpu - f_orc| <= rtol max(|f_orc|, s_k), s_k the median
    |f_k| of the population (f1 = -sum s[0] can pass near zero, where a
    relative bound carries no meaning)."""
    gf = np.asarray(gf, dtype=np.float64)
    scale = np.maximum(np.abs(of), np.median(np.abs(of), axis=0, keepdims=True))
    err = np.abs(gf - of)
    bad = err > rtol * scale
    assert not bad.any(), (int(bad.sum()), float((err / scale).max()))
    return float((err / scale).max())


def assert_gamma(g, o):
    eps = np.finfo(np.float64).eps
    tol = 64 * eps / np.sin(o) + 1e-12 * o
    err = np.abs(np.asarray(g) - o)
    assert (err <= tol).all(), float((err / tol).max())


def selection_mismatches(Fc, validc, V, gpu_assoc, gpu_surv, o, tie_rel=1e-6):
    """Unexplained differences between a GPU selection and the oracle's.

    Fc, validc: the combined population as the oracle saw it (FP64)."""
    n = len(Fc)
    z = o["zstar"]
    fp = Fc - z
    nf = np.linalg.norm(fp, axis=1)
    oa = o["assoc"]
    ga = np.asarray(gpu_assoc)
    bad_assoc = []
    tie = np.zeros(n, dtype=bool)
    for i in range(n):
        if not validc[i]:
            if ga[i] != -1:
                bad_assoc.append(i)
            continue
        if ga[i] == oa[i]:
            continue
        if ga[i] < 0 or ga[i] >= len(V):
            bad_assoc.append(i)
            continue
        dg, do = fp[i] @ V[ga[i]], fp[i] @ V[oa[i]]
        if abs(dg - do) <= tie_rel * nf[i]:
            tie[i] = True
        else:
            bad_assoc.append(i)
    bad_surv = []
    gs_all = np.asarray(gpu_surv)
    for j in range(len(V)):
        gs, os_ = int(gs_all[j]), int(o["survivor"][j])
        if gs == os_:
            continue
        mem_g = set(np.nonzero(ga == j)[0].tolist())
        mem_o = set(np.nonzero(oa == j)[0].tolist())
        if mem_g != mem_o and all(tie[i] for i in mem_g ^ mem_o):
            continue
        if gs >= 0 and os_ >= 0 and oa[gs] == j:
            a, b = o["apd"][gs], o["apd"][os_]
            if abs(a - b) <= APD_RTOL * max(abs(b), 1e-300):
                continue
        bad_surv.append(j)
    return bad_assoc, bad_surv


def draws_mask(counts, sites, d):
    """Mutation mask (N x d uint8) from recorded site lists: row c has ones at
    sites[c, :counts[c]] (every variable when counts[c] == -1).  Also checks
    that each list holds distinct variables in [0, d)."""
    counts = np.asarray(counts)
    sites = np.asarray(sites)
    N = len(counts)
    mask = np.zeros((N, d), dtype=np.uint8)
    for c in range(N):
        k = int(counts[c])
        if k < 0:
            mask[c, :] = 1
            continue
        s = sites[c, :k]
        assert len(set(s.tolist())) == k and (s >= 0).all() and (s < d).all(), (c, s)
        mask[c, s] = 1
    return mask


def assert_draws(orc, p, t, run, oracle_parents):
    """The mating draws and mutation masks of the run's last generation
    (recorded on the GPU) equal the oracle's, bit for bit."""
    gpar, gcnt, gsites = (x.cpu().numpy() for x in run.last_draws())
    assert np.array_equal(gpar, np.asarray(oracle_parents)), \
        int((gpar != np.asarray(oracle_parents)).sum())
    _, omask = orc.mutation(p, t, np.zeros((p.N, p.d)))
    gmask = draws_mask(gcnt, gsites, p.d)
    assert np.array_equal(gmask, omask), int((gmask != omask).sum())


def igd(F, front):
    d = np.linalg.norm(front[:, None, :] - F[None, :, :], axis=2)
    return d.min(1).mean()
