"""ctypes front end of the FP64 CPU oracle (``rvea_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline legs of ``bench.py``.  The product package never imports
this module.  ``build()`` compiles the C source with gcc (no FMA contraction,
so x86 and Arm hosts evaluate the same expressions).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rvea_oracle.c")
_HDR = os.path.join(_HERE, "rvea_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

DTLZ2, DTLZ1, NEURO, DTLZ3, DTLZ4 = 0, 1, 2, 3, 4
TAG_INIT, TAG_MATE, TAG_PAIR, TAG_SBX, TAG_MUTSITE, TAG_MUTMAG, TAG_NOISE = 1, 2, 3, 4, 5, 6, 7


class Params(C.Structure):
    _fields_ = [("m", C.c_int32), ("d", C.c_int32), ("N", C.c_int32), ("H", C.c_int32),
                ("problem", C.c_int32), ("t_max", C.c_int32),
                ("alpha", C.c_double), ("f_r", C.c_double), ("eta_c", C.c_double),
                ("eta_m", C.c_double), ("p_c", C.c_double), ("p_m", C.c_double),
                ("L", C.c_double), ("U", C.c_double), ("seed", C.c_uint64),
                ("op", C.c_int32), ("de_F", C.c_double), ("de_CR", C.c_double),
                ("cso_phi", C.c_double), ("pso_w", C.c_double), ("pso_c1", C.c_double),
                ("pso_c2", C.c_double)]


class Neuro(C.Structure):
    _fields_ = [("ns", C.c_int32), ("na", C.c_int32), ("h1", C.c_int32), ("h2", C.c_int32),
                ("steps", C.c_int32), ("sigma", C.c_double),
                ("A", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double))]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= newest:
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        i32, f64, u8 = P(C.c_int32), P(C.c_double), P(C.c_uint8)
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_lattice_count.argtypes = [C.c_int32, C.c_int32]
        L.orc_lattice_count.restype = C.c_int64
        L.orc_lattice_for.argtypes = [C.c_int32, C.c_int32]
        L.orc_lattice_for.restype = C.c_int32
        L.orc_lattice.argtypes = [C.c_int32, C.c_int32, C.c_int32, i32]
        L.orc_lattice.restype = C.c_int32
        L.orc_lattice_unit.argtypes = [C.c_int32, C.c_int32, i32, f64]
        L.orc_gamma.argtypes = [C.c_int32, C.c_int32, f64, f64]
        L.orc_objective_range.argtypes = [C.c_int32, C.c_int32, f64, u8, f64]
        L.orc_adapt.argtypes = [C.c_int32, C.c_int32, f64, f64, f64]
        L.orc_init_population.argtypes = [P(Params), f64]
        L.orc_evaluate.argtypes = [P(Params), C.c_int32, f64, f64, P(Neuro), C.c_int32]
        L.orc_neuro_noise.argtypes = [P(Params), P(Neuro), C.c_int32, f64]
        L.orc_mating.argtypes = [P(Params), C.c_int32, C.c_int32, i32, i32]
        L.orc_sbx.argtypes = [P(Params), C.c_int32, f64, f64, f64]
        L.orc_mutation.argtypes = [P(Params), C.c_int32, f64, u8]
        L.orc_select.argtypes = [C.c_int32, C.c_int32, f64, u8, C.c_int32, f64, f64,
                                 C.c_int32, C.c_int32, C.c_double,
                                 f64, i32, f64, f64, i32]
        L.orc_generation.argtypes = [P(Params), C.c_int32, f64, P(Neuro),
                                     f64, f64, u8, f64, f64, f64, f64, i32, i32, i32]
        L.orc_generation.restype = C.c_int32
        L.orc_random_offspring.argtypes = [P(Params), C.c_int32, f64]
        L.orc_de_picks.argtypes = [P(Params), C.c_int32, C.c_int32, C.c_int32, i32]
        L.orc_de_offspring.argtypes = [P(Params), C.c_int32, f64, C.c_int32, i32,
                                       C.c_double, C.c_double, f64]
        L.orc_cso_picks.argtypes = [P(Params), C.c_int32, C.c_int32, C.c_int32, i32]
        L.orc_cso_offspring.argtypes = [P(Params), C.c_int32, f64, f64, f64, C.c_int32, i32,
                                        f64, f64, f64]
        L.orc_pso_picks.argtypes = [P(Params), C.c_int32, C.c_int32, C.c_int32, i32]
        L.orc_pso_offspring.argtypes = [P(Params), C.c_int32, f64, f64, f64, f64, C.c_int32,
                                        i32, f64, f64]
        L.orc_pso_pbest.argtypes = [P(Params), C.c_int32, C.c_int32, i32, f64, f64, f64, f64,
                                    f64, f64]
        L.orc_generation_ex.argtypes = [P(Params), C.c_int32, f64, P(Neuro),
                                        f64, f64, u8, f64, f64, f64, f64, f64, f64, f64, f64,
                                        i32, i32, i32]
        L.orc_generation_ex.restype = C.c_int32
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_get_threads.restype = C.c_int32
        _lib = L
    return _lib


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


OP_SBX_PM, OP_DE, OP_RANDOM, OP_CSO, OP_PSO = 0, 1, 2, 3, 4


def make_params(m, d, N, H, problem=DTLZ2, t_max=100, alpha=2.0, f_r=0.1,
                eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0, L=0.0, U=1.0, seed=0,
                op=OP_SBX_PM, de_F=0.5, de_CR=0.9, cso_phi=0.0,
                pso_w=0.7298, pso_c1=1.49618, pso_c2=1.49618):
    return Params(m, d, N, H, problem, t_max, alpha, f_r, eta_c, eta_m, p_c, p_m,
                  L, U, seed, op, de_F, de_CR, cso_phi, pso_w, pso_c1, pso_c2)


def pso_picks(p: Params, t: int, K: int, o: int):
    """Positions in the valid list of offspring o's particle and of the two
    candidates for its leader (PSO)."""
    out = np.zeros(3, dtype=np.int32)
    lib().orc_pso_picks(C.byref(p), int(t), int(K), int(o), _p(out, C.c_int32))
    return int(out[0]), int(out[1]), int(out[2])


def pso_offspring(p: Params, t: int, X, Vel, Pb, apd, vlist):
    """PSO offspring positions and velocities (N x d each)."""
    X, Vel, Pb, apd = _f64(X), _f64(Vel), _f64(Pb), _f64(apd)
    vl = np.ascontiguousarray(vlist, dtype=np.int32)
    Xo = np.zeros((p.N, p.d))
    Vo = np.zeros((p.N, p.d))
    lib().orc_pso_offspring(C.byref(p), int(t), _p(X, C.c_double), _p(Vel, C.c_double),
                            _p(Pb, C.c_double), _p(apd, C.c_double), len(vl),
                            _p(vl, C.c_int32), _p(Xo, C.c_double), _p(Vo, C.c_double))
    return Xo, Vo


def pso_pbest(p: Params, t: int, vlist, Pb, FPb, Xc, Fc):
    """Personal bests (N x d) and their objectives (N x m) of the offspring."""
    Pb, FPb, Xc, Fc = _f64(Pb), _f64(FPb), _f64(Xc), _f64(Fc)
    vl = np.ascontiguousarray(vlist, dtype=np.int32)
    Po = np.zeros((p.N, p.d))
    FPo = np.zeros((p.N, p.m))
    lib().orc_pso_pbest(C.byref(p), int(t), len(vl), _p(vl, C.c_int32), _p(Pb, C.c_double),
                        _p(FPb, C.c_double), _p(Xc, C.c_double), _p(Fc, C.c_double),
                        _p(Po, C.c_double), _p(FPo, C.c_double))
    return Po, FPo


def cso_picks(p: Params, t: int, K: int, o: int):
    """Positions in the valid list of offspring o's two competitors (CSO)."""
    out = np.zeros(2, dtype=np.int32)
    lib().orc_cso_picks(C.byref(p), int(t), int(K), int(o), _p(out, C.c_int32))
    return int(out[0]), int(out[1])


def cso_offspring(p: Params, t: int, X, Vel, apd, vlist, xbar):
    """CSO offspring positions and velocities (N x d each)."""
    X, Vel, apd, xbar = _f64(X), _f64(Vel), _f64(apd), _f64(xbar)
    vl = np.ascontiguousarray(vlist, dtype=np.int32)
    Xo = np.zeros((p.N, p.d))
    Vo = np.zeros((p.N, p.d))
    lib().orc_cso_offspring(C.byref(p), int(t), _p(X, C.c_double), _p(Vel, C.c_double),
                            _p(apd, C.c_double), len(vl), _p(vl, C.c_int32),
                            _p(xbar, C.c_double), _p(Xo, C.c_double), _p(Vo, C.c_double))
    return Xo, Vo


def lattice_count(m, H) -> int:
    return int(lib().orc_lattice_count(m, H))


def lattice_for(m, n) -> int:
    """H of the largest lattice with at most n points (the population of a
    run asked for n, which need not be a lattice size), -1 if none."""
    return int(lib().orc_lattice_for(m, n))


def lattice(m, H):
    N = lattice_count(m, H)
    K = np.zeros((N, m), dtype=np.int32)
    rows = lib().orc_lattice(m, H, N, _p(K, C.c_int32))
    assert rows == N
    return K


def lattice_unit(K):
    K = np.ascontiguousarray(K, dtype=np.int32)
    N, m = K.shape
    V = np.zeros((N, m))
    lib().orc_lattice_unit(m, N, _p(K, C.c_int32), _p(V, C.c_double))
    return V


def gamma(V):
    V = _f64(V)
    r, m = V.shape
    g = np.zeros(r)
    lib().orc_gamma(m, r, _p(V, C.c_double), _p(g, C.c_double))
    return g


def objective_range(F, valid=None):
    F = _f64(F)
    n, m = F.shape
    rg = np.zeros(m)
    v = None if valid is None else np.ascontiguousarray(valid, dtype=np.uint8)
    lib().orc_objective_range(m, n, _p(F, C.c_double), _p(v, C.c_uint8), _p(rg, C.c_double))
    return rg


def adapt(V0, rng):
    V0 = _f64(V0)
    r, m = V0.shape
    rng = _f64(rng)
    V = np.zeros_like(V0)
    lib().orc_adapt(m, r, _p(V0, C.c_double), _p(rng, C.c_double), _p(V, C.c_double))
    return V


def init_population(p: Params):
    X = np.zeros((p.N, p.d))
    lib().orc_init_population(C.byref(p), _p(X, C.c_double))
    return X


class NeuroData:
    """Keeps the numpy arrays alive behind the ctypes struct."""

    def __init__(self, A, B, steps=1000, sigma=0.01, h1=64, h2=64):
        self.A = _f64(A)
        self.B = _f64(B)
        ns, na = self.B.shape
        self.struct = Neuro(ns, na, h1, h2, steps, sigma,
                            _p(self.A, C.c_double), _p(self.B, C.c_double))


def _nd(nd):
    return None if nd is None else C.byref(nd.struct)


def evaluate(p: Params, X, t=0, nd=None):
    X = _f64(X)
    n = X.shape[0]
    F = np.zeros((n, p.m))
    lib().orc_evaluate(C.byref(p), n, _p(X, C.c_double), _p(F, C.c_double), _nd(nd), t)
    return F


def neuro_noise(p: Params, nd, t):
    xi = np.zeros((nd.struct.steps, nd.struct.ns))
    lib().orc_neuro_noise(C.byref(p), C.byref(nd.struct), t, _p(xi, C.c_double))
    return xi


def mating(p: Params, t, vlist):
    vl = np.ascontiguousarray(vlist, dtype=np.int32)
    P = (p.N + 1) // 2
    par = np.zeros(2 * P, dtype=np.int32)
    lib().orc_mating(C.byref(p), t, len(vl), _p(vl, C.c_int32), _p(par, C.c_int32))
    return par


def sbx(p: Params, t, X1, X2):
    X1, X2 = _f64(X1), _f64(X2)
    P = (p.N + 1) // 2
    assert X1.shape == (P, p.d) and X2.shape == (P, p.d)
    Xc = np.zeros((2 * P, p.d))
    lib().orc_sbx(C.byref(p), t, _p(X1, C.c_double), _p(X2, C.c_double), _p(Xc, C.c_double))
    return Xc


def mutation(p: Params, t, Xc):
    Xm = np.array(Xc[: p.N], dtype=np.float64, copy=True, order="C")
    mask = np.zeros((p.N, p.d), dtype=np.uint8)
    lib().orc_mutation(C.byref(p), t, _p(Xm, C.c_double), _p(mask, C.c_uint8))
    return Xm, mask


def random_offspring(p: Params, t):
    """Random reproduction (the extensibility experiment's baseline): N x d
    uniform offspring on [L, U]."""
    X = np.zeros((p.N, p.d))
    lib().orc_random_offspring(C.byref(p), t, _p(X, C.c_double))
    return X


def de_picks(p: Params, t, K, o):
    """(target position, r1, r2, r3 positions in the valid list, j_rand) of
    DE offspring o."""
    out = np.zeros(5, dtype=np.int32)
    lib().orc_de_picks(C.byref(p), t, K, o, _p(out, C.c_int32))
    return tuple(int(v) for v in out)


def de_offspring(p: Params, t, X, vlist, F=0.5, CR=0.9):
    """DE/rand/1/bin offspring (N x d) of the population X (rows by slot)
    with the valid list vlist."""
    X = _f64(X)
    vl = np.ascontiguousarray(vlist, dtype=np.int32)
    out = np.zeros((p.N, p.d))
    lib().orc_de_offspring(C.byref(p), t, _p(X, C.c_double), len(vl), _p(vl, C.c_int32),
                           float(F), float(CR), _p(out, C.c_double))
    return out


def select(F, valid, V, gam, t, t_max, alpha):
    F = _f64(F)
    n, m = F.shape
    V = _f64(V)
    r = V.shape[0]
    gam = _f64(gam)
    v = None if valid is None else np.ascontiguousarray(valid, dtype=np.uint8)
    z = np.zeros(m)
    assoc = np.zeros(n, dtype=np.int32)
    theta = np.zeros(n)
    apd = np.zeros(n)
    surv = np.zeros(r, dtype=np.int32)
    lib().orc_select(m, n, _p(F, C.c_double), _p(v, C.c_uint8), r, _p(V, C.c_double),
                     _p(gam, C.c_double), t, t_max, alpha, _p(z, C.c_double),
                     _p(assoc, C.c_int32), _p(theta, C.c_double), _p(apd, C.c_double),
                     _p(surv, C.c_int32))
    return dict(zstar=z, assoc=assoc, theta=theta, apd=apd, survivor=surv)


class State:
    """Population in vector-slot order, as the oracle's generation consumes it."""

    def __init__(self, X, F, valid, V, gamma, t, vel=None, apd=None, pbest=None, fpbest=None):
        self.X = np.array(X, dtype=np.float64, order="C", copy=True)
        # the CSO swarm state: velocities (zero at first) and the APD that
        # kept each member (+inf before any selection)
        self.vel = (np.zeros_like(self.X) if vel is None
                    else np.array(vel, dtype=np.float64, order="C", copy=True))
        self.apd = (np.full(self.X.shape[0], np.inf) if apd is None
                    else np.array(apd, dtype=np.float64, order="C", copy=True))
        self.F = np.array(F, dtype=np.float64, order="C", copy=True)
        # the PSO personal bests and their objectives (the positions themselves
        # at first)
        self.pbest = (self.X.copy() if pbest is None
                      else np.array(pbest, dtype=np.float64, order="C", copy=True))
        self.fpbest = (self.F.copy() if fpbest is None
                       else np.array(fpbest, dtype=np.float64, order="C", copy=True))
        self.valid = np.array(valid, dtype=np.uint8, order="C", copy=True)
        self.V = np.array(V, dtype=np.float64, order="C", copy=True)
        self.gamma = np.array(gamma, dtype=np.float64, order="C", copy=True)
        self.t = int(t)   # index of the NEXT generation to run


def initial_state(p: Params, nd=None):
    K = lattice(p.m, p.H)
    V0 = lattice_unit(K)
    X = init_population(p)
    F = evaluate(p, X, 0, nd)
    return V0, State(X, F, np.ones(p.N, np.uint8), V0, gamma(V0), 1)


def generation(p: Params, V0, st: State, nd=None):
    """Run generation st.t in place; return the inspection outputs."""
    P = (p.N + 1) // 2
    Xc = np.zeros((p.N, p.d))
    Fc = np.zeros((p.N, p.m))
    par = np.zeros(2 * P, dtype=np.int32)
    assoc = np.zeros(2 * p.N, dtype=np.int32)
    surv = np.zeros(p.N, dtype=np.int32)
    V0 = _f64(V0)
    alive = lib().orc_generation_ex(C.byref(p), st.t, _p(V0, C.c_double), _nd(nd),
                                    _p(st.X, C.c_double), _p(st.F, C.c_double),
                                    _p(st.valid, C.c_uint8), _p(st.V, C.c_double),
                                    _p(st.gamma, C.c_double), _p(st.vel, C.c_double),
                                    _p(st.apd, C.c_double), _p(st.pbest, C.c_double),
                                    _p(st.fpbest, C.c_double), _p(Xc, C.c_double),
                                    _p(Fc, C.c_double), _p(par, C.c_int32),
                                    _p(assoc, C.c_int32), _p(surv, C.c_int32))
    st.t += 1
    return dict(Xchild=Xc, Fchild=Fc, parents=par, assoc=assoc, survivor=surv,
                alive=alive)


def adapt_period(p: Params) -> int:
    import math
    return max(1, int(math.floor(p.f_r * p.t_max + 0.5)))


def igd(F, valid, R):
    """Inverted generational distance (Appendix C, numerical benchmarks, the
    IGD equation): the mean over the reference points f* in R of the
    Euclidean distance to the nearest objective vector of a valid member of
    the population F (n x m), in FP64."""
    P = np.asarray(F, dtype=np.float64)[np.asarray(valid, dtype=bool)]
    R = np.asarray(R, dtype=np.float64)
    if len(P) == 0 or len(R) == 0:
        raise ValueError("IGD needs a valid member and a reference point")
    d = np.sqrt(((R[:, None, :] - P[None, :, :]) ** 2).sum(axis=2))
    return float(d.min(axis=1).mean())



def hypervolume(F, valid, ref):
    """Hypervolume (Appendix C, the HV equation): the measure of the union,
    over the valid members f of F (n x m, m = 2 or 3) that dominate the
    reference point (f < ref in every objective), of the boxes [f, ref], in
    FP64.  m = 3 by slicing: the members sorted by f3 cut [min f3, ref3] into
    slabs, each slab's area is the 2-D hypervolume of the members at or below
    it; the 2-D hypervolume is the staircase of the members sorted by f1,
    each step as wide as the gap to the next f1 and as high as ref2 minus the
    smallest f2 so far."""
    P = np.asarray(F, dtype=np.float64)[np.asarray(valid, dtype=bool)]
    ref = np.asarray(ref, dtype=np.float64)
    m = P.shape[1]
    if m not in (2, 3) or ref.shape != (m,):
        raise ValueError("hypervolume: m = 2 or 3, ref of length m")
    P = P[(P < ref).all(axis=1)]

    def area(Q):   # 2-D: Q sorted by f1
        Q = Q[np.argsort(Q[:, 0], kind="stable")]
        a, low = 0.0, ref[1]
        for j in range(len(Q)):
            low = min(low, Q[j, 1])
            right = Q[j + 1, 0] if j + 1 < len(Q) else ref[0]
            a += (right - Q[j, 0]) * (ref[1] - low)
        return a

    if m == 2:
        return float(area(P)) if len(P) else 0.0
    P = P[np.argsort(P[:, 2], kind="stable")]
    vol = 0.0
    for i in range(len(P)):
        top = P[i + 1, 2] if i + 1 < len(P) else ref[2]
        if top > P[i, 2]:
            vol += (top - P[i, 2]) * area(P[: i + 1, :2])
    return float(vol)
