"""Seeded synthetic workloads of many independent runs (no RVEA arithmetic):
the batched set of uneven runs and the request stream of the serving loop.

Every instance is drawn from its own seed, so instance s is the same
whichever set it belongs to:
  m uniform over {2, 3, 5, 10};
  H uniform over the Das-Dennis lattices of that m whose size
    N = C(H + m - 1, m - 1) lies in [100, 9870]
    (m = 2: H 99..9869, m = 3: 13..139, m = 5: 5..19, m = 10: 3..6);
  d = round(exp(U[ln 30, ln 5000]));
  problem = s mod 2 (0: spherical front DTLZ2, 1: linear front DTLZ1);
  generation budget: a fixed one for the batched set, U{50..1000} for a
    serving request.
Requests of the serving loop arrive as a Poisson process (exponential gaps).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

M_CHOICES = (2, 3, 5, 10)
N_MIN, N_MAX = 100, 9870
D_MIN, D_MAX = 30, 5000


def lattice_size(m: int, H: int) -> int:
    return math.comb(H + m - 1, m - 1)


def _lattice_hs(m: int) -> List[int]:
    hs = []
    H = 1
    while lattice_size(m, H) <= N_MAX:
        if lattice_size(m, H) >= N_MIN:
            hs.append(H)
        H += 1
    return hs


_HS = {m: _lattice_hs(m) for m in M_CHOICES}


@dataclass
class Instance:
    seed: int
    m: int
    H: int
    N: int
    d: int
    problem: int
    generations: int
    params: dict = field(default_factory=dict)

    def run_kwargs(self) -> dict:
        return dict(m=self.m, d=self.d, N=self.N, H=self.H, problem=self.problem,
                    t_max=self.generations, alpha=2.0, f_r=0.1, eta_c=20.0, eta_m=20.0,
                    p_c=1.0, p_m=1.0, seed=self.seed)


def instance(seed: int, generations: int | None = None) -> Instance:
    rng = np.random.default_rng([0x5EED, seed])
    m = int(rng.choice(M_CHOICES))
    H = int(rng.choice(_HS[m]))
    d = int(round(math.exp(rng.uniform(math.log(D_MIN), math.log(D_MAX)))))
    d = max(d, m)
    g = int(rng.integers(50, 1001)) if generations is None else int(generations)
    return Instance(seed, m, H, lattice_size(m, H), d, seed % 2, g)


def batched_set(n_runs: int = 256, generations: int = 500, seed0: int = 0) -> List[Instance]:
    """The batched uneven-runs workload: n_runs instances, seeds seed0.."""
    return [instance(seed0 + s, generations) for s in range(n_runs)]


def request_stream(rate_per_s: float = 200.0, duration_s: float = 60.0,
                   seed: int = 0) -> List[tuple]:
    """(arrival time in s, Instance) of a Poisson request stream."""
    rng = np.random.default_rng([0xA771, seed])
    t, out, s = 0.0, [], 0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            return out
        out.append((t, instance(1_000_000 + seed * 100_000 + s)))
        s += 1


def neuro_dynamics(seed: int = 0, ns: int = 17, na: int = 6, steps: int = 1000,
                   sigma: float = 0.01) -> dict:
    """Synthetic linear dynamics of the neuroevolution workload: A (ns x ns)
    Gaussian scaled to spectral radius 0.95 (eigenvalues in FP64), B (ns x na)
    Gaussian; process noise N(0, sigma^2)."""
    rng = np.random.default_rng([0xD1A, seed])
    A = rng.normal(size=(ns, ns))
    A *= 0.95 / float(np.max(np.abs(np.linalg.eigvals(A))))
    B = rng.normal(size=(ns, na))
    return {"A": A, "B": B, "steps": steps, "sigma": sigma, "h1": 64, "h2": 64}


def policy_size(ns: int = 17, na: int = 6, h1: int = 64, h2: int = 64) -> int:
    """d of an MLP policy ns -> h1 -> h2 -> na with biases."""
    return h1 * ns + h1 + h2 * h1 + h2 + na * h2 + na
