"""The seeded workload generators (inputs only, no RVEA arithmetic)."""
import math

import numpy as np
import pytest

from paper_2404_01159_gb300 import workloads as W


def test_batched_set_is_seeded_and_in_range():
    a, b = W.batched_set(256, 500), W.batched_set(256, 500)
    assert [x.__dict__ for x in a] == [x.__dict__ for x in b]
    assert {x.m for x in a} == {2, 3, 5, 10}
    for x in a:
        assert x.N == math.comb(x.H + x.m - 1, x.m - 1) and 100 <= x.N <= 9870
        assert 30 <= x.d <= 5000 and x.problem == x.seed % 2 and x.generations == 500
    # instance s does not depend on the set it belongs to
    assert W.batched_set(4, 500, seed0=10)[0].__dict__ == a[10].__dict__


def test_d_is_log_uniform():
    d = np.array([W.instance(s).d for s in range(4000)])
    u = (np.log(d) - math.log(30)) / (math.log(5000) - math.log(30))
    hist = np.histogram(u, bins=8, range=(0, 1))[0]
    assert hist.min() > 0.8 * 500 and hist.max() < 1.2 * 500


def test_request_stream_is_poisson():
    rs = W.request_stream(200.0, 30.0, seed=1)
    t = np.array([r[0] for r in rs])
    assert abs(len(t) - 6000) < 5 * math.sqrt(6000)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200) < 5 * (1 / 200) / math.sqrt(len(gaps))
    assert all(50 <= r[1].generations <= 1000 for r in rs)


def test_neuro_dynamics():
    dyn = W.neuro_dynamics(0)
    rho = max(abs(np.linalg.eigvals(dyn["A"])))
    assert abs(rho - 0.95) < 1e-12
    assert dyn["B"].shape == (17, 6) and W.policy_size() == 5702
