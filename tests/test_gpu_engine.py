"""The batched engine: kernel variants (plans), the autotuner and batches
captured as CUDA graphs.  Every variant must leave the results unchanged bit
for bit, so each case compares exported run states exactly."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import make_run, params, to_np  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _same(ra, rb):
    sa, sb = to_np(ra.export_state()), to_np(rb.export_state())
    for k in ("X", "F", "valid", "V", "gamma", "t"):
        assert np.array_equal(sa[k], sb[k], equal_nan=True), k


# (m, d, N, H, problem): pruned search and TMA-staged reproduction available;
# pruned only; staged only (m = 5 has no pruned search).
SHAPES = [(3, 2500, 1275, 49, 1), (2, 300, 1200, 1199, 0), (5, 1500, 126, 5, 0)]


@pytest.mark.parametrize("shape", SHAPES)
def test_every_plan_gives_the_same_bits(orc, shape):
    from paper_2404_01159_gb300 import get_plan, set_plan
    m, d, N, H, prob = shape
    p = params(orc, m, d, N, H, prob, t_max=40, seed=9)   # adapts every 4th generation
    ref = make_run(p)
    base = get_plan(ref)
    modes = [(0, 4), (0, 8), (0, 16)] + ([(1, 8), (2, 8)] if base["sel_mode"] > 0 else []) + \
        ([(3, 8)] if base["sel_mode"] == 3 else [])
    staged = [0, 1] if d > 1024 else [0]
    ref.step(10)
    for (mode, per_sm), st in itertools.product(modes, staged):
        run = make_run(p)
        set_plan(run, mode, per_sm, st)
        got = get_plan(run)
        assert (got["sel_mode"], got["repro_staged"]) == (mode, st)
        run.step(10)
        _same(ref, run)
        run.sync_status()


# A population whose vector tables exceed shared memory (N = 16290, m = 3:
# 261 KB of vectors): the fused tail reads its tables and the direction grid
# through L2, the shared-memory pruned kernels are refused, and the full scan
# gives the same bits over generations that adapt (the grid is rebuilt) and
# one stepped in a batch (full scan there, tiles kept current).
def test_tables_past_shared_memory(orc):
    from paper_2404_01159_gb300 import RveaError, get_plan, set_plan, step_batch
    p = params(orc, 3, 100, 16290, 179, 1, t_max=40, seed=4)   # adapts every 4th generation
    run = make_run(p)
    assert get_plan(run)["sel_mode"] == 3
    for mode in (1, 2):
        with pytest.raises(RveaError):
            set_plan(run, mode)
    ref = make_run(p)
    set_plan(ref, 0)
    run.step(6)
    ref.step(6)
    _same(ref, run)
    other = make_run(params(orc, 3, 40, 105, 13, 0, t_max=40, seed=5))
    for _ in range(3):              # t 7..9: an adaptation inside the batch
        step_batch([run, other])
    ref.step(3)
    _same(ref, run)
    run.step(4)                     # alone again, fused tail, tiles current
    ref.step(4)
    _same(ref, run)
    run.sync_status()
    ref.sync_status()


def test_variant_the_shape_lacks_is_refused(orc):
    from paper_2404_01159_gb300 import RveaError, set_plan
    run = make_run(params(orc, 5, 40, 126, 5, 0))
    with pytest.raises(RveaError):
        set_plan(run, 1)          # no pruned search for m = 5
    with pytest.raises(RveaError):
        set_plan(run, 0, 8, 1)    # no staged reproduction for d <= 1024
    with pytest.raises(RveaError):
        set_plan(run, 0, 99, 0)   # work items per SM out of range


def test_autotune_leaves_the_run_unchanged(orc):
    from paper_2404_01159_gb300 import autotune
    p = params(orc, 3, 2500, 1275, 49, 1, t_max=40, seed=4)
    tuned, plain = make_run(p), make_run(p)
    plan = autotune(tuned, use_cache=False)
    assert plan["repro_us"] > 0 and plan["sel_us"] > 0
    tuned.step(5)
    plain.step(5)
    plan = autotune(tuned, use_cache=False)   # mid-run, on an adaptation boundary's neighbour
    tuned.step(7)
    plain.step(7)
    _same(plain, tuned)
    # the cache returns the shape's latest tuned plan without timing
    again = make_run(p)
    cached = autotune(again, use_cache=True)
    assert (cached["sel_mode"], cached["sel_per_sm"], cached["repro_staged"]) == \
        (plan["sel_mode"], plan["sel_per_sm"], plan["repro_staged"])


def test_batch_graph_equals_alone(orc):
    """Uneven runs (m = 2..10, d from 3 to 2500, pruned and full-scan
    association, staged and direct reproduction, different adaptation
    periods) stepped as one CUDA graph per batched generation."""
    from paper_2404_01159_gb300 import Batch, autotune, set_plan
    shapes = [(3, 12, 105, 13, 0, 1, 30), (3, 2500, 1275, 49, 1, 2, 40), (10, 30, 220, 3, 0, 3, 50),
              (2, 300, 1200, 1199, 0, 4, 20), (5, 1500, 126, 5, 1, 5, 30), (3, 3, 105, 13, 1, 6, 60),
              (4, 64, 1771, 20, 0, 7, 40), (3, 1100, 105, 13, 3, 8, 30),
              (2, 1300, 100, 99, 4, 9, 30), (5, 60, 126, 5, 3, 10, 30)]
    ps = [params(orc, m, d, N, H, pr, t_max=tm, seed=s) for (m, d, N, H, pr, s, tm) in shapes]
    alone = [make_run(p) for p in ps]
    batch = [make_run(p) for p in ps]
    autotune(batch[1])
    set_plan(batch[3], 0, 16, 0)   # a pruned-capable run on the full scan
    b = Batch(batch)
    for _ in range(3):
        for r in alone:
            r.step(5)
        b.step(5)
    for ra, rb in zip(alone, batch):
        _same(ra, rb)
        rb.sync_status()
    b.free()


def test_batch_of_operators_equals_alone(orc):
    """Runs of every reproduction operator (SBX, DE, random, CSO with and
    without the centre, PSO) over the DTLZ problems, on the register and
    staged sizes and the fused-tail size, stepped together as batched
    generations (one launch per problem and operator) and alone: the same
    bits, swarm state included."""
    from paper_2404_01159_gb300 import Batch
    shapes = [(3, 12, 105, 13, 0, dict(op=0)), (3, 1001, 210, 19, 1, dict(op=1)),
              (2, 30, 100, 99, 3, dict(op=2)), (3, 2500, 1275, 49, 1, dict(op=3, cso_phi=0.1)),
              (10, 30, 220, 3, 0, dict(op=3, cso_phi=0.0)), (3, 1500, 105, 13, 4, dict(op=4)),
              (2, 4099, 100, 99, 1, dict(op=4, pso_w=0.5)), (5, 77, 126, 5, 1, dict(op=1))]
    ps = [params(orc, m, d, N, H, pr, t_max=20, seed=40 + i, **kw)
          for i, (m, d, N, H, pr, kw) in enumerate(shapes)]
    alone = [make_run(p) for p in ps]
    batch = [make_run(p) for p in ps]
    b = Batch(batch)
    for _ in range(2):
        for r in alone:
            r.step(3)
        b.step(3)
    for p, ra, rb in zip(ps, alone, batch):
        _same(ra, rb)
        if p.op in (3, 4):
            for x, y in zip(ra.export_swarm(), rb.export_swarm()):
                if x is not None:
                    assert np.array_equal(x.cpu().numpy(), y.cpu().numpy(), equal_nan=True)
        rb.sync_status()
    b.free()


@pytest.mark.parametrize("shape", [(3, 1001, 210, 19, 1), (3, 2500, 1275, 49, 1)])
def test_graph_stretches_equal_single_steps(orc, shape):
    """rvea_step replays captured stretches of non-adapting generations (and
    whole adaptation periods) as CUDA graphs; stepping one generation at a
    time gives the same bits, across an adaptation (t = 100)."""
    m, d, N, H, pr = shape
    p = params(orc, m, d, N, H, pr, t_max=1000, seed=12)
    a, b = make_run(p), make_run(p)
    a.step(3)
    a.step(107)   # t = 4..110: stretches of 8, then the adaptation at 100 step by step
    for _ in range(110):
        b.step(1)
    _same(a, b)
    a.sync_status()


def test_launch_counts(orc):
    """The launches a generation enqueues: reproduction, [mutation and
    evaluation when d > 1024], selection, finalize, [gamma and the tile table
    when it adapts]; a batched generation counts the kernel nodes of its
    graph."""
    from paper_2404_01159_gb300 import Batch, get_plan, set_plan
    big = make_run(params(orc, 3, 2500, 1275, 49, 1, t_max=40, seed=4))
    small = make_run(params(orc, 3, 12, 105, 13, 0, t_max=40, seed=5))
    # alone, the pruned-search run starts in the fused tail: reproduction + tail;
    # an adapting generation adds gamma, the tile table and the direction grid
    # (scale, count, scan, fill)
    assert get_plan(big)["sel_mode"] == 3
    assert big.launches_per_generation(False) == 2
    assert big.launches_per_generation(True) == 2 + 1 + 1 + 4
    set_plan(big, 1, 8, 1)
    assert big.launches_per_generation(False) == 4
    assert big.launches_per_generation(True) == 4 + 1 + 1 + 4
    assert small.launches_per_generation(False) == 3
    assert small.launches_per_generation(True) in (4, 5)
    b = Batch([big, small])
    try:
        # >= 1 reproduction group, 1 mutation group, >= 1 selection, finalize, gamma
        assert 5 <= b.launches_per_step() <= 9
    finally:
        b.free()


def test_bounded_wait_reports_timeout(orc):
    """Failure detection without a fault: a kernel waits on an mbarrier that
    nothing arrives at, with a short poll limit, and reports the timeout to
    the host; the context stays usable (a run steps cleanly afterwards)."""
    from paper_2404_01159_gb300 import _native
    L = _native.lib()
    assert L.rvea_selftest_wait(64, None) == _native.ERR_TIMEOUT
    run = make_run(params(orc, 3, 12, 105, 13, 0, t_max=10, seed=1))
    run.step(2)
    run.sync_status()
