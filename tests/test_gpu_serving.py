"""The serving loop: continuous batching of independent runs under an HBM
budget.  Requests arrive while others are on the GPU; each result must be
the bits the same run gets stepped alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# (m, d, N, H, problem, generations, seed, submitted before step k)
REQUESTS = [(3, 40, 105, 13, 0, 12, 1, 0), (2, 300, 1200, 1199, 1, 7, 2, 0),
            (5, 1500, 126, 5, 0, 9, 3, 0), (10, 30, 220, 3, 1, 5, 4, 2),
            (3, 2500, 1275, 49, 1, 6, 5, 3), (4, 64, 1771, 20, 0, 11, 6, 3),
            (3, 12, 105, 13, 1, 3, 7, 8)]


def test_served_results_equal_alone():
    from paper_2404_01159_gb300 import Run, Server, workspace_bytes
    sizes = [workspace_bytes(m, d, N) + 256 for (m, d, N, *_rest) in REQUESTS]
    arena = 2 * max(sizes) + min(sizes)     # far less than all of them together
    srv = Server(arena, max_live=3)
    ids, step, live_max, waited = {}, 0, 0, False
    pending = list(enumerate(REQUESTS))
    results = {}
    while pending or len(results) < len(REQUESTS):
        for q, req in [x for x in pending if x[1][7] <= step]:
            m, d, N, H, prob, gens, seed, _ = req
            ids[srv.submit(m, d, N, H, prob, gens, seed=seed)] = q
            pending.remove((q, req))
        st = srv.step()
        torch.cuda.synchronize()
        live_max = max(live_max, st["live"] + st["finished"])
        assert st["arena_used"] <= arena
        waited |= st["queued"] > 0
        for rid in srv.poll():
            results[ids[rid]] = srv.fetch(rid)
        step += 1
        assert step < 200
    assert waited, "the budget should have made some request wait"
    for q, req in enumerate(REQUESTS):
        m, d, N, H, prob, gens, seed, _ = req
        alone = Run(m=m, d=d, N=N, H=H, problem=prob, t_max=gens, seed=seed)
        alone.step(gens)
        Xa, va = alone.population()
        Fa, _ = alone.objectives()
        X, F, v = results[q]
        assert torch.equal(v, va), q
        ok = va.bool()
        assert torch.equal(X[ok], Xa[ok]), q
        assert torch.equal(F[ok], Fa[ok]), q
    srv.free()


def test_fetch_unknown_id_is_refused():
    from paper_2404_01159_gb300 import RveaError, Server
    srv = Server(1 << 24, max_live=1)
    with pytest.raises(RveaError):
        srv.meta[99] = (3, 12, 105)
        srv.fetch(99)
    srv.free()
