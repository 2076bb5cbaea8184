"""rvea_select_noalloc, the selection entry point for callers that cannot
allocate device memory (a plugin or server execution step whose host owns
every device byte, or a process whose memory another caching allocator has
reserved).  Its scratch is a fixed array inside the library, so it must give
the same results as rvea_select with caller scratch -- on the first call in
a fresh process (which sets the array up) and on the next call, which finds
the previous call's data still in the array.

The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(seed, m, n, r):
    rng = np.random.default_rng(seed)
    F = (rng.uniform(0, 2, (n, m)) ** 2).astype(np.float32)
    valid = (rng.uniform(size=n) > 0.1).astype(np.uint8)
    valid[0] = 1
    V = np.abs(rng.normal(size=(r, m)))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    g = rng.uniform(0.01, 0.2, r)
    dev = "cuda"
    return (torch.tensor(F, device=dev), torch.tensor(valid, device=dev),
            torch.tensor(V.astype(np.float32), device=dev),
            torch.tensor(g.astype(np.float32), device=dev))


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_select_matches_select():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_01159_gb300._native import ERR_NOMEM, OK, lib
    L = lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a larger call, then a smaller one with another m, so the second finds
    # stale data from the first in the shared array
    for seed, (m, n, r), t in [(0, (3, 2300, 1300), 7), (1, (5, 700, 126), 3)]:
        F, valid, V, g = _case(seed, m, n, r)
        need = L.rvea_select_scratch_bytes(n, r, m)
        raw = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        sp = (raw.data_ptr() + 255) & ~255
        a_ref = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        s_ref = torch.full((r,), -7, dtype=torch.int32, device="cuda")
        assert L.rvea_select(m, n, _p(F), _p(valid), r, _p(V), _p(g), t, 10, 2.0, _p(a_ref),
                             _p(s_ref), C.c_void_p(sp), need, stream) == OK
        a_na = torch.full((n,), -9, dtype=torch.int32, device="cuda")
        s_na = torch.full((r,), -9, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        assert L.rvea_select_noalloc(m, n, _p(F), _p(valid), r, _p(V), _p(g), t, 10, 2.0,
                                     _p(a_na), _p(s_na), stream) == OK
        torch.cuda.synchronize()
        if seed > 0:   # after the first call on the device, nothing more is reserved
            assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.equal(a_ref, a_na)
        assert torch.equal(s_ref, s_na)
        assert (s_na >= -1).all() and (s_na < n).all()
        del raw
    # beyond the stated maximum: rejected before any GPU work
    F, valid, V, g = _case(2, 3, 8, 4)
    a = torch.empty(70000, dtype=torch.int32, device="cuda")
    s = torch.empty(4, dtype=torch.int32, device="cuda")
    assert L.rvea_select_noalloc(3, 70000, _p(F), None, 4, _p(V), _p(g), 1, 10, 2.0,
                                 _p(a), _p(s), stream) == ERR_NOMEM
