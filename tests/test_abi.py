"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
exports every function that include/rvea.h declares, and rejects invalid
arguments before touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rvea.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rvea_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def native():
    from paper_2404_01159_gb300 import _native
    return _native


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["rvea_workspace_bytes", "rvea_init", "rvea_step", "rvea_step_batch",
                     "rvea_population", "rvea_objectives", "rvea_sync_status", "rvea_free",
                     "rvea_status_str"]:
        assert required in names


def test_library_exports_every_declared_symbol(native):
    native.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", native.lib_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(rvea_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_workspace_sizes(native):
    L = native.lib()
    b1 = L.rvea_workspace_bytes(3, 5000, 9870)
    # the pool (2N rows of d floats) dominates; the rest is the direction
    # grid (77284 cells of 32 bytes, 1225 blocks' shares of 2048 overflow
    # entries of 2 bytes) and tables of O(N) or O(N m)
    pool = 2 * 9870 * 5000 * 4
    grid = 278 * 278 * 32 + 1225 * 2048 * 2
    assert pool + grid <= b1 < (pool + grid) * 1.02
    assert L.rvea_workspace_bytes(1, 10, 10) == 0
    assert L.rvea_workspace_bytes(3, 2, 10) == 0
    assert L.rvea_workspace_bytes(3, 12, 40000) == 0


def test_status_strings(native):
    L = native.lib()
    for s in range(0, -8, -1):
        assert L.rvea_status_str(s)
    assert b"lattice" in L.rvea_status_str(native.ERR_LATTICE)


def test_init_rejects_bad_arguments_without_gpu(native):
    L = native.lib()
    h = C.c_void_p()
    ws = C.c_void_p(1 << 20)   # never dereferenced: validation fails first

    def init(m, d, N, H, t_max=100, alpha=2.0, f_r=0.1, eta=20.0, problem=0):
        return L.rvea_init(m, d, N, H, alpha, f_r, eta, eta, 0, problem, t_max, ws,
                           1 << 30, None, C.byref(h))
    assert init(3, 12, 100, 13) == native.ERR_LATTICE
    assert init(1, 12, 105, 13) == native.ERR_ARG
    assert init(3, 2, 105, 13) == native.ERR_ARG
    assert init(3, 12, 105, 13, t_max=0) == native.ERR_ARG
    assert init(3, 12, 105, 13, f_r=1.5) == native.ERR_ARG
    assert init(3, 12, 105, 13, eta=0.0) == native.ERR_ARG
    assert init(3, 12, 105, 13, problem=7) == native.ERR_ARG
    assert not h.value


def test_init_ex_requires_the_unit_box_for_dtlz(native):
    """The DTLZ problems are defined on [0, 1]^d: another box is refused
    before any device work (the reproduction kernels clip by saturation)."""
    L = native.lib()
    h = C.c_void_p()
    ws = C.c_void_p(1 << 20)   # never dereferenced: validation fails first
    cfg = native.Config(m=3, d=12, N=105, H=13, problem=0, t_max=100, alpha=2.0, f_r=0.1,
                        eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0, lower=-1.0, upper=1.0,
                        seed=0, neuro=None)
    assert L.rvea_init_ex(C.byref(cfg), ws, 1 << 30, None, C.byref(h)) == native.ERR_ARG
    cfg.problem, cfg.lower = 1, 0.0
    cfg.upper = 2.0
    assert L.rvea_init_ex(C.byref(cfg), ws, 1 << 30, None, C.byref(h)) == native.ERR_ARG
    assert not h.value


def test_cso_config_and_swarm_calls_without_gpu(native):
    """The CSO operator (reproduction 3): phi outside [0, 1] is refused; its
    workspace adds the velocity pool (2N rows of d_pad floats), the kept
    APDs, the swarm centre and its partial sums; the swarm calls refuse NULL
    handles and arrays before any device work."""
    L = native.lib()
    base = dict(m=3, d=1001, N=210, H=19, problem=1, t_max=100, alpha=2.0, f_r=0.1,
                eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0, lower=0.0, upper=1.0,
                seed=0, neuro=None, reproduction=native.REPRO_CSO, de_F=0.5, de_CR=0.9)
    sbx = L.rvea_workspace_bytes(3, 1001, 210)
    cso = L.rvea_workspace_bytes_ex(C.byref(native.Config(**base, cso_phi=0.1)))
    d_pad, N = 1008, 210
    swarm = 2 * N * d_pad * 4 + N * 4 + d_pad * 4 + ((N + 63) // 64) * d_pad * 4
    assert sbx > 0 and cso >= sbx + swarm and cso < sbx + swarm + 6 * 256
    for phi in (-0.1, 1.5, float("nan")):
        assert L.rvea_workspace_bytes_ex(C.byref(native.Config(**base, cso_phi=phi))) == 0
    cfg = native.Config(**dict(base, reproduction=5), cso_phi=0.1)
    assert L.rvea_workspace_bytes_ex(C.byref(cfg)) == 0
    h = C.c_void_p()
    # the rollout problem takes SBX or CSO: DE is refused (as is any run of it
    # without its dynamics)
    cfg = native.Config(**dict(base, problem=2, reproduction=native.REPRO_DE), cso_phi=0.1)
    assert L.rvea_init_ex(C.byref(cfg), C.c_void_p(1 << 20), 1 << 30, None, C.byref(h)) == native.ERR_ARG
    assert L.rvea_export_swarm(None, None, None, None, None, None) == native.ERR_ARG
    a = C.c_void_p(1 << 20)
    assert L.rvea_import_swarm(None, a, a, a, a, None) == native.ERR_ARG


def test_pso_config_without_gpu(native):
    """The PSO operator (reproduction 4): inertia outside [0, 1] or a weight
    outside [0, 4] is refused; its workspace adds the velocity and
    personal-best pools (2N rows of d_pad floats each), the personal bests'
    objectives and the kept APDs, and no swarm centre."""
    L = native.lib()
    base = dict(m=3, d=1001, N=210, H=19, problem=1, t_max=100, alpha=2.0, f_r=0.1,
                eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0, lower=0.0, upper=1.0,
                seed=0, neuro=None, reproduction=native.REPRO_PSO, de_F=0.5, de_CR=0.9,
                cso_phi=0.0)
    sbx = L.rvea_workspace_bytes(3, 1001, 210)
    pso = L.rvea_workspace_bytes_ex(C.byref(native.Config(**base, pso_w=0.7298, pso_c1=1.5,
                                                          pso_c2=1.5)))
    d_pad, N, m = 1008, 210, 3
    swarm = 2 * (2 * N * d_pad * 4) + m * 2 * N * 4 + N * 4
    assert sbx > 0 and swarm <= pso - sbx < swarm + 6 * 256
    for w, c1, c2 in ((-0.1, 1.5, 1.5), (1.2, 1.5, 1.5), (0.5, 4.5, 1.5), (0.5, 1.5, -1.0),
                      (float("nan"), 1.5, 1.5)):
        cfg = native.Config(**base, pso_w=w, pso_c1=c1, pso_c2=c2)
        assert L.rvea_workspace_bytes_ex(C.byref(cfg)) == 0


def test_metrics_and_counters_reject_null_without_gpu(native):
    """The metric and counter entry points check their handles before any
    device work: NULL run / batch / output pointers are refused."""
    L = native.lib()
    out = C.c_double(-1.0)
    ref = (C.c_double * 3)(1.0, 1.0, 1.0)
    assert L.rvea_hypervolume(None, ref, C.byref(out), None) == native.ERR_ARG
    assert L.rvea_igd(None, C.c_void_p(1 << 20), 4, C.byref(out), None) == native.ERR_ARG
    assert out.value == -1.0
    assert L.rvea_launches_per_generation(None, 0) == -1
    assert L.rvea_batch_launches_per_step(None) == -1
    assert L.rvea_selftest_wait(0, None) == native.ERR_ARG
    assert L.rvea_selftest_wait(1 << 21, None) == native.ERR_ARG


def test_server_admission_refusals_without_gpu(native):
    """Serving loop, host side only (no step runs, so the arena is never
    touched): an invalid request or one that can never fit the arena is
    refused at submission and not queued; a valid one is queued with id 1;
    nothing is finished; fetching an unknown id is a state error."""
    L = native.lib()
    srv = C.c_void_p()
    arena_bytes = 64 << 20
    assert L.rvea_server_create(C.c_void_p(1 << 20), arena_bytes, 4, 0, C.byref(srv)) == native.OK
    try:
        def cfg(**kw):
            base = dict(m=3, d=12, N=105, H=13, problem=0, t_max=100, alpha=2.0, f_r=0.1,
                        eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0, lower=0.0, upper=1.0,
                        seed=0, neuro=None)
            base.update(kw)
            return native.Config(**base)
        rid = C.c_int64(0)
        sub = lambda c, g=10: L.rvea_server_submit(srv, C.byref(c), g, C.byref(rid))
        assert sub(cfg(N=100)) == native.ERR_ARG            # not the lattice size of H = 13
        assert sub(cfg(eta_c=0.0)) == native.ERR_ARG
        assert sub(cfg(), g=0) == native.ERR_ARG
        big = cfg(m=3, d=5000, N=9870, H=139)                 # ~0.4 GB > the 64 MB arena
        assert L.rvea_workspace_bytes(3, 5000, 9870) > arena_bytes
        assert sub(big) == native.ERR_NOMEM
        assert rid.value == 0                                  # nothing queued so far
        assert sub(cfg()) == native.OK and rid.value == 1
        ids = (C.c_int64 * 4)()
        n = C.c_int(-1)
        assert L.rvea_server_poll(srv, ids, 4, C.byref(n)) == native.OK and n.value == 0
        assert L.rvea_server_fetch(srv, 1, None, None, None, None) == native.ERR_STATE
    finally:
        L.rvea_server_free(srv)


def test_server_reports_failed_admission_by_id(native):
    """A request whose admission fails is not lost: the step goes on, poll
    reports its id, fetch returns its error once.  Made without a GPU (the
    initialisation's CUDA calls fail on a machine with no device), so the
    test only runs where CUDA is unavailable; the arena address is never
    dereferenced."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("the failure is made by the absence of a device")
    L = native.lib()
    srv = C.c_void_p()
    assert L.rvea_server_create(C.c_void_p(1 << 20), 64 << 20, 4, 0, C.byref(srv)) == native.OK
    try:
        cfg = native.Config(m=3, d=12, N=105, H=13, problem=0, t_max=100, alpha=2.0, f_r=0.1,
                            eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0, lower=0.0, upper=1.0,
                            seed=0, neuro=None)
        ids = []
        for _ in range(2):
            rid = C.c_int64(0)
            assert L.rvea_server_submit(srv, C.byref(cfg), 5, C.byref(rid)) == native.OK
            ids.append(rid.value)
        st = native.ServerStats()
        assert L.rvea_server_step(srv, None, C.byref(st)) == native.OK
        assert st.queued == 0 and st.live == 0 and st.finished == 2
        out = (C.c_int64 * 4)()
        n = C.c_int(-1)
        assert L.rvea_server_poll(srv, out, 4, C.byref(n)) == native.OK
        assert sorted(out[q] for q in range(n.value)) == ids
        for rid in ids:
            assert L.rvea_server_fetch(srv, rid, None, None, None, None) == native.ERR_CUDA
            assert L.rvea_server_fetch(srv, rid, None, None, None, None) == native.ERR_STATE
    finally:
        L.rvea_server_free(srv)


def test_lattice_for_matches_the_oracle(native, orc):
    """The library's H for a requested population size equals the oracle's
    (host arithmetic, no GPU)."""
    L = native.lib()
    for m in (2, 3, 4, 5):
        for n in [2 ** k for k in range(1, 15)] + [100, 9870, 9871, 32768]:
            assert L.rvea_lattice_for(m, n) == orc.lattice_for(m, n), (m, n)
