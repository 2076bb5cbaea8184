"""GPU <-> oracle parity of the CUDA path, called through the C ABI.

Every case compares the CUDA library with the FP64 oracle on the same seeded
inputs, element by element, under the tolerances of tests/gpu_util.py.
Sizes span several CTAs / tiles with ragged tails; the full-size case runs
the 9870 x 5000 DTLZ1 workload in the launch configuration bench.py times.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import (assert_children, assert_draws, assert_gamma, assert_objectives,  # noqa: E402
                      igd, make_run, params, selection_mismatches, to_np)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_01159_gb300 import _native
    _native.lib()


# (m, d, N, H, problem): the small DTLZ2 benchmark shape, a ragged DTLZ1 case
# spanning several reproduction CTAs / selection blocks / vector tiles, and
# m = 2 / 5 / 10;
# (d > 1024) take the shared-memory-staged reproduction path, with segments
# of several chunks, a partial last chunk and row padding; two are large
# populations (N = 4200, 2100 pairs) on the register and the staged load
# path; the last four are DTLZ3 and DTLZ4 on both paths.
SHAPES = [
    (3, 12, 105, 13, 0),
    (3, 1001, 210, 19, 1),
    (2, 203, 100, 99, 0),
    (5, 77, 126, 5, 1),
    (10, 30, 220, 3, 0),
    (3, 3, 105, 13, 1),
    (3, 300, 1275, 49, 0),
    (3, 2500, 105, 13, 1),
    (2, 4099, 100, 99, 0),
    (2, 30, 4200, 4199, 1),
    (2, 1100, 4200, 4199, 0),
    # DTLZ3 (problem 3) and DTLZ4 (problem 4), small d and staged
    (3, 40, 105, 13, 3),
    (3, 1500, 105, 13, 3),
    (3, 60, 105, 13, 4),
    (2, 2000, 100, 99, 4),
]


def _state_to_oracle(orc, st, swarm=None):
    s = to_np(st)
    vel = apd = pb = fpb = None
    if swarm is not None:   # CSO, PSO: the GPU's swarm state (float32 values)
        vel = np.nan_to_num(swarm[0].cpu().numpy().astype(np.float64))
        apd = swarm[1].cpu().numpy().astype(np.float64)
        if swarm[2] is not None:
            pb = np.nan_to_num(swarm[2].cpu().numpy().astype(np.float64))
            fpb = np.nan_to_num(swarm[3].cpu().numpy().astype(np.float64))
    return orc.State(s["X"].astype(np.float64), s["F"].astype(np.float64), s["valid"],
                     s["V"], s["gamma"], s["t"], vel=vel, apd=apd, pbest=pb, fpbest=fpb)


@pytest.mark.parametrize("shape", SHAPES)
def test_init_matches_oracle(orc, shape):
    m, d, N, H, prob = shape
    p = params(orc, m, d, N, H, prob, seed=11)
    run = make_run(p)
    st = to_np(run.export_state())
    X0 = orc.init_population(p)
    assert np.array_equal(st["X"].astype(np.float64), X0)        # bit-exact
    assert_objectives(st["F"], orc.evaluate(p, X0))
    V0 = orc.lattice_unit(orc.lattice(m, H))
    assert np.array_equal(st["V"], V0)                            # bit-exact lattice
    assert_gamma(st["gamma"], orc.gamma(V0))
    assert st["valid"].all() and st["t"] == 1
    run.sync_status()


@pytest.mark.parametrize("shape", SHAPES)
def test_teacher_forced_generations(orc, shape):
    _teacher_forced(orc, shape, 9)


# Mutation rates other than one site per row: several sites per row (p_m = 4
# and the largest accepted, 8, with sites in every segment of a staged row)
# and every site (p_m = d); the fused tail with p_m = 8 (children with
# more sites than their group of eight lanes take the one-lane path).
@pytest.mark.parametrize("shape,p_m", [((3, 300, 105, 13, 1), 8.0),
                                       ((3, 2500, 1275, 49, 1), 8.0),
                                       ((3, 2500, 105, 13, 0), 4.0),
                                       ((3, 40, 105, 13, 0), 40.0),
                                       ((2, 1500, 100, 99, 1), 1500.0)])
def test_teacher_forced_mutation_rates(orc, shape, p_m):
    _teacher_forced(orc, shape, 3, p_m=p_m)


# The extensibility experiment's operators in place of SBX and mutation
# (Sec. 4.4): DE/rand/1/bin (op 1) and random reproduction (op 2), on the
# small and staged sizes, one run in the fused tail (N = 1275).
@pytest.mark.parametrize("shape,op", [((3, 12, 105, 13, 0), 1), ((3, 1001, 210, 19, 1), 1),
                                      ((3, 2500, 1275, 49, 1), 1), ((10, 30, 220, 3, 0), 1),
                                      ((2, 30, 100, 99, 0), 2), ((3, 1500, 105, 13, 3), 2)])
def test_teacher_forced_other_operators(orc, shape, op):
    _teacher_forced(orc, shape, 6, op=op)


# The competitive swarm optimizer (op 3, the operator the paper's
# neuroevolution experiment picks): with and without the swarm-centre term,
# on the small, staged, fused-tail and m = 10 shapes; velocities and kept
# APDs are carried through six generations (one adaptation at t = 4).
@pytest.mark.parametrize("shape,phi", [((3, 12, 105, 13, 0), 0.1), ((3, 1001, 210, 19, 1), 0.0),
                                       ((3, 2500, 1275, 49, 1), 0.1), ((10, 30, 220, 3, 0), 0.2),
                                       ((2, 4099, 100, 99, 3), 0.15)])
def test_teacher_forced_cso(orc, shape, phi):
    _teacher_forced(orc, shape, 6, op=3, cso_phi=phi)


# Particle swarm optimization (op 4): Clerc's constriction weights and a
# stronger inertia, on the small, staged, fused-tail and m = 10 shapes;
# velocities, personal bests and kept APDs carried through six generations.
@pytest.mark.parametrize("shape,w", [((3, 12, 105, 13, 0), 0.7298), ((3, 1001, 210, 19, 1), 0.9),
                                     ((3, 2500, 1275, 49, 1), 0.7298), ((10, 30, 220, 3, 0), 0.5),
                                     ((2, 4099, 100, 99, 4), 0.7298)])
def test_teacher_forced_pso(orc, shape, w):
    _teacher_forced(orc, shape, 6, op=4, pso_w=w)


# Population sizes of the paper's speed sweeps that are not lattice sizes
# (Sec. 4.1: n = 2^k at d = 100, d = 2^k at n = 100): the run takes the
# largest Das-Dennis lattice with at most n points (n = 128 -> H = 14,
# N = 120; n = 1024 -> H = 43, N = 990; n = 100 -> H = 12, N = 91;
# n = 16384 -> H = 179, N = 16290, tables past shared memory), on the
# register path, the fused tail (tables in shared memory and in L2) and the
# staged path.
@pytest.mark.parametrize("n,d", [(128, 100), (1024, 100), (100, 4096), (16384, 100)])
def test_teacher_forced_sweep_sizes(orc, n, d):
    from paper_2404_01159_gb300 import lattice_for, lattice_size
    H = lattice_for(3, n)
    assert H == orc.lattice_for(3, n)
    N = lattice_size(3, H)
    assert N <= n < lattice_size(3, H + 1)
    _teacher_forced(orc, (3, d, N, H, 1), 4)


def _teacher_forced(orc, shape, gens, **kw):
    m, d, N, H, prob = shape
    p = params(orc, m, d, N, H, prob, t_max=40, seed=5, **kw)   # adapts every 4th gen
    V0 = orc.lattice_unit(orc.lattice(m, H))
    run = make_run(p)
    if p.op == 0:
        run.record_draws(True)
    for gen in range(gens):
        st = run.export_state()
        sw = run.export_swarm() if p.op in (3, 4) else None
        ost = _state_to_oracle(orc, st, sw)
        t = ost.t
        Fpar = ost.F.copy()
        vpar = ost.valid.copy()
        out = orc.generation(p, V0, ost)
        run.step(1)
        gx, gf = run.offspring()
        ga, gsurv = run.last_selection()
        gx, gf = gx.cpu().numpy(), gf.cpu().numpy()
        if p.op == 0:   # mating indices and mutation masks: bit-exact
            assert_draws(orc, p, t, run, out["parents"])
        if p.op == 2:   # random reproduction: u24 on the box, exact in float32
            assert np.array_equal(gx.astype(np.float64), out["Xchild"])
        assert_children(gx, out["Xchild"], p.L, p.U)
        # float32 objectives of the same decision vectors: 1e-5 relative
        assert_objectives(gf, orc.evaluate(p, gx.astype(np.float64), t))
        # against the oracle's own (FP64) children the difference also carries
        # the ~1e-7 child difference times the objective's conditioning
        # (DTLZ1: d/dx of 100 cos(20 pi x) ~ 6e3): a looser sanity bound
        assert_objectives(gf, out["Fchild"], rtol=1e-3)
        # selection on the GPU's own combined population
        Fc = np.concatenate([np.nan_to_num(Fpar), gf.astype(np.float64)])
        vc = np.concatenate([vpar, np.ones(N, np.uint8)])
        o = orc.select(Fc, vc, to_np(st)["V"], to_np(st)["gamma"], t, p.t_max, p.alpha)
        bad_a, bad_s = selection_mismatches(Fc, vc, to_np(st)["V"], ga.cpu().numpy(),
                                            gsurv.cpu().numpy(), o)
        assert not bad_a and not bad_s, (gen, bad_a[:5], bad_s[:5])
        if p.op in (3, 4):
            _check_swarm(run, sw, gsurv.cpu().numpy(), out["survivor"], ost, o, N)
        if p.op == 4:
            _check_pbest(run, sw, st, gx, gf, gsurv.cpu().numpy(), out["survivor"], ost, N)
        # the adapted reference vectors and gamma follow the GPU's survivors
        nst = to_np(run.export_state())
        assert nst["t"] == t + 1
        if t % orc.adapt_period(p) == 0:
            rng = orc.objective_range(nst["F"].astype(np.float64), nst["valid"])
            Vw = orc.adapt(V0, rng)
            assert np.allclose(nst["V"], Vw, rtol=0, atol=1e-15)
            assert_gamma(nst["gamma"], orc.gamma(Vw))
        else:
            assert np.array_equal(nst["V"], to_np(st)["V"])
    run.sync_status()


def _check_swarm(run, sw_prev, gsurv, osurv, ost, o, N):
    """CSO state after a generation: every kept APD is the APD (Eq. 4) of
    its survivor in the selection on the GPU's own combined population (where
    that selection associated the survivor with the same vector: an
    association tie within the tolerance can put it on a neighbour, whose
    gamma differs); a parent's velocity moves with it unchanged (bit for
    bit); a child's velocity matches the oracle's where both kept the same
    child."""
    vel, apd = (x.cpu().numpy() for x in run.export_swarm()[:2])
    vprev = sw_prev[0].cpu().numpy()
    live = gsurv >= 0
    assert np.isinf(apd[~live]).all()
    same = live.copy()
    same[live] = o["assoc"][gsurv[live]] == np.flatnonzero(live)
    assert same.sum() >= 0.9 * live.sum()
    ref = o["apd"][gsurv[same]]
    assert np.allclose(apd[same].astype(np.float64), ref, rtol=1e-5, atol=1e-30), \
        float((np.abs(apd[same] - ref) / ref).max())
    par = live & (gsurv < N)
    assert np.array_equal(vel[par], vprev[gsurv[par]])
    kid = live & (gsurv >= N) & (osurv == gsurv)
    assert kid.any()
    err = np.abs(vel[kid].astype(np.float64) - ost.vel[kid])
    assert err.max() <= 1e-5, float(err.max())


def _check_pbest(run, sw_prev, st_prev, gx, gf, gsurv, osurv, ost, N):
    """PSO personal bests after a generation.  The GPU's decision for each
    kept child, taken on its own float32 objectives, is the dominance rule
    recomputed here on the same float32 values (the old best is kept iff it
    dominates the child), and the row and objectives are that choice bit for
    bit; a kept parent keeps its best bit for bit; where the oracle kept the
    same child and took the same decision, its best matches within 1e-5."""
    _, _, pb, fpb = (x.cpu().numpy() for x in run.export_swarm())
    pb_prev, fpb_prev = sw_prev[2].cpu().numpy(), sw_prev[3].cpu().numpy()
    valid_prev = to_np(st_prev)["valid"]
    vlist = np.flatnonzero(valid_prev)
    K = len(vlist)
    live = gsurv >= 0
    par = live & (gsurv < N)
    assert np.array_equal(pb[par], pb_prev[gsurv[par]])
    assert np.array_equal(fpb[par], fpb_prev[gsurv[par]])
    agree = 0
    kids = np.flatnonzero(live & (gsurv >= N))
    for j in kids:
        c = gsurv[j] - N
        ip = vlist[c % K]
        fo, fc = fpb_prev[ip], gf[c]
        keep_old = bool(np.all(fo <= fc) and np.any(fo < fc))
        want_p, want_f = (pb_prev[ip], fo) if keep_old else (gx[c], fc)
        assert np.array_equal(pb[j], want_p) and np.array_equal(fpb[j], want_f), (j, keep_old)
        if osurv[j] == gsurv[j]:
            o_keep = np.array_equal(ost.pbest[j], pb_prev[ip].astype(np.float64))
            if o_keep == keep_old:
                agree += 1
                assert np.abs(ost.pbest[j] - pb[j]).max() <= 1e-5
    assert agree >= 0.9 * np.sum(osurv[kids] == gsurv[kids])


@pytest.mark.parametrize("m,n,r,seed", [(3, 700, 1300, 0), (2, 257, 100, 1), (5, 1000, 126, 2),
                                        (7, 300, 600, 3), (10, 513, 220, 4), (3, 1, 5, 5)])
def test_select_operator(orc, m, n, r, seed):
    from paper_2404_01159_gb300 import select
    rng = np.random.default_rng(seed)
    F32 = (rng.uniform(0, 2, (n, m)) ** 2).astype(np.float32)
    valid = (rng.uniform(size=n) > 0.1).astype(np.uint8)
    valid[0] = 1
    V = np.abs(rng.normal(size=(r, m)))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    V32 = V.astype(np.float32)
    V64 = V32.astype(np.float64)
    gam = orc.gamma(V64)
    gam32 = gam.astype(np.float32)
    for t in (1, 7, 10):
        ga, gs = select(torch.tensor(F32, device="cuda"), torch.tensor(valid, device="cuda"),
                        torch.tensor(V32, device="cuda"), torch.tensor(gam32, device="cuda"),
                        t, 10, 2.0)
        o = orc.select(F32.astype(np.float64), valid, V64, gam32.astype(np.float64), t, 10, 2.0)
        bad_a, bad_s = selection_mismatches(F32.astype(np.float64), valid, V64,
                                            ga.cpu().numpy(), gs.cpu().numpy(), o)
        assert not bad_a and not bad_s, (t, bad_a[:5], bad_s[:5])


def test_select_operator_ties_and_ideal_point(orc):
    from paper_2404_01159_gb300 import select
    # duplicated solutions (exact APD ties: lower index wins) and a solution at z*
    F = np.array([[0.0, 0.0], [1.0, 0.5], [1.0, 0.5], [0.25, 2.0], [0.25, 2.0]], np.float32)
    V = np.array([[1.0, 0.0], [0.0, 1.0], [0.6, 0.8], [0.8, 0.6]], np.float32)
    V64 = V.astype(np.float64)
    gam = orc.gamma(V64).astype(np.float32)
    ga, gs = select(torch.tensor(F, device="cuda"), None, torch.tensor(V, device="cuda"),
                    torch.tensor(gam, device="cuda"), 3, 10, 2.0)
    o = orc.select(F.astype(np.float64), None, V64, gam.astype(np.float64), 3, 10, 2.0)
    assert np.array_equal(ga.cpu().numpy(), o["assoc"])
    assert np.array_equal(gs.cpu().numpy(), o["survivor"])
    assert gs.cpu().numpy()[0] == 0


@pytest.mark.parametrize("m,H", [(3, 13), (2, 99), (5, 5), (10, 3), (3, 139)])
def test_gamma_operator(orc, m, H):
    from paper_2404_01159_gb300 import gamma
    V0 = orc.lattice_unit(orc.lattice(m, H))
    for V in (V0, orc.adapt(V0, np.linspace(0.5, 3.0, m))):
        g = gamma(torch.tensor(V, device="cuda")).cpu().numpy()
        assert_gamma(g, orc.gamma(V))


def _front(orc, m, prob):
    """A sample of the true Pareto front: the unit Das-Dennis lattice of
    H = 30 (DTLZ2's sphere) or the same lattice on the simplex sum f = 1/2
    (DTLZ1)."""
    L = orc.lattice(m, 30)
    return 0.5 * L / 30.0 if prob == 1 else orc.lattice_unit(L)


# t_{0.995, 9}: two-sided 99 % quantile of Student's t with 9 degrees of freedom
T99_DF9 = 3.2498


@pytest.mark.parametrize("d,prob,gens", [(12, 0, 100), (7, 1, 400)])
def test_free_running_igd_matches_oracle(orc, d, prob, gens):
    """Free-running statistical parity: FP32 (GPU) and FP64 (oracle)
    trajectories from the same seed diverge chaotically, so their final
    populations are compared as distributions.  Ten seeds on each side; the
    99 % confidence intervals of the mean final IGD (Appendix C) must overlap
    (each widened by 0.5 % of the oracle's mean: converged runs of both sides
    can have near-zero spread, and a difference below that is no difference
    in quality).
    DTLZ2: m = 3, d = 12, N = 105 (the small benchmark shape); DTLZ1: m = 3,
    d = 7 (the paper's DTLZ1 setting), N = 105."""
    m, N, H = 3, 105, 13
    front = _front(orc, m, prob)
    ig = {"gpu": [], "oracle": []}
    for seed in range(10):
        p = params(orc, m, d, N, H, prob, t_max=gens, seed=100 + seed)
        run = make_run(p)
        run.step(gens)
        F, valid = run.objectives()
        run.sync_status()
        F, valid = F.cpu().numpy().astype(np.float64), valid.cpu().numpy().astype(bool)
        ig["gpu"].append(igd(F[valid], front))
        V0, st = orc.initial_state(p)
        for _ in range(gens):
            orc.generation(p, V0, st)
        ig["oracle"].append(igd(st.F[st.valid.astype(bool)], front))
    ci = {}
    for k, v in ig.items():
        v = np.asarray(v)
        h = T99_DF9 * v.std(ddof=1) / np.sqrt(len(v)) + 0.005 * np.mean(ig["oracle"])
        ci[k] = (v.mean() - h, v.mean() + h)
    assert ci["gpu"][0] <= ci["oracle"][1] and ci["oracle"][0] <= ci["gpu"][1], (ig, ci)
    if prob == 0:   # DTLZ2 converges within 100 generations
        assert max(ig["gpu"]) < 0.1, ig


def test_checkpoint_roundtrip_bit_identical(orc):
    p = params(orc, 3, 1001, 210, 19, 1, t_max=40, seed=9)
    a = make_run(p)
    a.step(7)
    st = a.export_state()
    b = make_run(params(orc, 3, 1001, 210, 19, 1, t_max=40, seed=9))
    b.import_state(st["X"], st["F"], st["valid"], st["V"], st["gamma"], st["t"])
    a.step(6)
    b.step(6)
    sa, sb = to_np(a.export_state()), to_np(b.export_state())
    for k in ("X", "F", "valid", "V", "gamma"):
        assert np.array_equal(sa[k], sb[k], equal_nan=True), k
    assert sa["t"] == sb["t"] == 14


@pytest.mark.parametrize("op,kw", [(3, dict(cso_phi=0.1)), (4, dict(pso_w=0.7298))])
def test_checkpoint_roundtrip_swarm(orc, op, kw):
    """A CSO or PSO run resumed from its exported state and swarm state
    (velocities, kept APDs, personal bests) continues bit for bit; without
    the swarm state the resumed run starts a new swarm and differs."""
    p = params(orc, 3, 1001, 210, 19, 1, t_max=40, seed=9, op=op, **kw)
    a = make_run(p)
    a.step(7)
    st, sw = a.export_state(), a.export_swarm()
    b = make_run(p)
    b.import_state(st["X"], st["F"], st["valid"], st["V"], st["gamma"], st["t"])
    b.import_swarm(*sw)
    c = make_run(p)
    c.import_state(st["X"], st["F"], st["valid"], st["V"], st["gamma"], st["t"])
    for r in (a, b, c):
        r.step(6)
    sa, sb, sc = (to_np(r.export_state()) for r in (a, b, c))
    for k in ("X", "F", "valid", "V", "gamma"):
        assert np.array_equal(sa[k], sb[k], equal_nan=True), k
    wa, wb = ([x.cpu().numpy() for x in r.export_swarm() if x is not None] for r in (a, b))
    for x, y in zip(wa, wb):
        assert np.array_equal(x, y, equal_nan=True)
    assert not np.array_equal(sa["X"], sc["X"], equal_nan=True)


def test_import_refuses_population_without_valid_member(orc):
    """A state with no valid member is refused (mating would have nothing to
    draw from) and the run keeps its state."""
    from paper_2404_01159_gb300 import RveaError
    from paper_2404_01159_gb300._native import ERR_ARG
    p = params(orc, 3, 12, 105, 13, 0, t_max=100, seed=8)
    run = make_run(p)
    run.step(3)
    st = run.export_state()
    none = torch.zeros_like(st["valid"])
    with pytest.raises(RveaError) as e:
        run.import_state(st["X"], st["F"], none, st["V"], st["gamma"], st["t"])
    assert e.value.status == ERR_ARG
    after = to_np(run.export_state())
    for k in ("X", "F", "valid", "V", "gamma"):
        assert np.array_equal(to_np(st)[k], after[k], equal_nan=True), k
    run.step(1)
    run.sync_status()


def test_graph_replay_equals_direct_launches(orc):
    p = params(orc, 3, 12, 105, 13, 0, t_max=100, seed=4)   # adaptation period 10
    a, b = make_run(p), make_run(p)
    a.step(35)                        # graph replays of whole periods
    for _ in range(35):
        b.step(1)                     # one generation per call
    sa, sb = to_np(a.export_state()), to_np(b.export_state())
    for k in ("X", "F", "valid", "V", "gamma"):
        assert np.array_equal(sa[k], sb[k], equal_nan=True), k


def test_batch_equals_alone(orc):
    """A run stepped alone and the same run inside a batch give identical bits.
    Alone, runs with m <= 4 and N >= 1000 take the pruned association kernel;
    in a batch every run takes the full scan, so this also checks that the
    pruning is exact."""
    from paper_2404_01159_gb300 import step_batch
    shapes = [(3, 12, 105, 13, 0, 1), (3, 1001, 210, 19, 1, 2), (10, 30, 220, 3, 0, 3),
              (2, 203, 100, 99, 1, 4), (3, 64, 1275, 49, 1, 5), (2, 40, 1200, 1199, 0, 6),
              (4, 20, 1771, 20, 0, 7), (3, 40, 105, 13, 3, 8), (3, 1200, 210, 19, 4, 9)]
    ps = [params(orc, m, d, N, H, pr, t_max=30, seed=s) for (m, d, N, H, pr, s) in shapes]
    alone = [make_run(p) for p in ps]
    batch = [make_run(p) for p in ps]
    for _ in range(12):
        for r in alone:
            r.step(1)
        step_batch(batch)
    for ra, rb in zip(alone, batch):
        sa, sb = to_np(ra.export_state()), to_np(rb.export_state())
        for k in ("X", "F", "valid", "V", "gamma"):
            assert np.array_equal(sa[k], sb[k], equal_nan=True), k
        rb.sync_status()


@pytest.mark.parametrize("f_r", [0.1, 0.003])
def test_full_size_dtlz1(orc, f_r):
    """The 9870 x 5000 DTLZ1 workload of the benchmark, one teacher-forced
    generation (t = 3) at full size: the mating draws and mutation masks bit
    for bit, every child row element-wise, every objective against the
    oracle's evaluation of the GPU's children, and the whole selection.  With
    f_r = 0.003 (adaptation every 3 generations) the generation also rescales
    the reference vectors, checked with gamma against the oracle."""
    import os
    orc.set_threads(os.cpu_count() or 1)
    try:
        m, d, N, H = 3, 5000, 9870, 139
        p = params(orc, m, d, N, H, 1, t_max=1000, seed=0, f_r=f_r)
        run = make_run(p)
        run.step(2)
        run.record_draws(True)
        st = run.export_state()
        ost = _state_to_oracle(orc, st)
        t = ost.t
        assert t == 3
        Fpar, vpar = ost.F.copy(), ost.valid.copy()
        V0 = orc.lattice_unit(orc.lattice(m, H))
        out = orc.generation(p, V0, ost)
        run.step(1)
        gx, gf = run.offspring()
        ga, gs = run.last_selection()
        assert_draws(orc, p, t, run, out["parents"])
        gx = gx.cpu().numpy()
        assert_children(gx, out["Xchild"])
        gf = gf.cpu().numpy()
        assert_objectives(gf, orc.evaluate(p, gx.astype(np.float64), t))
        assert_objectives(gf, out["Fchild"], rtol=1e-3)
        Fc = np.concatenate([np.nan_to_num(Fpar), gf.astype(np.float64)])
        vc = np.concatenate([vpar, np.ones(N, np.uint8)])
        o = orc.select(Fc, vc, to_np(st)["V"], to_np(st)["gamma"], t, p.t_max, p.alpha)
        bad_a, bad_s = selection_mismatches(Fc, vc, to_np(st)["V"], ga.cpu().numpy(),
                                            gs.cpu().numpy(), o)
        assert not bad_a and not bad_s, (bad_a[:5], bad_s[:5])
        nst = to_np(run.export_state())
        if t % orc.adapt_period(p) == 0:
            rng = orc.objective_range(nst["F"].astype(np.float64), nst["valid"])
            Vw = orc.adapt(V0, rng)
            assert np.allclose(nst["V"], Vw, rtol=0, atol=1e-15)
            assert_gamma(nst["gamma"], orc.gamma(Vw))
            assert not np.array_equal(nst["V"], to_np(st)["V"])
        else:
            assert np.array_equal(nst["V"], to_np(st)["V"])
        run.sync_status()
    finally:
        orc.set_threads(1)


@pytest.mark.parametrize("shape", [(3, 12, 105, 13, 0), (3, 300, 1275, 49, 1), (2, 1500, 100, 99, 4)])
def test_igd_matches_oracle(orc, shape):
    """IGD of the GPU population (Appendix C) against the oracle's definition
    on the same objective vectors, with the problem's front as reference:
    the unit sphere (DTLZ2/DTLZ4, the unit lattice) or the simplex sum f =
    1/2 (DTLZ1, the lattice halved)."""
    m, d, N, H, prob = shape
    p = params(orc, m, d, N, H, prob, t_max=50, seed=21)
    run = make_run(p)
    run.step(7)
    st = to_np(run.export_state())
    L = orc.lattice(m, H)
    R = (0.5 * L / H if prob == 1 else orc.lattice_unit(L)).astype(np.float32)
    g = run.igd(torch.tensor(R, device="cuda"))
    o = orc.igd(st["F"].astype(np.float64), st["valid"], R.astype(np.float64))
    assert abs(g - o) <= 1e-5 * o + 1e-7, (g, o)
    run.sync_status()


@pytest.mark.parametrize("shape", [(3, 12, 105, 13, 0), (3, 300, 1275, 49, 1),
                                   (2, 1500, 100, 99, 4), (2, 40, 1200, 1199, 0)])
def test_hypervolume_matches_oracle(orc, shape):
    """Hypervolume of the GPU population (Appendix C) against the oracle's
    slicing on the same objective vectors, for a reference point beyond
    every member and for one at the per-objective 75th percentile (members
    beyond it drop out on both sides)."""
    m, d, N, H, prob = shape
    p = params(orc, m, d, N, H, prob, t_max=50, seed=23)
    run = make_run(p)
    run.step(6)
    st = to_np(run.export_state())
    F = st["F"].astype(np.float64)
    Fv = F[st["valid"].astype(bool)]
    for ref in (1.1 * Fv.max(axis=0), np.percentile(Fv, 75, axis=0)):
        g = run.hypervolume(ref.tolist())
        o = orc.hypervolume(F, st["valid"], ref)
        assert abs(g - o) <= 1e-9 * o, (g, o, ref)
    assert o <= orc.hypervolume(F, st["valid"], 1.1 * Fv.max(axis=0))
    run.sync_status()
