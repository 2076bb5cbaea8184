"""Neuroevolution rollout (the linear-dynamics stand-in for the paper's
control tasks): BF16 tensor-core policy GEMMs with FP32 accumulation against
the FP64 oracle, within 1e-2 (gpu_util.assert_rollout_objectives)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import (assert_children, assert_rollout_objectives, params,  # noqa: E402
                      selection_mismatches, to_np)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _setup(orc, N, H, steps, seed, t_max=40, gemv=0, cso_phi=None):
    from paper_2404_01159_gb300 import NEURO_LINEAR, Run
    from paper_2404_01159_gb300.workloads import neuro_dynamics, policy_size
    dyn = dict(neuro_dynamics(seed, steps=steps), gemv=gemv)
    d = policy_size()
    op = dict() if cso_phi is None else dict(op=orc.OP_CSO, cso_phi=cso_phi)
    p = params(orc, 2, d, N, H, orc.NEURO, t_max=t_max, seed=seed, L=-1.0, U=1.0, **op)
    nd = orc.NeuroData(dyn["A"], dyn["B"], steps=steps, sigma=dyn["sigma"])
    run = Run(m=2, d=d, N=N, H=H, problem=NEURO_LINEAR, t_max=t_max, seed=seed, neuro=dyn,
              reproduction=p.op, cso_phi=p.cso_phi)
    return p, nd, run


# gemv 0: the policy GEMVs on the tensor cores (BF16 hi/lo, FP32 accumulate);
# gemv 1: on the CUDA cores in FP32
@pytest.mark.parametrize("gemv", [0, 1])
def test_initial_population_and_rollout(orc, gemv):
    p, nd, run = _setup(orc, 10, 9, 200, 3, gemv=gemv)
    st = to_np(run.export_state())
    X0 = orc.init_population(p)
    # Box-Muller weights: float32 on the GPU, FP64 in the oracle
    assert np.allclose(st["X"], X0, rtol=0, atol=2e-7)
    # the rollouts of the GPU's own weights
    err = assert_rollout_objectives(st["F"], orc.evaluate(p, st["X"].astype(np.float64), 0, nd))
    assert err < 1e-2
    run.sync_status()


@pytest.mark.parametrize("gemv", [0, 1])
def test_teacher_forced_neuro_generations(orc, gemv):
    p, nd, run = _setup(orc, 10, 9, 100, 5, gemv=gemv)
    V0 = orc.lattice_unit(orc.lattice(2, 9))
    for gen in range(5):
        st = run.export_state()
        s = to_np(st)
        ost = orc.State(s["X"].astype(np.float64), s["F"].astype(np.float64), s["valid"],
                        s["V"], s["gamma"], s["t"])
        t = ost.t
        Fpar, vpar = ost.F.copy(), ost.valid.copy()
        out = orc.generation(p, V0, ost, nd)
        run.step(1)
        gx, gf = run.offspring()
        ga, gsurv = run.last_selection()
        gx, gf = gx.cpu().numpy(), gf.cpu().numpy()
        assert_children(gx, out["Xchild"], p.L, p.U)
        assert_rollout_objectives(gf, orc.evaluate(p, gx.astype(np.float64), t, nd))
        Fc = np.concatenate([np.nan_to_num(Fpar), gf.astype(np.float64)])
        vc = np.concatenate([vpar, np.ones(p.N, np.uint8)])
        o = orc.select(Fc, vc, s["V"], s["gamma"], t, p.t_max, p.alpha)
        bad_a, bad_s = selection_mismatches(Fc, vc, s["V"], ga.cpu().numpy(),
                                            gsurv.cpu().numpy(), o)
        assert not bad_a and not bad_s, (gen, bad_a[:5], bad_s[:5])
    run.sync_status()


# CSO on the rollout problem (the operator the paper's neuroevolution
# experiment picks): the competitions and the learning on the GPU, the
# children evaluated by the rollout, velocities and kept APDs carried.
@pytest.mark.parametrize("phi", [0.0, 0.1])
def test_teacher_forced_neuro_cso(orc, phi):
    p, nd, run = _setup(orc, 10, 9, 100, 6, gemv=1, cso_phi=phi)
    V0 = orc.lattice_unit(orc.lattice(2, 9))
    for gen in range(4):
        st = run.export_state()
        vel, apd, _, _ = run.export_swarm()
        s = to_np(st)
        ost = orc.State(s["X"].astype(np.float64), s["F"].astype(np.float64), s["valid"],
                        s["V"], s["gamma"], s["t"],
                        vel=np.nan_to_num(vel.cpu().numpy().astype(np.float64)),
                        apd=apd.cpu().numpy().astype(np.float64))
        t = ost.t
        Fpar, vpar = ost.F.copy(), ost.valid.copy()
        out = orc.generation(p, V0, ost, nd)
        run.step(1)
        gx, gf = run.offspring()
        ga, gsurv = run.last_selection()
        gx, gf = gx.cpu().numpy(), gf.cpu().numpy()
        assert_children(gx, out["Xchild"], p.L, p.U)
        assert_rollout_objectives(gf, orc.evaluate(p, gx.astype(np.float64), t, nd))
        Fc = np.concatenate([np.nan_to_num(Fpar), gf.astype(np.float64)])
        vc = np.concatenate([vpar, np.ones(p.N, np.uint8)])
        o = orc.select(Fc, vc, s["V"], s["gamma"], t, p.t_max, p.alpha)
        bad_a, bad_s = selection_mismatches(Fc, vc, s["V"], ga.cpu().numpy(),
                                            gsurv.cpu().numpy(), o)
        assert not bad_a and not bad_s, (gen, bad_a[:5], bad_s[:5])
    run.sync_status()


@pytest.mark.parametrize("gemv", [0, 1])
def test_full_size_rollout_sampled(orc, gemv):
    """The 100-policy, 1000-step configuration of the neuroevolution
    workload: every policy of the initial population against the oracle."""
    import os
    orc.set_threads(os.cpu_count() or 1)
    p, nd, run = _setup(orc, 100, 99, 1000, 0, t_max=1000, gemv=gemv)
    st = to_np(run.export_state())
    of = orc.evaluate(p, st["X"].astype(np.float64), 0, nd)
    assert_rollout_objectives(st["F"], of)
    run.step(2)
    gx, gf = run.offspring()
    t = run.t - 1
    assert_rollout_objectives(gf.cpu().numpy(), orc.evaluate(p, gx.cpu().numpy().astype(np.float64), t, nd))
    run.sync_status()
