"""Pins of the oracle's whole generation (Algorithm 2) and of the
neuroevolution objective.

- the generation is the composition of its operators (mating -> SBX ->
  mutation -> evaluation -> selection), checked piece by piece;
- results do not depend on the oracle's thread count;
- reference vectors change only on adaptation generations;
- free-running quality: on DTLZ2 (m=3, d=12, N=105) the IGD to the unit-sphere
  front falls well below its initial value in 100 generations;
- the rollout objective reduces to closed forms when the policy is constant.
"""
import numpy as np
import pytest
from scipy import stats


def _small(orc, **kw):
    base = dict(m=3, d=12, N=105, H=13, problem=orc.DTLZ2, t_max=100, alpha=2.0,
                f_r=0.1, seed=3)
    base.update(kw)
    return orc.make_params(**base)


def igd(F, front):
    d = np.linalg.norm(front[:, None, :] - F[None, :, :], axis=2)
    return d.min(1).mean()


def test_generation_is_composition(orc):
    """Algorithm 2's loop body glues the separately pinned operators in the
    paper's order: mating, SBX, mutation, evaluation, selection of the union
    of parents and children, the survivors into their vectors' slots."""
    p = _small(orc)
    V0, st = orc.initial_state(p)
    for _ in range(3):
        orc.generation(p, V0, st)
    before = orc.State(st.X, st.F, st.valid, st.V, st.gamma, st.t)
    t = st.t
    out = orc.generation(p, V0, st)
    vlist = np.nonzero(before.valid)[0].astype(np.int32)
    par = orc.mating(p, t, vlist)
    assert np.array_equal(par, out["parents"])
    P = (p.N + 1) // 2
    Xc = orc.sbx(p, t, before.X[par[:P]], before.X[par[P:]])
    Xm, _ = orc.mutation(p, t, Xc)
    assert np.array_equal(Xm, out["Xchild"])
    Fc = orc.evaluate(p, Xm, t)
    assert np.array_equal(Fc, out["Fchild"])
    Fall = np.concatenate([before.F, Fc])
    vall = np.concatenate([before.valid, np.ones(p.N, np.uint8)])
    sel = orc.select(np.nan_to_num(Fall, nan=0.0), vall, before.V, before.gamma, t,
                     p.t_max, p.alpha)
    assert np.array_equal(sel["survivor"], out["survivor"])
    for j, i in enumerate(out["survivor"]):
        if i < 0:
            assert st.valid[j] == 0
        else:
            src = before.X[i] if i < p.N else Xm[i - p.N]
            assert np.array_equal(st.X[j], src)


def test_thread_count_invariance(orc):
    p = _small(orc, d=40, N=210, H=19)
    res = []
    for th in (1, 4):
        orc.set_threads(th)
        V0, st = orc.initial_state(p)
        for _ in range(12):
            orc.generation(p, V0, st)
        res.append(st)
    orc.set_threads(1)
    a, b = res
    assert np.array_equal(a.X, b.X, equal_nan=True)
    assert np.array_equal(a.F, b.F, equal_nan=True)
    assert np.array_equal(a.V, b.V)


def test_adaptation_schedule(orc):
    p = _small(orc, t_max=30, f_r=0.2)       # period 6
    assert orc.adapt_period(p) == 6
    V0, st = orc.initial_state(p)
    prev = st.V.copy()
    for t in range(1, 19):
        orc.generation(p, V0, st)
        changed = not np.array_equal(prev, st.V)
        assert changed == (t % 6 == 0), t
        if changed:
            rng = orc.objective_range(st.F, st.valid)
            assert np.array_equal(st.V, orc.adapt(V0, rng))
            assert np.array_equal(st.gamma, orc.gamma(st.V))
        prev = st.V.copy()


def test_free_running_quality_dtlz2(orc):
    p = _small(orc)
    V0, st = orc.initial_state(p)
    front = orc.lattice_unit(orc.lattice(3, 30))
    igd0 = igd(st.F, front)
    for _ in range(100):
        out = orc.generation(p, V0, st)
    F = st.F[st.valid == 1]
    igd1 = igd(F, front)
    assert igd1 < 0.1 < igd0, (igd0, igd1)
    assert out["alive"] >= 90


def test_neuro_noise_is_standard_normal(orc):
    p = orc.make_params(m=2, d=5702, N=100, H=99, problem=orc.NEURO, seed=11)
    nd = orc.NeuroData(np.zeros((17, 17)), np.zeros((17, 6)), steps=2000)
    xi = orc.neuro_noise(p, nd, 4)
    assert stats.kstest(xi.ravel(), "norm").pvalue > 1e-3
    w = orc.philox([0, 0, 4, orc.TAG_NOISE], [11, 0])
    u1 = 1 - (w[0] >> 8) / 2 ** 24
    u2 = (w[1] >> 8) / 2 ** 24
    assert np.isclose(xi[0, 0], np.sqrt(-2 * np.log(u1)) * np.cos(2 * np.pi * u2))


def _policy(b3, ns=17, na=6, h=64):
    x = np.zeros(h * ns + h + h * h + h + na * h + na)
    x[-na:] = b3
    return x


@pytest.mark.parametrize("a", [0.0, 0.5])
def test_neuro_constant_policy_closed_form(orc, a):
    steps = 50
    rng = np.random.default_rng(2)
    B = rng.normal(size=(17, 6))
    c = rng.normal(size=6)
    u = np.tanh(c)
    nd = orc.NeuroData(a * np.eye(17), B, steps=steps, sigma=0.0)
    p = orc.make_params(m=2, d=5702, N=1, H=1, problem=orc.NEURO, L=-1, U=1)
    F = orc.evaluate(p, _policy(c)[None, :], 1, nd)
    Bu0 = (B @ u)[0]
    tau = np.arange(1, steps + 1)
    s0 = Bu0 * (1 - a ** tau) / (1 - a)          # geometric series of s[0]
    assert np.isclose(F[0, 0], -s0.sum(), rtol=1e-12)
    assert np.isclose(F[0, 1], steps * (u @ u), rtol=1e-12)


def test_neuro_layer_layout(orc):
    # one path through every layer: s has only noise in component 3 at step 0;
    # W1[0,3], W2[0,0], W3[2,0] carry it to u[2] at step 1; B[0,2] to s[0].
    ns, na, h = 17, 6, 64
    x = np.zeros(h * ns + h + h * h + h + na * h + na)
    W1 = x[: h * ns].reshape(h, ns)
    o = h * ns + h
    W2 = x[o: o + h * h].reshape(h, h)
    o += h * h + h
    W3 = x[o: o + na * h].reshape(na, h)
    W1[0, 3], W2[0, 0], W3[2, 0] = 0.8, 0.7, 0.6
    B = np.zeros((17, 6))
    B[0, 2] = 1.0
    nd = orc.NeuroData(np.zeros((17, 17)), B, steps=2, sigma=0.01)
    p = orc.make_params(m=2, d=5702, N=1, H=1, problem=orc.NEURO, seed=5)
    xi = orc.neuro_noise(p, nd, 1)
    F = orc.evaluate(p, x[None, :], 1, nd)
    s1 = 0.01 * xi[0]                               # u_0 = 0
    u1 = np.tanh(0.6 * np.tanh(0.7 * np.tanh(0.8 * s1[3])))
    s2_0 = u1 + 0.01 * xi[1, 0]
    assert np.isclose(F[0, 0], -(s1[0] + s2_0), rtol=1e-12)
    assert np.isclose(F[0, 1], u1 ** 2, rtol=1e-12)
