"""GPU parity of the thermostatted integrators (md_set_integrator) against
the CPU oracle on the same seeded inputs:

  * Langevin (BAOAB; the per-particle noise from Philox-4x32-10 keyed on
    (tag, step, seed) is bit-identical on both sides): FP64 trajectory through
    md_run's CUDA graphs, sorted at every rebuild, within 1e-9 by tag;
  * Nose-Hoover (one thermostat, MTK splitting, one kinetic-energy sum per
    step): FP64 trajectory, thermostat state (xi, eta) and thermo rows;
    batched replicas each with their own thermostat equal standalone runs;
  * both forms in mixed precision hold the target temperature, and the
    Nose-Hoover extended energy is conserved as well as the oracle conserves
    it over the same run;
  * argument errors.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1412_3387_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3387_gb300 import md  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1412_3387_gb300 import build
    build.build()
    oracle.build()


def by_tag(g, L):
    x = g["pos"][:, :3] + g["image"][:, :3] * L
    xo, vo = np.empty_like(x), np.empty_like(x)
    xo[g["tag"]] = x
    vo[g["tag"]] = g["vel"][:, :3]
    return xo, vo


@pytest.mark.parametrize("graph", (0, 50))
def test_langevin_fp64_trajectory_matches_oracle(graph):
    st = inputs.lj_fluid(4000, 0.8442, 1.0, seed=51, jitter=0.05)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 100, r_cut=2.5, r_skin=0.3, dt=0.005,
                     integrator="langevin", gamma=2.0, t_kT=1.5, t_seed=77, thermo_period=10)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, thermo_period=10, graph_steps=graph,
                    sort_period=1)
    s.set_integrator("langevin", kT=1.5, param=2.0, seed=77)
    s.prepare()
    th = s.run_with_thermo(100).cpu().numpy()[:, 0, :]
    s.check_error()
    x, v = by_tag(s.state_numpy(), L)
    assert np.max(np.abs(x - (out["pos"][:, :3] + out["image"][:, :3] * L))) < 1e-9
    assert np.max(np.abs(v - out["vel"][:, :3])) < 1e-8
    assert np.allclose(th[:, [0, 4]], out["thermo"][:, [0, 4]], rtol=1e-9)


@pytest.mark.parametrize("graph", (0, 50))
def test_nose_hoover_fp64_trajectory_matches_oracle(graph):
    st = inputs.lj_fluid(4000, 0.8442, 0.9, seed=52, jitter=0.05)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 100, r_cut=2.5, r_skin=0.3, dt=0.005,
                     shift_energy=True, integrator="nose-hoover", tau=0.4, t_kT=1.3,
                     thermo_period=10)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, shift_energy=True, thermo_period=10,
                    graph_steps=graph, sort_period=1)
    s.set_integrator("nose-hoover", kT=1.3, param=0.4)
    s.prepare()
    th = s.run_with_thermo(100).cpu().numpy()[:, 0, :]
    s.check_error()
    x, v = by_tag(s.state_numpy(), L)
    assert np.max(np.abs(x - (out["pos"][:, :3] + out["image"][:, :3] * L))) < 1e-9
    assert np.max(np.abs(v - out["vel"][:, :3])) < 1e-8
    assert np.allclose(th, out["thermo"], rtol=1e-9, atol=1e-9)
    xi_eta = s.thermostat()[0]
    assert np.allclose(xi_eta, out["nh_state"], rtol=1e-9, atol=1e-12)
    assert abs(xi_eta[0]) > 1e-3  # the thermostat was working


def test_nose_hoover_batched_replicas_equal_standalone():
    ens = inputs.replica_ensemble(4, seed=8, n_min=2000, n_max=5000, jitter=0.05)
    kw = dict(r_cut=2.5, r_skin=0.3, dt=0.005, sort_period=1, graph_steps=20, thermo_period=20)
    b = md.MDSystem(ens, **kw)
    b.set_integrator("nose-hoover", kT=1.1, param=0.5)
    b.run(60)
    gb, xb = b.state_numpy(), b.thermostat()
    for r in (0, 3):
        sub = inputs.select_replica(ens, r)
        a = md.MDSystem(sub, **kw)
        a.set_integrator("nose-hoover", kT=1.1, param=0.5)
        a.run(60)
        o0, o1 = ens.offsets[r], ens.offsets[r + 1]
        assert np.array_equal(a.state_numpy()["pos"], gb["pos"][o0:o1]), r
        assert np.array_equal(a.thermostat()[0], xb[r]), r


@pytest.mark.parametrize("kind", ("langevin", "nose-hoover"))
def test_mixed_thermostats_hold_the_temperature(kind):
    """Mixed precision, 8000 particles, kT = 1.25 from a T = 1.1 start: the
    kinetic temperature averaged over steps 1000..6000 equals kT within 2 %.
    The Nose-Hoover temperature oscillates (period about 2 pi tau / sqrt(2)
    ~ 440 steps here, weakly damped), so its mean is taken over ~11 periods
    after the start transient; the FP64 oracle on the same start gives its
    own mean over the same steps, and the two agree within 2 %."""
    st = inputs.lj_fluid(8000, 0.8442, 1.1, seed=53)
    param = 1.0 if kind == "langevin" else 0.5
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, precision="mixed", thermo_period=10,
                    graph_steps=100, sort_period=1)
    s.set_integrator(kind, kT=1.25, param=param, seed=5)
    th = s.run_with_thermo(6000).cpu().numpy()[:, 0, :]
    s.check_error()
    T = np.mean(th[100:, 4])
    assert T == pytest.approx(1.25, rel=0.02)
    if kind == "nose-hoover":
        out = oracle.run(st.pos, st.vel, st.image, st.box[0], 6000, r_cut=2.5, r_skin=0.3,
                         dt=0.005, integrator="nose-hoover", tau=param, t_kT=1.25,
                         thermo_period=10)
        assert T == pytest.approx(np.mean(out["thermo"][100:, 4]), rel=0.02)


@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_nose_hoover_extended_energy_as_conserved_as_the_oracle(prec):
    """H = KE + PE + g kT tau^2 xi^2 / 2 + g kT eta over 1500 steps (thermo
    every 10) from a cold start: its largest deviation on the GPU stays within
    twice the oracle's on the same start (the two trajectories separate, the
    integrator error does not depend on which one)."""
    n, kT, tau, dt = 864, 1.3, 0.3, 0.005
    g = 3 * n - 3
    st = inputs.lj_fluid(n, 0.8442, 0.8, seed=25)
    L = st.box[0]
    kw = dict(r_cut=2.5, r_skin=0.3, dt=dt, shift_energy=True)
    ref, state, nh = [], (st.pos, st.vel, st.image), np.zeros(2)
    for k in range(150):
        out = oracle.run(*state, L, 10, step0=10 * k, nh_state=nh, integrator="nose-hoover",
                         tau=tau, t_kT=kT, thermo_period=10, **kw)
        state, nh = (out["pos"], out["vel"], out["image"]), out["nh_state"]
        ref.append((out["thermo"][-1, 0] + out["thermo"][-1, 1]
                    + g * kT * tau * tau * nh[0] ** 2 / 2 + g * kT * nh[1]) / n)
    s = md.MDSystem(st, precision=prec, thermo_period=10, graph_steps=10, sort_period=1, **kw)
    s.set_integrator("nose-hoover", kT=kT, param=tau)
    H = []
    for k in range(150):
        th = s.run_with_thermo(10).cpu().numpy()[-1, 0]
        xi, eta = s.thermostat()[0]
        H.append((th[0] + th[1] + g * kT * tau * tau * xi ** 2 / 2 + g * kT * eta) / n)
    s.check_error()
    dev, dev_ref = np.abs(np.array(H) - H[0]).max(), np.abs(np.array(ref) - ref[0]).max()
    assert dev < 2.0 * dev_ref, (dev, dev_ref)


def test_set_integrator_argument_errors():
    st = inputs.lj_fluid(2048, 0.8442, 1.0, seed=54)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005)
    for kind, kT, param in (("langevin", -1.0, 1.0), ("langevin", 1.0, -0.5),
                            ("nose-hoover", 1.0, 0.0), ("nose-hoover", 0.0, 1.0)):
        with pytest.raises(md.MDError) as e:
            s.set_integrator(kind, kT=kT, param=param)
        assert e.value.code == 1
    d = md.MDSystem(inputs.dpd_fluid(3000, 3.0, 1.0, seed=1), r_cut=1.0, r_skin=0.3, dt=0.02,
                    pair="dpd", coeff=[[25.0, 4.5]])
    with pytest.raises(md.MDError):
        d.set_integrator("langevin", kT=1.0, param=1.0)
