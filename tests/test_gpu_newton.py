"""GPU parity of the half neighbour list with Newton's third law
(md_set_newton, FP64 forms) against the CPU oracle, through the C ABI.

Tolerances: rows are compared as sets (every pair within r_list exactly once,
bit-exact); FP64 forces |dF| <= 1e-12 |F| where |F| >= 1e-2 S, else
|dF| <= 1e-14 S (the atomic adds of the partner forces change the summation
order from run to run, which this rule absorbs).
"""
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


def fp64_force_check(f_gpu, f_ref, absf, what=""):
    d = np.linalg.norm(f_gpu[:, :3] - f_ref[:, :3], axis=1)
    F = np.linalg.norm(f_ref[:, :3], axis=1)
    big = F >= 1e-2 * absf
    assert np.all(d[big] <= 1e-12 * F[big]), (what, np.max(d[big] / F[big]))
    assert np.all(d[~big] <= 1e-14 * absf[~big] + 1e-300), what


def liquid(n=4000, seed=3):
    st = inputs.lj_fluid(n, 0.8442, 1.2, seed=seed)
    out = oracle.run(st.pos, st.vel, st.image, st.box[0], 300, r_cut=2.5, r_skin=0.3, dt=0.005)
    s2 = st.copy()
    s2.pos, s2.vel, s2.image = out["pos"], out["vel"], out["image"]
    return s2


@pytest.mark.parametrize("w", (1, 2, 8))
def test_half_rows_list_every_pair_once(w):
    st = liquid()
    L = st.box[0]
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005)
    s.set_newton(True)
    s.set_tuning(md.KERNEL_PAIR, 128, w)
    s.set_tuning(md.KERNEL_NLIST, 128, 1)
    s.prepare()
    counts, rows = (x.cpu().numpy() for x in s.nlist())
    s.check_error()
    cb, rb = oracle.neighbors(st.pos, L, 2.8, max_nb=256, method="brute")
    want = {(i, int(j)) for i in range(st.n) for j in rb[i, :cb[i]] if i < j}
    got = []
    for i in range(st.n):
        for j in rows[i, :counts[i]]:
            got.append((min(i, int(j)), max(i, int(j))))
    assert len(got) == len(set(got)), "a pair listed twice"
    assert set(got) == want
    assert counts.sum() * 2 == cb.sum()


@pytest.mark.parametrize("w", (1, 2, 4))
def test_half_list_lj_forces_energy_virial(w):
    st = liquid()
    L = st.box[0]
    ref, vref, absf = oracle.lj_forces(st.pos, L, 2.5, shift_energy=True)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, shift_energy=True)
    s.set_newton(True)
    s.set_tuning(md.KERNEL_PAIR, 128, w)
    s.prepare()
    s.compute_pair(want_virial=True)
    f, v = (x.cpu().numpy() for x in s.forces(virial=True))
    s.check_error()
    fp64_force_check(f, ref, absf, f"w={w}")
    assert np.allclose(f[:, 3], ref[:, 3], rtol=1e-12, atol=1e-12 * absf.max())
    assert np.allclose(v, vref, rtol=1e-11, atol=1e-12 * absf.max())
    # switching back gives the full rows and the same forces
    s.set_newton(False)
    s.prepare()
    f2 = s.forces().cpu().numpy()
    fp64_force_check(f2, ref, absf, "full again")


def test_half_list_dpd_forces_match_oracle():
    st = inputs.dpd_fluid(3001, 3.0, 1.0, seed=31)
    L = st.box[0]
    step, seed = 12345, 0xDEADBEEF12
    coeff = [[25.0, 4.5]]
    ref, _, absf = oracle.dpd_forces(st.pos, st.vel, L, 1.0, coeff, 1.0, 0.02, step, seed)
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=coeff, kT=1.0,
                    seed=seed)
    s.set_newton(True)
    s.set_step(step)
    s.prepare()
    f = s.forces().cpu().numpy()
    s.check_error()
    fp64_force_check(f, ref, absf, "dpd")


def test_half_list_fp64_trajectory_and_batched_replicas():
    # a 100-step FP64 run in graphs with sorts, against the oracle's MD loop
    st = inputs.lj_fluid(4000, 0.8442, 1.44, seed=21, jitter=0.05)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 100, r_cut=2.5, r_skin=0.3, dt=0.005,
                     shift_energy=True, thermo_period=10)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, shift_energy=True, thermo_period=10,
                    graph_steps=50, sort_period=1)
    s.set_newton(True)
    s.prepare()
    th = s.run_with_thermo(100).cpu().numpy()[:, 0, :]
    s.check_error()
    g = s.state_numpy()
    by_tag = np.argsort(g["tag"])
    x0 = out["pos"][:, :3] + out["image"][:, :3] * L
    x1 = (g["pos"][:, :3] + g["image"][:, :3] * L)[by_tag]
    assert np.max(np.abs(x1 - x0)) < 1e-9
    assert np.allclose(th, out["thermo"], rtol=1e-9, atol=1e-9)
    # several replicas in one system: each replica's forces against the oracle
    ens = inputs.replica_ensemble(6, seed=5, jitter=0.05)
    sb = md.MDSystem(ens, r_cut=2.5, r_skin=0.3, dt=0.005)
    sb.set_newton(True)
    sb.prepare()
    fb = sb.forces().cpu().numpy()
    sb.check_error()
    for r in range(ens.n_replicas):
        a, b = ens.offsets[r], ens.offsets[r + 1]
        ref, _, absf = oracle.lj_forces(ens.pos[a:b], ens.box[r], 2.5)
        fp64_force_check(fb[a:b], ref, absf, f"replica {r}")


def test_half_list_refused_for_mixed_precision():
    st = liquid(n=2000, seed=4)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, precision="mixed")
    with pytest.raises(md.MDError):
        s.set_newton(True)
    s.set_newton(False)  # the full list stays available
