"""GPU parity of the Gaussian, Morse and Yukawa pairs (Sec. 3 lists them
among the supported pair potentials) through the C ABI, against the CPU
oracle on the same seeded inputs.  Same tolerances as the LJ tests:
  * FP64 forces: |dF| <= 1e-12 |F| where |F| >= 1e-2 S, else |dF| <= 1e-14 S;
  * mixed forces: RMS relative error <= 1e-5, max <= 1e-3 over particles with
    |F| >= 1e-2 S.
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

# one type; and two types whose cross coefficients differ from both diagonals
ONE = {"gauss": [[1.0, 1.0]], "morse": [[1.0, 2.0, 1.1]], "yukawa": [[1.0, 1.0]]}
TWO = {
    "gauss": [[[1.0, 1.0], [1.5, 0.9]], [[1.5, 0.9], [0.7, 1.2]]],
    "morse": [[[1.0, 2.0, 1.1], [0.6, 1.5, 1.0]], [[0.6, 1.5, 1.0], [1.3, 2.5, 1.2]]],
    "yukawa": [[[1.0, 1.0], [2.0, 0.8]], [[2.0, 0.8], [0.5, 1.5]]],
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1412_3387_gb300 import build
    build.build()
    oracle.build()


_EQ = {}


def liquid(n=4000):
    """An LJ liquid snapshot produced by the oracle (never by the CUDA path)."""
    if n not in _EQ:
        st = inputs.lj_fluid(n, 0.8442, 1.2, seed=3)
        out = oracle.run(st.pos, st.vel, st.image, st.box[0], 400, r_cut=2.5, r_skin=0.3,
                         dt=0.005)
        s2 = st.copy()
        s2.pos, s2.vel, s2.image = out["pos"], out["vel"], out["image"]
        _EQ[n] = s2
    return _EQ[n].copy()


def fp64_force_check(f_gpu, f_ref, absf, what=""):
    d = np.linalg.norm(f_gpu[:, :3] - f_ref[:, :3], axis=1)
    F = np.linalg.norm(f_ref[:, :3], axis=1)
    big = F >= 1e-2 * absf
    assert np.all(d[big] <= 1e-12 * F[big]), (what, np.max(d[big] / F[big]))
    assert np.all(d[~big] <= 1e-14 * absf[~big] + 1e-300), what


def mixed_force_stats(f_gpu, f_ref, absf):
    d = np.linalg.norm(f_gpu[:, :3] - f_ref[:, :3], axis=1)
    F = np.linalg.norm(f_ref[:, :3], axis=1)
    big = (F >= 1e-2 * absf) & (absf > 0)
    rel = d[big] / F[big]
    return float(np.sqrt(np.mean(rel ** 2))), float(rel.max())


@pytest.mark.parametrize("pair", ("gauss", "morse", "yukawa"))
@pytest.mark.parametrize("prec", ("fp64", "mixed"))
@pytest.mark.parametrize("w", (1, 4))
def test_forces_energy_virial_match_oracle(pair, prec, w):
    st = liquid()
    L = st.box[0]
    ref, vref, absf = oracle.pair_forces(pair, st.pos, L, 2.5, ONE[pair], shift_energy=True)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair=pair, coeff=ONE[pair],
                    precision=prec, shift_energy=True)
    s.set_tuning(md.KERNEL_PAIR, 128, w)
    s.prepare()
    s.compute_pair(want_virial=True)
    f, v = (x.cpu().numpy() for x in s.forces(virial=True))
    s.check_error()
    if prec == "fp64":
        fp64_force_check(f, ref, absf, f"{pair} w={w}")
        assert np.allclose(f[:, 3], ref[:, 3], rtol=1e-12, atol=1e-12 * absf.max())
        assert np.allclose(v, vref, rtol=1e-11, atol=1e-12 * absf.max())
    else:
        rms, mx = mixed_force_stats(f, ref, absf)
        assert rms <= 1e-5 and mx <= 1e-3, (pair, rms, mx)
        assert abs(f[:, 3].sum() - ref[:, 3].sum()) <= 1e-5 * np.abs(ref[:, 3]).sum()
        assert abs(v[:, [0, 3, 5]].sum() - vref[:, [0, 3, 5]].sum()) <= 1e-5 * np.abs(vref).sum()


@pytest.mark.parametrize("pair", ("gauss", "morse", "yukawa"))
@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_two_types_index_coefficients_by_type_pair(pair, prec):
    st = liquid()
    st.type = (np.arange(st.n) % 3 == 0).astype(np.int32)
    L = st.box[0]
    ref, _, absf = oracle.pair_forces(pair, st.pos, L, 2.5, TWO[pair], type=st.type)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair=pair, coeff=TWO[pair],
                    precision=prec)
    s.set_tuning(md.KERNEL_PAIR, 128, 2)
    s.prepare()
    s.compute_pair()
    f = s.forces().cpu().numpy()
    s.check_error()
    if prec == "fp64":
        fp64_force_check(f, ref, absf, pair)
    else:
        rms, mx = mixed_force_stats(f, ref, absf)
        assert rms <= 1e-5 and mx <= 1e-3, (pair, rms, mx)


def test_morse_fp64_trajectory_matches_oracle():
    """100 FP64 steps of a Morse liquid (graphs with thermo closes) against the
    oracle's MD loop: positions within 1e-9, thermo rows within 1e-9."""
    st = inputs.lj_fluid(4000, 0.8442, 1.0, seed=8, jitter=0.05)
    L = st.box[0]
    c = [[0.5, 2.0, 1.15]]
    out = oracle.run(st.pos, st.vel, st.image, L, 100, r_cut=2.5, r_skin=0.3, dt=0.004,
                     pair="morse", coeff=c, shift_energy=True, thermo_period=10)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.004, pair="morse", coeff=c,
                    shift_energy=True, thermo_period=10, graph_steps=50)
    s.prepare()
    th = s.run_with_thermo(100).cpu().numpy()[:, 0, :]
    s.check_error()
    g = s.state_numpy()
    x0 = out["pos"][:, :3] + out["image"][:, :3] * L
    x1 = g["pos"][:, :3] + g["image"][:, :3] * L
    assert np.max(np.abs(x1 - x0)) < 1e-9
    assert np.allclose(th, out["thermo"], rtol=1e-9, atol=1e-9)


def test_bad_coefficients_are_refused():
    st = liquid()
    with pytest.raises(ValueError):
        md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair="morse", coeff=[[1.0, 2.0]])
    with pytest.raises(ValueError):
        md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair="cosine", coeff=[[1.0, 2.0]])
    with pytest.raises(Exception):
        md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair="yukawa",
                    coeff=[[1.0, float("nan")]])


def lj_table(n_points, r_min, r_cut, eps=1.0, sigma=1.0):
    """(V, F) samples of LJ on the table grid (the table's input)."""
    r = r_min + (r_cut - r_min) * np.arange(n_points) / (n_points - 1)
    out = np.zeros((n_points, 2))
    for j, x in enumerate(r):
        fr, v = oracle.lj_pair(x * x, eps, sigma)
        out[j] = (v, fr * x)
    return out


@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_tabulated_pair_matches_oracle(prec):
    """A tabulated pair (Sec. 3) with two types: the GPU interpolates the same
    samples as the oracle (forces, energies, virials; the 1e-12 rule for FP64,
    the mixed tolerance for FP32)."""
    st = liquid()
    st.type = (np.arange(st.n) % 4 == 0).astype(np.int32)
    L = st.box[0]
    n_points, r_min = 1201, 0.6
    tab = np.zeros((2, 2, n_points, 2))
    for a, b, eps in ((0, 0, 1.0), (0, 1, 0.8), (1, 0, 0.8), (1, 1, 1.3)):
        tab[a, b] = lj_table(n_points, r_min, 2.5, eps=eps)
    ref, vref, absf = oracle.table_forces(st.pos, L, 2.5, tab, r_min, type=st.type)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair="table", table_points=n_points,
                    n_types=2, precision=prec)
    s.set_pair_table(tab, r_min)
    s.set_tuning(md.KERNEL_PAIR, 128, 2)
    s.prepare()
    s.compute_pair(want_virial=True)
    f, v = (x.cpu().numpy() for x in s.forces(virial=True))
    s.check_error()
    if prec == "fp64":
        fp64_force_check(f, ref, absf, "table")
        assert np.allclose(f[:, 3], ref[:, 3], rtol=1e-12, atol=1e-12 * absf.max())
        assert np.allclose(v, vref, rtol=1e-11, atol=1e-12 * absf.max())
    else:
        rms, mx = mixed_force_stats(f, ref, absf)
        assert rms <= 1e-5 and mx <= 1e-3, (rms, mx)
    # a run on the table stays close to LJ's own energy scale and reports no error
    s.run(20)
    s.check_error()


def test_table_arguments_are_checked():
    st = liquid(n=2000)
    with pytest.raises(md.MDError):  # no sample count
        md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair="table", n_types=1)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, pair="table", table_points=10,
                    n_types=1)
    with pytest.raises(md.MDError):
        s.set_pair_table(np.zeros((1, 1, 10, 2)), 2.6)  # r_min beyond r_cut
    with pytest.raises(md.MDError):
        s.set_pair_table(np.full((1, 1, 10, 2), np.nan), 0.5)
    s.set_pair_table(np.zeros((1, 1, 10, 2)), 0.5)
