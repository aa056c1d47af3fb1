"""GPU parity of FENE bonds (md_set_bond_style; Sec. 3 lists FENE bonds)
against the CPU oracle, through the C ABI: the diblock melt with its bonds
as FENE springs (K = 30, R0 = 1.5) plus the DPD pair forces.  Tolerances as
in the other parity tests (FP64: the 1e-12 rule; mixed: RMS 1e-5, max 1e-3).
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

K, R0 = 30.0, 1.5
COEFF = np.array([[[25.0, 4.5], [40.0, 4.5]], [[40.0, 4.5], [25.0, 4.5]]])


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


@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_fene_bonds_and_dpd_match_oracle(prec):
    st = inputs.diblock_melt(64, 32, 3.0, 1.0, seed=41)
    L = st.box[0]
    step, seed = 7, 99
    ref, vref, absf = oracle.dpd_forces(st.pos, st.vel, L, 1.0, COEFF, 1.0, 0.02, step, seed,
                                        type=st.type)
    ref, vref, absf, broken = oracle.fene_bond_forces(st.bonds, st.pos, L, K, R0, ref, vref,
                                                      absf)
    assert broken == 0
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=COEFF, kT=1.0,
                    seed=seed, precision=prec, bond_K=K, bond_r0=R0)
    s.set_bond_style("fene")
    s.set_step(step)
    s.prepare()
    s.compute_forces(want_virial=True)
    f, v = (x.cpu().numpy() for x in s.forces(virial=True))
    s.check_error()
    if prec == "fp64":
        fp64_force_check(f, ref, absf)
        assert np.allclose(f[:, 3], ref[:, 3], rtol=1e-12, atol=1e-12 * absf.max())
        assert np.allclose(v, vref, rtol=1e-11, atol=1e-12 * absf.max())
    else:
        d = np.linalg.norm(f[:, :3] - ref[:, :3], axis=1)
        F = np.linalg.norm(ref[:, :3], axis=1)
        big = (F >= 1e-2 * absf) & (absf > 0)
        rel = d[big] / F[big]
        assert np.sqrt(np.mean(rel ** 2)) <= 1e-5 and rel.max() <= 1e-3


def test_fene_fp64_trajectory_matches_oracle():
    """50 FP64 steps of the FENE diblock melt (pair LJ-free: DPD noise needs
    the same keys on both sides) against the oracle's MD loop."""
    st = inputs.diblock_melt(32, 32, 3.0, 1.0, seed=43)
    L = st.box[0]
    seed = 5
    out = oracle.run(st.pos, st.vel, st.image, L, 50, r_cut=1.0, r_skin=0.3, dt=0.01,
                     pair="dpd", type=st.type, coeff=COEFF, kT=1.0, seed=seed, bonds=st.bonds,
                     K=K, r0=R0, bond_style="fene", max_nb=192)
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.01, pair="dpd", coeff=COEFF, kT=1.0,
                    seed=seed, bond_K=K, bond_r0=R0, max_nb=192)
    s.set_bond_style("fene")
    s.prepare()
    s.run(50)
    s.check_error()
    g = s.state_numpy()
    x0 = out["pos"][:, :3] + out["image"][:, :3] * L
    x1 = g["pos"][:, :3] + g["image"][:, :3] * L
    assert np.max(np.abs(x1 - x0)) < 1e-8


def test_overstretched_fene_bond_is_reported():
    st = inputs.diblock_melt(8, 32, 3.0, 1.0, seed=47)
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=COEFF, kT=1.0,
                    bond_K=K, bond_r0=0.8)  # the chains' bonds are 0.9 long
    s.set_bond_style("fene")
    s.prepare()
    code, detail = s.poll_error()
    assert code == 10, (code, detail)
    assert 0 <= detail < st.n
    with pytest.raises(md.MDError):
        md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=COEFF, kT=1.0,
                    bond_K=K, bond_r0=0.0).set_bond_style("fene")


def chain_angles(n_chains, length):
    """Consecutive triplets of each chain (tags), vertex in the middle."""
    return np.array([[c * length + k, c * length + k + 1, c * length + k + 2]
                     for c in range(n_chains) for k in range(length - 2)], np.int32)


@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_angles_with_fene_bonds_match_oracle(prec):
    """Harmonic angles (Sec. 3) on the diblock chains, with FENE bonds and the
    DPD pair forces, against the oracle; then after a sort (per-particle angle
    tables are keyed by tag)."""
    st = inputs.diblock_melt(64, 32, 3.0, 1.0, seed=41)
    L = st.box[0]
    tri = chain_angles(64, 32)
    Ka, th0 = 6.0, 2.2
    step, seed = 7, 99
    ref, vref, absf = oracle.dpd_forces(st.pos, st.vel, L, 1.0, COEFF, 1.0, 0.02, step, seed,
                                        type=st.type)
    ref, vref, absf, _ = oracle.fene_bond_forces(st.bonds, st.pos, L, K, R0, ref, vref, absf)
    ref, vref, absf = oracle.angle_forces(tri, st.pos, L, Ka, th0, ref, vref, absf)
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=COEFF, kT=1.0,
                    seed=seed, precision=prec, bond_K=K, bond_r0=R0, max_angles=3)
    s.set_bond_style("fene")
    s.set_angles(tri, Ka, th0)
    s.set_step(step)
    s.prepare()
    s.compute_forces(want_virial=True)
    f, v = (x.cpu().numpy() for x in s.forces(virial=True))
    s.check_error()
    if prec == "fp64":
        fp64_force_check(f, ref, absf)
        assert np.allclose(f[:, 3], ref[:, 3], rtol=1e-12, atol=1e-12 * absf.max())
        assert np.allclose(v, vref, rtol=1e-11, atol=1e-12 * absf.max())
        # particle arrays sorted along the curve: forces by tag are unchanged
        s2 = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=COEFF, kT=1.0,
                         seed=seed, bond_K=K, bond_r0=R0, max_angles=3)
        s2.set_bond_style("fene")
        s2.set_angles(tri, Ka, th0)
        s2.set_step(step)
        s2.build_cells()
        s2.sort()
        s2.prepare()
        s2.compute_forces()
        tag = s2.tag.cpu().numpy()
        assert not np.array_equal(tag, np.arange(st.n))
        fp64_force_check(s2.forces().cpu().numpy(), ref[tag], absf[tag], "after sort")
    else:
        d = np.linalg.norm(f[:, :3] - ref[:, :3], axis=1)
        F = np.linalg.norm(ref[:, :3], axis=1)
        big = (F >= 1e-2 * absf) & (absf > 0)
        rel = d[big] / F[big]
        assert np.sqrt(np.mean(rel ** 2)) <= 1e-5 and rel.max() <= 1e-3


def test_angles_fp64_trajectory_matches_oracle():
    st = inputs.diblock_melt(32, 32, 3.0, 1.0, seed=43)
    L = st.box[0]
    tri = chain_angles(32, 32)
    out = oracle.run(st.pos, st.vel, st.image, L, 50, r_cut=1.0, r_skin=0.3, dt=0.01,
                     pair="dpd", type=st.type, coeff=COEFF, kT=1.0, seed=5, bonds=st.bonds,
                     K=K, r0=R0, bond_style="fene", angles=tri, angle_K=6.0, angle_theta0=2.2,
                     max_nb=192)
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.01, pair="dpd", coeff=COEFF, kT=1.0,
                    seed=5, bond_K=K, bond_r0=R0, max_nb=192, max_angles=3)
    s.set_bond_style("fene")
    s.set_angles(tri, 6.0, 2.2)
    s.prepare()
    s.run(50)
    s.check_error()
    g = s.state_numpy()
    x0 = out["pos"][:, :3] + out["image"][:, :3] * L
    x1 = g["pos"][:, :3] + g["image"][:, :3] * L
    assert np.max(np.abs(x1 - x0)) < 1e-8


def test_angle_arguments_are_checked():
    st = inputs.diblock_melt(8, 32, 3.0, 1.0, seed=47)
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=COEFF, kT=1.0,
                    bond_K=4.0, max_angles=1)
    tri = chain_angles(8, 32)
    with pytest.raises(md.MDError):   # a middle bead is in three angles
        s.set_angles(tri, 1.0, 2.0)
    with pytest.raises(md.MDError):
        s.set_angles([[0, 0, 1]], 1.0, 2.0)
    with pytest.raises(md.MDError):
        s.set_angles([[0, 1, 2]], 1.0, 4.0)  # theta0 beyond pi
    s.set_angles([[0, 1, 2]], 1.0, 2.0)
