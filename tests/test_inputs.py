"""The seeded input recipe: each generator produces the stated shape of its
workload (density, lattice and vacancies, zero momentum and the exact kinetic
energy, chain geometry and block types, the ensemble's distributions), and the
same seed gives the same arrays."""
import math

import numpy as np
import pytest

from paper_1412_3387_gb300 import inputs


def _ke(v):
    return 0.5 * float(np.sum(v[:, :3] ** 2))


@pytest.mark.parametrize("n, m", ((4000, 10), (5000, 11), (4 * 7 ** 3, 7), (4 * 7 ** 3 + 1, 8)))
def test_lj_fluid_lattice_density_and_velocities(n, m):
    st = inputs.lj_fluid(n, 0.8442, 1.44, seed=3)
    L = st.box[0, 0]
    assert st.n == n and st.n_replicas == 1
    assert math.isclose(L ** 3, n / 0.8442, rel_tol=1e-12)
    x = st.pos[:, :3]
    assert np.all(x >= 0) and np.all(x < L)
    # every particle on a site of the m^3-cell fcc lattice (a = L / m): the
    # coordinates are (integer or half-integer + 1/4) lattice constants
    a = L / m
    u = x / a - 0.25
    assert np.allclose(2 * u, np.rint(2 * u), atol=1e-9)
    # no two particles on one site; 4 m^3 - n seeded vacancies
    keys = np.rint(2 * u).astype(np.int64)
    assert len({tuple(k) for k in keys}) == n
    assert 4 * m ** 3 - n >= 0 and 4 * (m - 1) ** 3 < n
    v = st.vel[:, :3]
    assert np.allclose(v.sum(axis=0), 0.0, atol=1e-9)
    assert math.isclose(_ke(st.vel), 0.5 * (3 * n - 3) * 1.44, rel_tol=1e-12)
    assert np.array_equal(st.tag, np.arange(n)) and not st.type.any()


def test_headline_lattice_size():
    """16,777,216 particles: a 162^3-cell fcc lattice (4 x 162^3 sites) with
    228,896 vacancies (4 x 256^3 would be 67,108,864 particles)."""
    n = 16_777_216
    m = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
    assert m == 162 and 4 * m ** 3 - n == 228_896 and 4 * 161 ** 3 < n


def test_jitter_stays_within_its_bound():
    st0 = inputs.lj_fluid(4000, 0.8442, 1.0, seed=5)
    st1 = inputs.lj_fluid(4000, 0.8442, 1.0, seed=5, jitter=0.1)
    L = st0.box[0, 0]
    a = L / 10
    d = st1.pos[:, :3] - st0.pos[:, :3]
    d -= L * np.rint(d / L)
    assert np.all(np.abs(d) <= 0.1 * a + 1e-12) and np.abs(d).max() > 0.05 * a


def test_dpd_fluid_uniform_at_density_three():
    n = 30000
    st = inputs.dpd_fluid(n, 3.0, 1.0, seed=8)
    L = st.box[0, 0]
    assert math.isclose(L ** 3, n / 3.0, rel_tol=1e-12)
    x = st.pos[:, :3]
    assert np.all(x >= 0) and np.all(x < L)
    # uniform: each octant holds n/8 particles within a few standard deviations
    octant = (x >= L / 2).astype(int) @ np.array([1, 2, 4])
    counts = np.bincount(octant, minlength=8)
    assert np.all(np.abs(counts - n / 8) < 5 * math.sqrt(n / 8))
    assert math.isclose(_ke(st.vel), 0.5 * (3 * n - 3) * 1.0, rel_tol=1e-12)
    assert np.allclose(st.vel[:, :3].sum(axis=0), 0.0, atol=1e-9)


def test_diblock_melt_chains_bonds_and_blocks():
    n_chains, n_beads = 64, 32
    st = inputs.diblock_melt(n_chains, n_beads, 3.0, 1.0, seed=4)
    n = n_chains * n_beads
    L = st.box[0, 0]
    assert st.n == n and math.isclose(L ** 3, n / 3.0, rel_tol=1e-12)
    # bonds join consecutive beads of each chain, by tag
    assert st.bonds.shape == (n_chains * (n_beads - 1), 2)
    assert np.all(st.bonds[:, 1] == st.bonds[:, 0] + 1)
    assert np.all(st.bonds[:, 0] % n_beads != n_beads - 1)
    # the unwrapped bond vectors have length 0.9
    x = st.pos[:, :3] + st.image[:, :3] * L
    d = x[st.bonds[:, 1]] - x[st.bonds[:, 0]]
    assert np.allclose(np.linalg.norm(d, axis=1), 0.9, rtol=1e-12)
    # wrapped positions in the box; the first half of each chain is A (0)
    assert np.all(st.pos[:, :3] >= 0) and np.all(st.pos[:, :3] < L)
    t = st.type.reshape(n_chains, n_beads)
    assert np.all(t[:, :16] == 0) and np.all(t[:, 16:] == 1)


def test_replica_ensemble_distributions():
    st = inputs.replica_ensemble(256, seed=11)
    R = st.n_replicas
    assert R == 256 and st.offsets[0] == 0 and st.offsets[-1] == st.n
    sizes = np.diff(st.offsets)
    assert np.all(sizes >= 2000) and np.all(sizes <= 64000)
    # log-uniform: the median of ln N near the middle of [ln 2000, ln 64000]
    mid = 0.5 * (math.log(2000) + math.log(64000))
    assert abs(np.median(np.log(sizes)) - mid) < 0.35
    rho = sizes / np.prod(st.box, axis=1)
    assert np.all(rho >= 0.70 - 1e-12) and np.all(rho <= 0.90 + 1e-12)
    assert np.allclose(rho, st.meta["rho"], rtol=1e-12)
    T = np.array(st.meta["T"])
    assert np.all(T >= 0.8) and np.all(T <= 1.5)
    for r in (0, 17, 255):
        sub = inputs.select_replica(st, r)
        assert math.isclose(_ke(sub.vel), 0.5 * (3 * sub.n - 3) * T[r], rel_tol=1e-12)
        assert np.all(sub.pos[:, :3] < sub.box[0, 0]) and np.all(sub.pos[:, :3] >= 0)


def test_same_seed_same_arrays_other_seed_other_arrays():
    a = inputs.lj_fluid(5000, 0.8442, 1.2, seed=9, jitter=0.05)
    b = inputs.lj_fluid(5000, 0.8442, 1.2, seed=9, jitter=0.05)
    c = inputs.lj_fluid(5000, 0.8442, 1.2, seed=10, jitter=0.05)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)
    assert not np.array_equal(a.pos, c.pos)
    d1 = inputs.diblock_melt(8, 32, 3.0, 1.0, seed=2)
    d2 = inputs.diblock_melt(8, 32, 3.0, 1.0, seed=2)
    assert np.array_equal(d1.pos, d2.pos) and np.array_equal(d1.image, d2.image)
