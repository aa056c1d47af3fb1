"""Pins for the CPU FP64 oracle (no GPU).

Each test checks the oracle against something other than itself: published
known-answer values, closed forms, lattice symmetry, crystallographic shell
counts, conservation laws, brute force on small inputs, or the mathematics of
the integrator.  A plausible slip in the oracle (dropped term, wrong sign,
wrong index, transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1412_3387_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# LJ pair

def test_lj_special_values():
    vals = {"1": 1.0, "2^(1/6)": 2.0 ** (1.0 / 6.0)}
    for q, r, v in _golden_rows("lj_special_values.txt"):
        fr, pot = oracle.lj_pair(vals[r] ** 2)
        got = pot if q == "V" else fr * vals[r]
        assert got == pytest.approx(float(v), abs=1e-13)


def test_lj_scaling_with_eps_and_sigma():
    # V(r; eps, s) = eps V(r/s; 1, 1) and F(r; eps, s) = eps/s F(r/s; 1, 1)
    for eps, s, x in [(2.0, 1.5, 1.1), (0.5, 0.8, 1.7), (3.0, 1.0, 2.4)]:
        fr1, v1 = oracle.lj_pair(x * x)
        frs, vs = oracle.lj_pair((x * s) ** 2, eps, s)
        assert vs == pytest.approx(eps * v1, rel=1e-14)
        assert frs * (x * s) == pytest.approx(eps / s * fr1 * x, rel=1e-14)


def test_lj_two_particles_direction_and_image():
    # particle 1 at distance 1 from particle 0 across the periodic boundary
    L = 10.0
    pos = np.zeros((2, 4))
    pos[0, :3] = [0.3, 5.0, 5.0]
    pos[1, :3] = [L - 0.7, 5.0, 5.0]  # separation x0 - x1 = +1 (minimum image)
    f, vir, absf = oracle.lj_forces(pos, L, 2.5)
    # at r = sigma the pair force has magnitude 24 and is repulsive
    assert f[0, 0] == pytest.approx(24.0, abs=1e-12)
    assert f[1, 0] == pytest.approx(-24.0, abs=1e-12)
    assert np.allclose(f[:, 1:3], 0.0)
    assert f[0, 3] == pytest.approx(0.0, abs=1e-14)  # V(sigma) = 0, half each
    # virial: half of r f per particle (x0 - x1 = +1, f_x = +24)
    assert vir[0, 0] == pytest.approx(12.0, abs=1e-12)
    assert absf[0] == pytest.approx(24.0, abs=1e-12)


def _fcc_shells():
    return [(int(k), int(z)) for k, z in _golden_rows("fcc_shells.txt")]


@pytest.mark.parametrize("rho,r_cut", [(0.8442, 2.5), (1.0, 3.0), (0.7, 2.5)])
def test_lj_perfect_fcc_lattice_sum(rho, r_cut):
    st = inputs.lj_fluid(4 * 6 ** 3, rho, 1.0, seed=1)  # perfect 6^3 lattice
    L = st.box[0, 0]
    a = L / 6
    f, vir, absf = oracle.lj_forces(st.pos, L, r_cut)
    # zero net force on every site by inversion symmetry
    assert np.max(np.abs(f[:, :3])) <= 1e-12 * np.max(absf)
    # energy and virial per particle from the crystallographic shells
    pe, w = 0.0, 0.0
    for k, z in _fcc_shells():
        r = a * math.sqrt(k / 2.0)
        if r >= r_cut:
            continue
        fr, v = oracle.lj_pair(r * r)
        pe += 0.5 * z * v
        w += 0.5 * z * fr * r * r
    assert np.allclose(f[:, 3], pe, rtol=1e-12, atol=1e-13)
    assert np.allclose(vir[:, 0] + vir[:, 3] + vir[:, 5], w, rtol=1e-11, atol=1e-12)
    # neighbour rows: the number of sites inside r_cut is the shell count sum
    counts, _ = oracle.neighbors(st.pos, L, r_cut, max_nb=256)
    z_in = sum(z for k, z in _fcc_shells() if a * math.sqrt(k / 2.0) < r_cut)
    assert np.all(counts == z_in)


def test_lj_newton_third_law_and_shift():
    st = inputs.lj_fluid(500, 0.8442, 1.0, seed=3, jitter=0.08)
    L = st.box[0, 0]
    f, _, absf = oracle.lj_forces(st.pos, L, 2.5)
    assert np.abs(f[:, :3].sum(0)).max() <= 1e-12 * absf.sum()
    fs, _, _ = oracle.lj_forces(st.pos, L, 2.5, shift_energy=True)
    # shifting changes only the energy, by V(r_c) per pair
    assert np.array_equal(fs[:, :3], f[:, :3])
    counts, _ = oracle.neighbors(st.pos, L, 2.5)
    _, vc = oracle.lj_pair(2.5 ** 2)
    assert np.allclose(fs[:, 3], f[:, 3] - 0.5 * counts * vc, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Gaussian, Morse and Yukawa pairs (Sec. 3 lists them; textbook forms)

def test_gauss_morse_yukawa_special_values():
    """Values the definitions fix: the Gaussian's height eps at r -> 0 and half
    height at r = sigma sqrt(2 ln 2), its force eps/sigma e^-1/2 at r = sigma;
    the Morse minimum -D0 at r0 with zero force, its zero at r0 - ln2/alpha
    and -3 D0 / 4 at r0 + ln2/alpha; Yukawa with kappa = 0 is Coulomb
    (V = eps/r, |F| = eps/r^2), and eps kappa / e at r = 1/kappa."""
    eps, sig = 1.7, 0.8
    fr, v = oracle.pair_eval("gauss", 1e-300, [eps, sig])
    assert v == pytest.approx(eps, rel=1e-15)
    fr, v = oracle.pair_eval("gauss", 2 * math.log(2) * sig * sig, [eps, sig])
    assert v == pytest.approx(eps / 2, rel=1e-14)
    fr, v = oracle.pair_eval("gauss", sig * sig, [eps, sig])
    assert fr * sig == pytest.approx(eps / sig * math.exp(-0.5), rel=1e-14)

    d0, al, r0 = 2.5, 1.3, 1.1
    fr, v = oracle.pair_eval("morse", r0 * r0, [d0, al, r0])
    assert v == pytest.approx(-d0, rel=1e-15) and abs(fr) < 1e-15
    fr, v = oracle.pair_eval("morse", (r0 - math.log(2) / al) ** 2, [d0, al, r0])
    assert abs(v) < 1e-14 and fr > 0  # repulsive inside the minimum
    fr, v = oracle.pair_eval("morse", (r0 + math.log(2) / al) ** 2, [d0, al, r0])
    assert v == pytest.approx(-0.75 * d0, rel=1e-14) and fr < 0

    for r in (0.5, 1.0, 2.3):
        fr, v = oracle.pair_eval("yukawa", r * r, [eps, 0.0])
        assert v == pytest.approx(eps / r, rel=1e-15)
        assert fr * r == pytest.approx(eps / r ** 2, rel=1e-14)
    kap = 0.7
    fr, v = oracle.pair_eval("yukawa", 1.0 / kap ** 2, [eps, kap])
    assert v == pytest.approx(eps * kap / math.e, rel=1e-14)


@pytest.mark.parametrize("pair,c", [("gauss", [1.3, 0.9]), ("morse", [2.0, 1.7, 1.05]),
                                    ("yukawa", [0.8, 1.4]), ("lj", [1.0, 1.0])])
def test_pair_force_is_minus_dV_dr(pair, c):
    """-dV/dr by central differences of the oracle's own V equals the force
    factor times r (a wrong sign, power or factor in either fails)."""
    for r in (0.85, 1.0, 1.37, 2.2):
        h = 1e-5
        _, vm = oracle.pair_eval(pair, (r - h) ** 2, c)
        _, vp = oracle.pair_eval(pair, (r + h) ** 2, c)
        fr, _ = oracle.pair_eval(pair, r * r, c)
        assert fr * r == pytest.approx((vm - vp) / (2 * h), rel=1e-7, abs=1e-9)


def test_morse_dimer_oscillation_period():
    """Two Morse particles near r0 oscillate with the harmonic period
    2 pi sqrt(mu / k), k = V''(r0) = 2 D0 alpha^2, mu = m/2 (small amplitude),
    through the oracle's MD loop (pair kind dispatch, force sign)."""
    d0, al, r0 = 1.0, 1.5, 1.2
    L = 12.0
    pos = np.array([[5.0, 6.0, 6.0, 0.0], [5.0 + r0 + 0.01, 6.0, 6.0, 0.0]])
    vel = np.zeros((2, 4))
    img = np.zeros((2, 4), np.int32)
    dt, steps = 0.002, 3000
    k = 2 * d0 * al * al
    period = 2 * math.pi * math.sqrt(0.5 / k)
    seps = []
    p, v, im = pos, vel, img
    for _ in range(steps // 10):
        out = oracle.run(p, v, im, L, 10, r_cut=3.0, r_skin=0.3, dt=dt, pair="morse",
                         coeff=[[d0, al, r0]], max_nb=8)
        p, v, im = out["pos"], out["vel"], out["image"]
        seps.append(p[1, 0] - p[0, 0] - r0)
    seps = np.array(seps)
    t = dt * 10 * np.arange(1, len(seps) + 1)
    up = [t[i] for i in range(1, len(seps)) if seps[i - 1] < 0 <= seps[i]]
    measured = np.mean(np.diff(up))
    assert measured == pytest.approx(period, rel=0.01)


@pytest.mark.parametrize("pair,c,r_cut", [("gauss", [1.0, 1.0], 2.6), ("morse", [1.0, 2.0, 1.1], 2.6),
                                          ("yukawa", [1.0, 1.0], 2.6)])
def test_new_pairs_fcc_lattice_sum(pair, c, r_cut):
    """Brute-force sums on the perfect fcc lattice: zero net force per site
    and the per-site energy and virial of the crystallographic shells."""
    st = inputs.lj_fluid(4 * 6 ** 3, 0.8442, 1.0, seed=1)
    L = st.box[0, 0]
    a = L / 6
    f, vir, absf = oracle.pair_forces(pair, st.pos, L, r_cut, [c])
    assert np.max(np.abs(f[:, :3])) <= 1e-12 * np.max(absf)
    pe, w = 0.0, 0.0
    for k, z in _fcc_shells():
        r = a * math.sqrt(k / 2.0)
        if r >= r_cut:
            continue
        fr, v = oracle.pair_eval(pair, r * r, c)
        pe += 0.5 * z * v
        w += 0.5 * z * fr * r * r
    assert np.allclose(f[:, 3], pe, rtol=1e-12, atol=1e-13)
    assert np.allclose(vir[:, 0] + vir[:, 3] + vir[:, 5], w, rtol=1e-11, atol=1e-12)


def test_pair_forces_lj_kind_equals_lj_forces_and_rows_equal_brute():
    """The generic pair sums with the LJ kind equal the LJ functions bit for
    bit, and the row-driven sums equal the brute-force ones for a new kind."""
    st = inputs.lj_fluid(864, 0.8442, 1.0, seed=4, jitter=0.1)
    L = st.box[0, 0]
    f1, v1, a1 = oracle.lj_forces(st.pos, L, 2.5)
    f2, v2, a2 = oracle.pair_forces("lj", st.pos, L, 2.5, [[1.0, 1.0]])
    assert np.array_equal(f1, f2) and np.array_equal(v1, v2)
    nl = oracle.neighbors(st.pos, L, 2.8, max_nb=128)
    fb, _, absf = oracle.pair_forces("yukawa", st.pos, L, 2.5, [[1.0, 1.0]])
    fn, _, _ = oracle.pair_forces("yukawa", st.pos, L, 2.5, [[1.0, 1.0]], nlist=nl)
    assert np.max(np.abs(fb[:, :3] - fn[:, :3])) <= 1e-13 * np.max(absf)


# --------------------------------------------------------------------------
# Tabulated pair potential (Sec. 3 lists tabulated potentials)

def test_table_reproduces_linear_samples_and_converges_to_lj():
    """Linear interpolation in r is exact for V and F that are linear in r
    (any point, not only samples); below r_min the values at r_min hold; a
    table sampled from LJ converges to LJ with the interpolation error
    O(dr^2) (halving dr quarters it)."""
    rmin, rc, n = 0.8, 2.5, 35
    r = rmin + (rc - rmin) * np.arange(n) / (n - 1)
    tab = np.stack([3.0 - 2.0 * r, 1.5 + 0.25 * r], axis=1)  # V, F = a + b r
    for x in (0.8, 0.93, 1.37777, 2.2, 2.4999):
        fr, v = oracle.table_eval(x * x, tab, rmin, rc)
        assert v == pytest.approx(3.0 - 2.0 * x, rel=1e-14)
        assert fr * x == pytest.approx(1.5 + 0.25 * x, rel=1e-14)
    fr, v = oracle.table_eval(0.5 ** 2, tab, rmin, rc)
    assert v == pytest.approx(3.0 - 2.0 * rmin) and fr * 0.5 == pytest.approx(1.5 + 0.25 * rmin)
    errs = []
    for n in (100, 200):
        r = rmin + (rc - rmin) * np.arange(n) / (n - 1)
        fv = [oracle.lj_pair(x * x) for x in r]
        tab = np.array([[v, f * x] for (f, v), x in zip(fv, r)])
        e = 0.0
        for x in np.linspace(1.0, 2.4, 4001):
            fr, v = oracle.table_eval(x * x, tab, rmin, rc)
            f0, v0 = oracle.lj_pair(x * x)
            e = max(e, abs(fr - f0) * x)
        errs.append(e)
    assert errs[1] == pytest.approx(errs[0] / 4, rel=0.1)


def test_table_sums_on_the_lattice_equal_lj_sums():
    """A fine table sampled from LJ gives the LJ per-site energies on the fcc
    lattice to the interpolation error, and the lattice's symmetry leaves no
    net force (the tabulated pair sums, type indexing and energy split)."""
    rmin, rc = 0.5, 2.5
    st = inputs.lj_fluid(4 * 6 ** 3, 0.8442, 1.0, seed=1)
    L = st.box[0, 0]
    n = 20001
    r = rmin + (rc - rmin) * np.arange(n) / (n - 1)
    fv = [oracle.lj_pair(x * x) for x in r]
    tab = np.array([[[[v, f * x] for (f, v), x in zip(fv, r)]]])
    f_t, vir_t, absf = oracle.table_forces(st.pos, L, rc, tab, rmin)
    f_l, vir_l, _ = oracle.lj_forces(st.pos, L, rc)
    # interpolation error at this resolution: ~ dr^2 |F''| / 8
    assert np.allclose(f_t[:, 3], f_l[:, 3], rtol=1e-7, atol=1e-9)
    assert np.max(np.abs(f_t[:, :3])) <= 1e-12 * np.max(absf)  # symmetric lattice


def test_lj_multitype_coefficients_index_by_type_pair():
    st = inputs.lj_fluid(256, 0.8, 1.0, seed=4, jitter=0.1)
    L = st.box[0, 0]
    t = np.arange(256) % 2
    coeff = np.array([[[1.0, 1.0], [0.5, 1.1]], [[0.5, 1.1], [2.0, 0.9]]])
    f, _, absf = oracle.lj_forces(st.pos, L, 2.5, coeff=coeff, type=t)
    # brute recomputation from the pair function with per-pair coefficients
    i = 7
    acc = np.zeros(3)
    for j in range(256):
        if j == i:
            continue
        d = st.pos[i, :3] - st.pos[j, :3]
        d -= L * np.rint(d / L)
        r2 = d @ d
        if r2 < 6.25:
            e, s = coeff[t[i], t[j]]
            fr, _ = oracle.lj_pair(r2, e, s)
            acc += fr * d
    assert np.allclose(f[i, :3], acc, rtol=1e-12, atol=1e-12)
    assert np.abs(f[:, :3].sum(0)).max() <= 1e-12 * absf.sum()


# --------------------------------------------------------------------------
# neighbour rows and cells

@pytest.mark.parametrize("seed,n,rho,r_list", [(5, 1000, 0.8442, 2.8), (6, 3000, 3.0, 1.3),
                                                (7, 700, 0.5, 2.9)])
def test_neighbors_cells_equal_brute_force(seed, n, rho, r_list):
    st = inputs.lj_fluid(n, rho, 1.0, seed=seed, jitter=0.3)
    L = st.box[0, 0]
    cb, rb = oracle.neighbors(st.pos, L, r_list, method="brute")
    cc, rc = oracle.neighbors(st.pos, L, r_list, method="cells")
    assert np.array_equal(cb, cc)
    assert np.array_equal(rb, rc)
    # symmetric relation
    pairs = {(i, j) for i in range(n) for j in rb[i, :cb[i]]}
    assert all((j, i) in pairs for i, j in pairs)


def test_neighbors_exact_distance_threshold():
    # a pair exactly at r_list is excluded (strict), slightly inside included
    L = 12.0
    pos = np.zeros((3, 4))
    pos[0, :3] = [1.0, 1.0, 1.0]
    pos[1, :3] = [3.5, 1.0, 1.0]           # r = 2.5 exactly
    pos[2, :3] = [1.0, 1.0, 1.0 + 2.4999]  # inside
    c, r = oracle.neighbors(pos, L, 2.5, method="brute")
    assert c.tolist() == [1, 0, 1]
    assert r[0, 0] == 2


def test_cell_coords_bounds_and_counts():
    st = inputs.dpd_fluid(5000, 3.0, 1.0, seed=8)
    L = st.box[0, 0]
    nc = oracle.cells_per_dim(L, 1.3)
    assert nc == math.floor(L / 1.3)
    cc = oracle.cell_coords(st.pos, L, [nc] * 3)
    assert cc.min() >= 0 and cc.max() < nc
    h = L / nc
    x = st.pos[:, :3]
    assert np.all(x >= cc * h - 1e-12) and np.all(x < (cc + 1) * h + 1e-12)
    assert oracle.cells_per_dim(5.0, 2.0) == 0  # fewer than 3 cells


# --------------------------------------------------------------------------
# Philox and DPD

def test_philox_known_answers():
    for row in _golden_rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(v[:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_dpd_theta_symmetric_and_unit_variance():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 2 ** 31 - 1, 20000)
    b = rng.integers(0, 2 ** 31 - 1, 20000)
    th = np.array([oracle.dpd_theta(x, y, 17, 99) for x, y in zip(a, b)])
    th2 = np.array([oracle.dpd_theta(y, x, 17, 99) for x, y in zip(a, b)])
    assert np.array_equal(th, th2)
    assert abs(th.mean()) < 0.03
    assert abs(th.var() - 1.0) < 0.03
    assert th.max() < math.sqrt(3) and th.min() > -math.sqrt(3)
    # the noise changes with the step and the seed
    assert oracle.dpd_theta(1, 2, 17, 99) != oracle.dpd_theta(1, 2, 18, 99)
    assert oracle.dpd_theta(1, 2, 17, 99) != oracle.dpd_theta(1, 2, 17, 98)


def test_dpd_two_particle_closed_forms():
    L = 10.0
    pos = np.zeros((2, 4))
    vel = np.zeros((2, 4))
    pos[0, :3] = [5.5, 5.0, 5.0]
    pos[1, :3] = [5.0, 5.0, 5.0]  # e = +x, r = 0.5, w = 0.5
    # conservative only: A w = 12.5 repulsive; V = A rc w^2 / 2 = 3.125
    f, _, _ = oracle.dpd_forces(pos, vel, L, 1.0, [[25.0, 0.0]], kT=0.0, dt=0.02,
                                step=0, seed=1)
    assert f[0, 0] == pytest.approx(12.5, abs=1e-13)
    assert f[1, 0] == pytest.approx(-12.5, abs=1e-13)
    assert f[0, 3] + f[1, 3] == pytest.approx(3.125, abs=1e-13)
    # dissipative only: -gamma w^2 (e . v_ij), v_ij = v_0 - v_1 = +1 along e
    vel[0, 0] = 1.0
    f, _, _ = oracle.dpd_forces(pos, vel, L, 1.0, [[0.0, 4.5]], kT=0.0, dt=0.02,
                                step=0, seed=1)
    assert f[0, 0] == pytest.approx(-4.5 * 0.25, abs=1e-13)
    # random only (gamma > 0, kT > 0, no relative velocity):
    # sigma w theta / sqrt(dt), sigma = sqrt(2 gamma kT) = 3
    vel[:] = 0.0
    f, _, _ = oracle.dpd_forces(pos, vel, L, 1.0, [[0.0, 4.5]], kT=1.0, dt=0.02,
                                step=5, seed=1)
    th = oracle.dpd_theta(0, 1, 5, 1)
    assert f[0, 0] == pytest.approx(3.0 * 0.5 * th / math.sqrt(0.02), rel=1e-13)
    assert f[1, 0] == pytest.approx(-f[0, 0], rel=1e-15)


def test_dpd_momentum_conservation_and_tag_invariance():
    st = inputs.dpd_fluid(1500, 3.0, 1.0, seed=9)
    L = st.box[0, 0]
    f, _, absf = oracle.dpd_forces(st.pos, st.vel, L, 1.0, [[25.0, 4.5]], 1.0, 0.02,
                                   step=3, seed=11)
    assert np.abs(f[:, :3].sum(0)).max() <= 1e-12 * absf.sum()
    # permuting particles (with their tags) permutes the forces exactly
    perm = np.random.default_rng(1).permutation(1500)
    fp, _, _ = oracle.dpd_forces(st.pos[perm], st.vel[perm], L, 1.0, [[25.0, 4.5]], 1.0,
                                 0.02, step=3, seed=11, tag=st.tag[perm])
    assert np.allclose(fp, f[perm], rtol=1e-12, atol=1e-12 * absf.max())


def test_dpd_nlist_equals_brute():
    st = inputs.dpd_fluid(2000, 3.0, 1.0, seed=10)
    L = st.box[0, 0]
    nl = oracle.neighbors(st.pos, L, 1.3, max_nb=128, method="cells")
    coeff = [[25.0, 4.5]]
    fb, vb, _ = oracle.dpd_forces(st.pos, st.vel, L, 1.0, coeff, 1.0, 0.02, 4, 7)
    fn, vn, _ = oracle.dpd_forces(st.pos, st.vel, L, 1.0, coeff, 1.0, 0.02, 4, 7, nlist=nl)
    assert np.allclose(fb, fn, rtol=1e-13, atol=1e-12)
    assert np.allclose(vb, vn, rtol=1e-13, atol=1e-12)


# --------------------------------------------------------------------------
# bonds and integration

def test_bond_two_bead_closed_form():
    L = 20.0
    pos = np.zeros((2, 4))
    pos[0, :3] = [1.0, 2.0, 3.0]
    pos[1, :3] = [1.9, 2.0, 3.0]  # r = 0.9 along +x from 0 to 1
    f, vir, _ = oracle.bond_forces([[0, 1]], pos, L, K=4.0, r0=0.0)
    assert f[0, 0] == pytest.approx(3.6, abs=1e-13)   # pulled toward 1
    assert f[1, 0] == pytest.approx(-3.6, abs=1e-13)
    assert f[0, 3] + f[1, 3] == pytest.approx(0.5 * 4.0 * 0.81, abs=1e-13)
    f, _, _ = oracle.bond_forces([[0, 1]], pos, L, K=4.0, r0=1.0)
    # stretched below r0 = 1: pushed apart with K (r0 - r) = 0.4
    assert f[0, 0] == pytest.approx(-0.4, abs=1e-13)


def test_harmonic_dimer_oscillation_period():
    # a bonded dimer (no pair forces) oscillates with omega = sqrt(2K/m)
    K, dt = 4.0, 1e-3
    L = np.array([50.0, 50.0, 50.0])
    pos = np.zeros((2, 4))
    vel = np.zeros((2, 4))
    pos[0, :3] = [25.0, 25.0, 25.0]
    pos[1, :3] = [25.5, 25.0, 25.0]
    img = np.zeros((2, 4), np.int32)
    period = 2 * math.pi / math.sqrt(2 * K)
    n = int(round(period / dt))
    f, _, _ = oracle.bond_forces([[0, 1]], pos, L, K, 0.0)
    for _ in range(n):
        pos, vel, img = oracle.vv_first(pos, vel, img, f, dt, L)
        f, _, _ = oracle.bond_forces([[0, 1]], pos, L, K, 0.0)
        vel = oracle.vv_second(vel, f, dt)
    sep = pos[1, 0] - pos[0, 0]
    assert sep == pytest.approx(0.5, abs=2e-3)
    assert abs(vel[0, 0]) < 0.01


def test_fene_bond_closed_forms_and_stretch():
    """FENE (Sec. 3 lists FENE bonds): |F| = K r / (1 - (r/R0)^2), so 2 K R0 / 3
    at r = R0/2; V(R0/sqrt 2) = K R0^2 ln2 / 2; -dV/dr by central differences;
    attractive along the bond; a bond at r >= R0 is counted and skipped."""
    K, R0 = 30.0, 1.5
    L = np.array([20.0, 20.0, 20.0])
    pos = np.zeros((2, 4))
    pos[0, :3] = [5.0, 5.0, 5.0]
    pos[1, :3] = [5.0 + R0 / 2, 5.0, 5.0]
    f, _, _, nb = oracle.fene_bond_forces([[0, 1]], pos, L, K, R0)
    assert nb == 0
    assert f[0, 0] == pytest.approx(2 * K * R0 / 3, rel=1e-14)  # pulled toward particle 1
    assert f[1, 0] == pytest.approx(-2 * K * R0 / 3, rel=1e-14)
    pos[1, :3] = [5.0, 5.0 + R0 / math.sqrt(2), 5.0]
    f, _, _, _ = oracle.fene_bond_forces([[0, 1]], pos, L, K, R0)
    assert f[:, 3].sum() == pytest.approx(0.5 * K * R0 * R0 * math.log(2), rel=1e-14)
    for r in (0.3, 0.9, 1.3):
        h = 1e-6
        e = []
        for x in (r - h, r + h, r):
            pos[1, :3] = [5.0 + x, 5.0, 5.0]
            f, _, _, _ = oracle.fene_bond_forces([[0, 1]], pos, L, K, R0)
            e.append((f[:, 3].sum(), f[1, 0]))
        assert e[2][1] == pytest.approx(-(e[1][0] - e[0][0]) / (2 * h), rel=1e-7)
    pos[1, :3] = [5.0 + R0, 5.0, 5.0]
    f, _, _, nb = oracle.fene_bond_forces([[0, 1]], pos, L, K, R0)
    assert nb == 1 and not f.any()


def test_fene_dimer_small_oscillation_period():
    """For r << R0 the FENE bond is a harmonic spring of constant K: a dimer
    oscillating through r = 0 has period 2 pi / sqrt(2 K / m) (through the
    oracle's MD loop with the FENE bond style; the pair potential has eps = 0)."""
    K, R0, dt = 4.0, 10.0, 1e-3
    L = 12.0
    pos = np.zeros((2, 4))
    vel = np.zeros((2, 4))
    pos[0, :3] = [6.0, 6.0, 6.0]
    pos[1, :3] = [6.2, 6.0, 6.0]
    img = np.zeros((2, 4), np.int32)
    period = 2 * math.pi / math.sqrt(2 * K)
    n = int(round(period / dt))
    out = oracle.run(pos, vel, img, L, n, r_cut=2.5, r_skin=0.3, dt=dt, coeff=[[0.0, 1.0]],
                     bonds=[[0, 1]], K=K, r0=R0, bond_style="fene", max_nb=4)
    sep = out["pos"][1, 0] - out["pos"][0, 0]
    assert sep == pytest.approx(0.2, abs=5e-4)  # back after one period (anharmonic ~(r/R0)^2)


def test_harmonic_angle_gradient_invariances_and_values():
    """Harmonic angles (Sec. 3): forces equal -grad of the total energy by
    central differences; zero net force and torque; a right angle with
    theta0 = 0 has V = K/2 (pi/2)^2 split in thirds; theta = theta0 gives no
    force; the virial trace is sum x . F."""
    rng = np.random.default_rng(8)
    L = np.array([30.0, 30.0, 30.0])
    K, th0 = 7.0, 1.9
    for _ in range(5):
        pos = np.zeros((3, 4))
        pos[:, :3] = 15.0 + rng.normal(scale=0.8, size=(3, 3))
        f, vir, _ = oracle.angle_forces([[0, 1, 2]], pos, L, K, th0)
        assert np.abs(f[:, :3].sum(axis=0)).max() < 1e-12 * np.abs(f[:, :3]).max()
        torque = np.cross(pos[:, :3], f[:, :3]).sum(axis=0)
        assert np.abs(torque).max() < 1e-10 * np.abs(f[:, :3]).max() * 15
        assert np.sum(vir[:, [0, 3, 5]]) == pytest.approx(np.sum(pos[:, :3] * f[:, :3]), rel=1e-10)
        h = 1e-6
        for m in range(3):
            for k in range(3):
                pp, pm = pos.copy(), pos.copy()
                pp[m, k] += h
                pm[m, k] -= h
                ep = oracle.angle_forces([[0, 1, 2]], pp, L, K, th0)[0][:, 3].sum()
                em = oracle.angle_forces([[0, 1, 2]], pm, L, K, th0)[0][:, 3].sum()
                assert f[m, k] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-8)
    pos = np.zeros((3, 4))
    pos[:, :3] = [[16.0, 15.0, 15.0], [15.0, 15.0, 15.0], [15.0, 17.0, 15.0]]
    f, _, _ = oracle.angle_forces([[0, 1, 2]], pos, L, K, 0.0)
    assert f[:, 3] == pytest.approx([K / 2 * (math.pi / 2) ** 2 / 3] * 3, rel=1e-14)
    f, _, _ = oracle.angle_forces([[0, 1, 2]], pos, L, K, math.pi / 2)
    assert np.abs(f).max() < 1e-14


def test_chain_with_angles_conserves_energy():
    """A bonded, angled chain (no pair forces in range of eps = 0) in the
    oracle's MD loop: energy stays constant to O(dt^2) (halving dt quarters
    the energy error), which pins the angle forces inside the loop."""
    L = 20.0
    n = 8
    pos = np.zeros((n, 4))
    pos[:, 0] = 6.0 + 0.9 * np.arange(n)
    pos[:, 1] = 10.0 + 0.3 * np.sin(np.arange(n))
    pos[:, 2] = 10.0
    rng = np.random.default_rng(3)
    vel = np.zeros((n, 4))
    vel[:, :3] = rng.normal(scale=0.3, size=(n, 3))
    vel[:, :3] -= vel[:, :3].mean(axis=0)
    img = np.zeros((n, 4), np.int32)
    bonds = [[i, i + 1] for i in range(n - 1)]
    angles = [[i, i + 1, i + 2] for i in range(n - 2)]
    errs = []
    for dt in (0.004, 0.002):
        steps = int(round(2.0 / dt))
        out = oracle.run(pos, vel, img, L, steps, r_cut=2.5, r_skin=0.3, dt=dt,
                         coeff=[[0.0, 1.0]], bonds=bonds, K=20.0, r0=0.9, angles=angles,
                         angle_K=5.0, angle_theta0=2.6, thermo_period=int(round(0.1 / dt)),
                         max_nb=16)
        e = out["thermo"][:, 0] + out["thermo"][:, 1]
        errs.append(np.max(np.abs(e - e[0])))
    assert errs[0] < 1e-2
    assert errs[1] == pytest.approx(errs[0] / 4, rel=0.25)


def test_vv_first_wraps_and_counts_images():
    L = np.array([10.0, 10.0, 10.0])
    pos = np.array([[9.95, 0.02, 5.0, 0.0]])
    vel = np.array([[10.0, -10.0, 0.0, 0.0]])
    f = np.zeros((1, 4))
    img = np.zeros((1, 4), np.int32)
    p, v, im = oracle.vv_first(pos, vel, img, f, 0.01, L)
    assert p[0, 0] == pytest.approx(0.05, abs=1e-12) and im[0, 0] == 1
    assert p[0, 1] == pytest.approx(9.92, abs=1e-12) and im[0, 1] == -1
    assert np.all(p[0, :3] >= 0) and np.all(p[0, :3] < 10.0)


def test_thermo_of_maxwell_boltzmann_input():
    st = inputs.lj_fluid(4000, 0.8442, 1.44, seed=12)
    th = oracle.thermo(st.vel, np.zeros((4000, 4)), None, st.box[0])
    assert th["temperature"] == pytest.approx(1.44, rel=1e-12)
    assert th["ke"] == pytest.approx(0.5 * (3 * 4000 - 3) * 1.44, rel=1e-12)
    assert max(abs(th["px"]), abs(th["py"]), abs(th["pz"])) < 1e-10
    V = st.box[0, 0] ** 3
    assert th["pressure"] == pytest.approx(2 * th["ke"] / (3 * V), rel=1e-12)


@pytest.mark.parametrize("rho,r_cut", [(0.8442, 2.5), (1.0, 3.0)])
def test_thermo_virial_pressure_is_minus_dU_dV_on_the_lattice(rho, r_cut):
    """At T = 0 the pressure of a perfect fcc lattice is -dU/dV (thermodynamic
    route).  U(V) is the oracle's summed potential energy at three nearby
    densities (no neighbour shell crosses r_cut in between); the thermo row's
    pressure W / (3V) at the middle density, with W the summed virial trace,
    must equal its central difference.  A wrong sign, a missing 1/3 or a
    virial off by a factor fails this.  W itself equals the shell sum."""
    n, eps = 4 * 6 ** 3, 1e-5
    vel = np.zeros((n, 4))
    U, V, P, W = [], [], [], []
    for r in (rho * (1 - eps), rho, rho * (1 + eps)):
        st = inputs.lj_fluid(n, r, 1.0, seed=1)  # perfect 6^3 lattice
        L = st.box[0]
        f, vir, _ = oracle.lj_forces(st.pos, L, r_cut)
        th = oracle.thermo(vel, f, vir, L)
        U.append(th["pe"])
        V.append(float(np.prod(L)))
        P.append(th["pressure"])
        W.append(th["virial"])
    dUdV = (U[2] - U[0]) / (V[2] - V[0])
    assert P[1] == pytest.approx(-dUdV, rel=1e-6)
    # the virial trace is the crystallographic shell sum times N
    a = (4.0 / rho) ** (1.0 / 3.0)
    w = 0.0
    for k, z in _fcc_shells():
        rr = a * math.sqrt(k / 2.0)
        if rr < r_cut:
            fr, _ = oracle.lj_pair(rr * rr)
            w += 0.5 * z * fr * rr * rr
    assert W[1] == pytest.approx(n * w, rel=1e-11)
    assert P[1] == pytest.approx(W[1] / (3.0 * V[1]), rel=1e-12)


def test_thermo_ideal_gas_and_two_particle_virial():
    """No pair inside r_cut: P V = (N - 1) T (ideal gas with the 3N - 3
    degrees of freedom of the temperature); two particles at r = sigma add
    W = r . f = 24 and P = W / (3V) beyond the kinetic part."""
    st = inputs.lj_fluid(500, 0.01, 2.0, seed=5)  # dilute: spacing 5.8 > r_cut
    L = st.box[0]
    f, vir, absf = oracle.lj_forces(st.pos, L, 2.5)
    assert absf.max() == 0.0
    th = oracle.thermo(st.vel, f, vir, L)
    V = float(np.prod(L))
    assert th["pressure"] * V == pytest.approx((500 - 1) * th["temperature"], rel=1e-12)
    pos = np.zeros((2, 4))
    pos[0, :3] = [5.0, 5.0, 5.0]
    pos[1, :3] = [5.0, 6.0, 5.0]
    f, vir, _ = oracle.lj_forces(pos, 10.0, 2.5)
    th = oracle.thermo(np.zeros((2, 4)), f, vir, 10.0)
    assert th["virial"] == pytest.approx(24.0, abs=1e-12)
    assert th["pressure"] == pytest.approx(24.0 / 3000.0, abs=1e-15)


def test_time_reversibility_lj():
    st = inputs.lj_fluid(864, 0.8442, 1.44, seed=13)
    L = st.box[0]
    kw = dict(r_cut=2.5, r_skin=0.3, dt=0.005)
    a = oracle.run(st.pos, st.vel, st.image, L, 60, **kw)
    b = oracle.run(a["pos"], -a["vel"], a["image"], L, 60, **kw)
    x0 = st.pos[:, :3] + st.image[:, :3] * L
    x1 = b["pos"][:, :3] + b["image"][:, :3] * L
    assert np.max(np.abs(x1 - x0)) < 1e-9
    assert np.max(np.abs(b["vel"][:, :3] + st.vel[:, :3])) < 1e-9
    assert a["builds"] > 1  # the list was rebuilt along the way


def test_nve_energy_drift_small_lj():
    # melting fcc start; velocity Verlet conserves the shifted LJ energy up to
    # the small drift caused by truncating the force at r_cut.  (The 1e-4
    # eps/particle bound over 1e4 steps is checked at N = 4000 on the GPU;
    # this short CPU run bounds the drift rate loosely but still catches a
    # broken half-kick or a wrong energy term by orders of magnitude.)
    n = 2048
    st = inputs.lj_fluid(n, 0.8442, 1.44, seed=14)
    L = st.box[0]
    eq = oracle.run(st.pos, st.vel, st.image, L, 400, r_cut=2.5, r_skin=0.3, dt=0.005)
    out = oracle.run(eq["pos"], eq["vel"], eq["image"], L, 2000, r_cut=2.5, r_skin=0.3,
                     dt=0.005, shift_energy=True, thermo_period=10, step0=400)
    e = (out["thermo"][:, 0] + out["thermo"][:, 1]) / n
    t = np.arange(e.size) * 10 * 0.005
    slope = np.polyfit(t, e, 1)[0]
    assert abs(slope) * 1e4 * 0.005 < 3e-4
    assert np.max(np.abs(e - e[0])) < 1e-3
    # without the energy shift the same trajectory does not conserve "energy"
    raw = oracle.run(eq["pos"], eq["vel"], eq["image"], L, 200, r_cut=2.5, r_skin=0.3,
                     dt=0.005, shift_energy=False, thermo_period=10, step0=400)
    e_raw = (raw["thermo"][:, 0] + raw["thermo"][:, 1]) / n
    assert np.max(np.abs(e_raw - e_raw[0])) > np.max(np.abs(e[:20] - e[0]))


def test_run_nlist_forces_equal_brute_force_after_steps():
    st = inputs.lj_fluid(500, 0.8442, 1.44, seed=15)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 50, r_cut=2.5, r_skin=0.3, dt=0.005)
    fb, _, _ = oracle.lj_forces(out["pos"], L, 2.5)
    assert np.allclose(out["force"], fb, rtol=1e-12, atol=1e-11)


def test_dpd_thermostat_temperature():
    st = inputs.dpd_fluid(3000, 3.0, 1.0, seed=16)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 600, r_cut=1.0, r_skin=0.3, dt=0.02,
                     pair="dpd", coeff=[[25.0, 4.5]], kT=1.0, seed=5, thermo_period=10)
    T = out["thermo"][20:, 4].mean()
    assert T == pytest.approx(1.0, abs=0.05)
    p = out["thermo"][:, 5:8]
    assert np.abs(p).max() < 1e-9  # pairwise-symmetric noise conserves momentum


# --------------------------------------------------------------------------
# space-filling curve

@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_is_a_unit_step_bijection(bits):
    m = 1 << bits
    idx = {}
    for x in range(m):
        for y in range(m):
            for z in range(m):
                idx[oracle.hilbert3(x, y, z, bits)] = (x, y, z)
    assert sorted(idx) == list(range(m ** 3))
    for h in range(m ** 3 - 1):
        a, b = np.array(idx[h]), np.array(idx[h + 1])
        assert np.abs(a - b).sum() == 1
    assert idx[0] == (0, 0, 0)


def test_sfc_order_is_permutation_walking_adjacent_bricks():
    L = 24.0
    nc = 8  # r_list 2.99 -> 8 cells of width 3, 4 bricks of 2 x 2 x 2 cells per edge
    cells = np.array([(x, y, z) for x in range(nc) for y in range(nc) for z in range(nc)])
    rng = np.random.default_rng(2)
    perm = rng.permutation(len(cells))
    pos = np.zeros((len(cells), 4))
    pos[:, :3] = (cells[perm] + 0.5) * 3.0
    order = oracle.sfc_order(pos, L, 2.99)
    assert sorted(order.tolist()) == list(range(len(cells)))
    walk = cells[perm][order]
    bricks = walk // 2
    # each run of 8 is one brick, its particles in index order (ties by index)
    for k in range(0, len(walk), 8):
        assert np.all(bricks[k:k + 8] == bricks[k])
        assert np.all(np.diff(order[k:k + 8]) > 0)
    # and the bricks follow the Hilbert curve: unit steps, starting at the origin
    b = bricks[::8]
    assert np.all(np.abs(np.diff(b, axis=0)).sum(1) == 1)
    assert b[0].tolist() == [0, 0, 0]


def test_sfc_order_odd_grid_and_many_per_cell():
    # 7 cells per edge (the last brick layer is one cell thick), several
    # particles per cell: bricks form contiguous runs along a unit-step walk
    L, rl = 21.0, 2.99
    rng = np.random.default_rng(4)
    pos = np.zeros((3000, 4))
    pos[:, :3] = rng.uniform(0.0, L, (3000, 3))
    order = oracle.sfc_order(pos, L, rl)
    assert sorted(order.tolist()) == list(range(3000))
    b = oracle.cell_coords(pos, L, [7, 7, 7])[order] // 2
    keys = [tuple(x) for x in b]
    runs = [keys[0]] + [keys[k] for k in range(1, len(keys)) if keys[k] != keys[k - 1]]
    assert len(runs) == len(set(runs)) == 4 ** 3  # every brick one contiguous run
    steps = np.abs(np.diff(np.array(runs), axis=0)).sum(1)
    assert np.all(steps == 1)
    for k in range(1, len(keys)):  # ties by index inside a brick
        if keys[k] == keys[k - 1]:
            assert order[k] > order[k - 1]


def test_local_neighbourhood_answers_equal_whole_system_ones():
    """The per-particle oracle answers the headline-size GPU test uses (the
    particle and its 27 cells) equal the whole-system oracle answers, for
    random particles and the ones next to each face of the box."""
    from local_ref import local_reference
    st = inputs.lj_fluid(32000, 0.8442, 1.2, seed=12345, jitter=0.05)
    pos, L = st.pos, st.box[0, 0]
    rng = np.random.default_rng(3)
    edge = np.concatenate([np.argsort(pos[:, k])[:3] for k in range(3)] +
                          [np.argsort(pos[:, k])[-3:] for k in range(3)])
    samples = np.unique(np.concatenate([rng.choice(st.n, 100, replace=False), edge]))
    rows, f, absf = local_reference(pos, L, samples, 2.5, 0.4)
    cb, rb = oracle.neighbors(pos, L, 2.9, max_nb=256, method="cells")
    fr, _, afr = oracle.lj_forces(pos, L, 2.5, nlist=(cb, rb))
    for k, i in enumerate(samples):
        assert np.array_equal(rows[k], np.sort(rb[i, :cb[i]])), int(i)
        d = np.linalg.norm(f[k, :3] - fr[i, :3])
        assert d <= 1e-12 * max(np.linalg.norm(fr[i, :3]), 1e-2 * afr[i]), int(i)
    assert np.allclose(absf, afr[samples], rtol=1e-12)


def test_cell_list_rows_in_a_box_that_is_an_exact_multiple_of_r_list():
    """Box 12 = 4 r_list: the cell list uses 3 cells (the 1e-12 margin), and
    pairs straddling the planes x = k r_list at r_list (1 - 1e-14) are rows of
    each other, as brute force says."""
    L, rl = 12.0, 3.0
    assert oracle.cells_per_dim(L, rl) == 3
    d = rl * (1 - 1e-14)
    pos = np.zeros((8, 4))
    yz = ((0.5, 0.5), (6.5, 0.5), (0.5, 6.5), (6.5, 6.5))
    for k, x0 in enumerate((3.0, 6.0, 9.0, 12.0)):
        pos[2 * k, :3] = [x0 - 0.5 * d, *yz[k]]
        pos[2 * k + 1, :3] = [x0 + 0.5 * d, *yz[k]]
    pos[:, :3] = np.mod(pos[:, :3], L)
    cb, rb = oracle.neighbors(pos, L, rl, method="brute")
    cc, rc = oracle.neighbors(pos, L, rl, method="cells")
    assert cb.tolist() == [1] * 8
    assert np.array_equal(cb, cc) and np.array_equal(rb, rc)


# --------------------------------------------------------------------------
# thermostats: Langevin (BAOAB) and Nose-Hoover (one thermostat, MTK splitting)

def test_langevin_noise_statistics_and_keys():
    th = np.array([oracle.langevin_noise(t, s, 3) for t in range(4000) for s in (1, 2)])
    assert th.shape == (8000, 3)
    assert np.abs(th.mean(0)).max() < 0.04
    assert np.abs(th.var(0) - 1.0).max() < 0.04
    assert th.max() < math.sqrt(3) and th.min() > -math.sqrt(3)
    assert abs(np.corrcoef(th[:, 0], th[:, 1])[0, 1]) < 0.04  # components independent
    a = oracle.langevin_noise(7, 11, 3)
    assert not np.array_equal(a, oracle.langevin_noise(8, 11, 3))
    assert not np.array_equal(a, oracle.langevin_noise(7, 12, 3))
    assert not np.array_equal(a, oracle.langevin_noise(7, 11, 4))


def test_baoab_without_friction_is_velocity_verlet():
    st = inputs.lj_fluid(864, 0.8442, 1.44, seed=21)
    L = st.box[0]
    kw = dict(r_cut=2.5, r_skin=0.3, dt=0.005)
    a = oracle.run(st.pos, st.vel, st.image, L, 50, **kw)
    b = oracle.run(st.pos, st.vel, st.image, L, 50, integrator="langevin", gamma=0.0, t_kT=1.0,
                   t_seed=5, **kw)
    xa = a["pos"][:, :3] + a["image"][:, :3] * L
    xb = b["pos"][:, :3] + b["image"][:, :3] * L
    assert np.max(np.abs(xa - xb)) < 1e-10
    assert np.max(np.abs(a["vel"] - b["vel"])) < 1e-9


def _free_gas(n=3000, L=200.0, seed=22):
    # particles more than r_cut apart: no pair forces, only the thermostat acts
    g = np.stack(np.meshgrid(*[np.arange(15)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    pos = np.zeros((n, 4))
    pos[:, :3] = (g + 0.5) * (L / 15)
    return pos, np.zeros((n, 4), np.int32), np.array([L, L, L])


def test_langevin_o_step_relaxation_of_free_particles():
    """Without forces BAOAB's velocities follow the O step exactly:
    v_n = c^n v_0 + noise, c = exp(-gamma dt), so from rest E[v_n^2] =
    (1 - c^(2n)) kT/m, and from Maxwell-Boltzmann velocities at kT the
    autocorrelation is E[v_n v_0] / E[v_0^2] = c^n."""
    pos, img, L = _free_gas()
    n = len(pos)
    gamma, dt, kT, steps = 2.0, 0.01, 1.5, 50
    c = math.exp(-gamma * dt)
    kw = dict(r_cut=2.5, r_skin=0.3, dt=dt, integrator="langevin", gamma=gamma, t_kT=kT,
              t_seed=9, max_nb=8)
    out = oracle.run(pos, np.zeros((n, 4)), img, L, steps, **kw)
    v2 = np.mean(out["vel"][:, :3] ** 2)
    assert v2 == pytest.approx((1 - c ** (2 * steps)) * kT, rel=0.04)
    v0 = np.zeros((n, 4))
    v0[:, :3] = np.random.default_rng(1).standard_normal((n, 3)) * math.sqrt(kT)
    out = oracle.run(pos, v0, img, L, steps, **kw)
    acf = np.mean(out["vel"][:, :3] * v0[:, :3]) / np.mean(v0[:, :3] ** 2)
    assert acf == pytest.approx(c ** steps, abs=0.03)


def test_langevin_lj_fluid_equipartition():
    st = inputs.lj_fluid(864, 0.8442, 0.6, seed=23)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 3000, r_cut=2.5, r_skin=0.3, dt=0.005,
                     integrator="langevin", gamma=1.0, t_kT=1.2, t_seed=4, thermo_period=10)
    T = out["thermo"][100:, 4].mean()
    assert T == pytest.approx(1.2, rel=0.03)


def test_nose_hoover_with_a_slow_thermostat_is_velocity_verlet():
    st = inputs.lj_fluid(864, 0.8442, 1.44, seed=24)
    L = st.box[0]
    kw = dict(r_cut=2.5, r_skin=0.3, dt=0.005)
    a = oracle.run(st.pos, st.vel, st.image, L, 50, **kw)
    b = oracle.run(st.pos, st.vel, st.image, L, 50, integrator="nose-hoover", tau=1e9, t_kT=1.0,
                   **kw)
    xa = a["pos"][:, :3] + a["image"][:, :3] * L
    xb = b["pos"][:, :3] + b["image"][:, :3] * L
    assert np.max(np.abs(xa - xb)) < 1e-10
    assert abs(b["nh_state"][0]) < 1e-15


def _nh_run(dt, t_end, n=864, kT=1.3, tau=0.3, seed=25):
    st = inputs.lj_fluid(n, 0.8442, 0.8, seed=seed)
    L = st.box[0]
    g = 3 * n - 3
    kw = dict(r_cut=2.5, r_skin=0.3, dt=dt, shift_energy=True, integrator="nose-hoover",
              tau=tau, t_kT=kT, thermo_period=10)
    state, nh, H, T = (st.pos, st.vel, st.image), np.zeros(2), [], []
    for k in range(int(round(t_end / (10 * dt)))):
        out = oracle.run(*state, L, 10, step0=10 * k, nh_state=nh, **kw)
        state, nh = (out["pos"], out["vel"], out["image"]), out["nh_state"]
        ke, pe = out["thermo"][-1, 0], out["thermo"][-1, 1]
        H.append((ke + pe + g * kT * tau * tau * nh[0] ** 2 / 2 + g * kT * nh[1]) / n)
        T.append(out["thermo"][-1, 4])
    return np.array(H), np.array(T)


def test_nose_hoover_conserved_quantity_and_temperature():
    """H = KE + PE + g kT tau^2 xi^2 / 2 + g kT eta (g = 3N - 3) is conserved
    by the Nose-Hoover dynamics; the splitting conserves it up to an error of
    second order in dt (halving dt divides the largest deviation by about
    four; a wrong term or coefficient leaves a first-order or constant drift
    instead).  Started at T = 0.8 with kT = 1.3, so the thermostat does real
    work; the kinetic temperature then averages to kT."""
    H1, T1 = _nh_run(0.005, 7.5)
    H2, _ = _nh_run(0.0025, 7.5)
    e1, e2 = np.abs(H1 - H1[0]).max(), np.abs(H2 - H2[0]).max()
    assert 3.0 < e1 / e2 < 5.5, (e1, e2)
    assert e2 < 2.5e-3
    assert T1[0] < 1.0  # started cold
    assert np.mean(T1[40:]) == pytest.approx(1.3, rel=0.04)
