"""GPU parity on the configurations the benchmark times (through the C ABI,
against the CPU oracle on the same seeded inputs):

  * md_run's CUDA-graph path (a step's second half-kick folded into the next
    step's first, thermo rows closing graph segments, a sort at every
    rebuild): FP64 trajectory against the oracle's;
  * md_autotune on a 65,536-particle fluid, then rows and forces;
  * the mixed-precision batched ensemble of 256 replicas of 2,000-64,000
    particles, as benchmarked, against the oracle replica by replica;
  * harmonic bonds after a space-filling-curve sort;
  * pairs placed within a few ulps of r_list^2 and r_cut^2 at the far corners
    of bricks, where the FP32 stage coordinates are largest;
  * DPD over many steps: FP64 trajectory, thermostat temperature, momentum.

Tolerances as in test_gpu_parity.py.
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
from test_gpu_parity import fp64_force_check, mixed_force_stats  # noqa: E402

U32 = 2.0 ** -24  # FP32 unit roundoff


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1412_3387_gb300 import build
    build.build()
    oracle.build()


def unwrapped_by_tag(g, L):
    x = g["pos"][:, :3] + g["image"][:, :3] * L
    out = np.empty_like(x)
    out[g["tag"]] = x
    return out


def vel_by_tag(g):
    out = np.empty_like(g["vel"][:, :3])
    out[g["tag"]] = g["vel"][:, :3]
    return out


def test_graph_run_fp64_trajectory_matches_oracle():
    """200 steps in 100-step graphs, thermo every 10 steps, sorted at every
    rebuild: positions within 1e-9 by tag, thermo rows within 1e-9."""
    st = inputs.lj_fluid(4000, 0.8442, 1.44, seed=22, jitter=0.05)
    L = st.box[0]
    out = oracle.run(st.pos, st.vel, st.image, L, 200, r_cut=2.5, r_skin=0.3, dt=0.005,
                     shift_energy=True, thermo_period=10)
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, shift_energy=True, thermo_period=10,
                    graph_steps=100, sort_period=1)
    s.prepare()
    th = s.run_with_thermo(200).cpu().numpy()[:, 0, :]
    s.check_error()
    g = s.state_numpy()
    assert not np.array_equal(g["tag"], np.arange(st.n))  # it did sort
    x0 = out["pos"][:, :3] + out["image"][:, :3] * L
    assert np.max(np.abs(unwrapped_by_tag(g, L) - x0)) < 1e-9
    assert np.max(np.abs(vel_by_tag(g) - out["vel"][:, :3])) < 1e-8
    assert th.shape == out["thermo"].shape
    assert np.allclose(th, out["thermo"], rtol=1e-9, atol=1e-9)
    assert s.get_step() == 200
    assert out["builds"] > 3


def test_autotune_then_rows_and_forces_match_oracle():
    st = inputs.lj_fluid(65536, 0.8442, 1.2, seed=23, jitter=0.1)
    L = st.box[0]
    s = md.MDSystem(st, r_cut=2.5, r_skin=0.4, dt=0.005, precision="mixed")
    s.prepare()
    tune = s.autotune(n_samples=3, block_stride=4)
    assert all(b % 32 == 0 and w in (1, 2, 4, 8, 16, 32) for b, w in tune.values())
    assert tune["nlist"][1] <= tune["pair"][1]
    s.check_error()
    counts, rows = (x.cpu().numpy() for x in s.nlist())
    cb, rb = oracle.neighbors(st.pos, L, 2.9, max_nb=s.max_nb, method="cells")
    assert np.array_equal(counts, cb)
    for i in range(st.n):
        assert np.array_equal(np.sort(rows[i, :counts[i]]), rb[i, :cb[i]]), i
    ref, _, absf = oracle.lj_forces(st.pos, L, 2.5, nlist=(cb, rb))
    rms, mx = mixed_force_stats(s.forces().cpu().numpy(), ref, absf)
    assert rms <= 1e-5 and mx <= 1e-3, (rms, mx)
    s.close()


def test_batched_mixed_ensemble_as_benchmarked():
    """The 256-replica ensemble (N log-uniform in [2000, 64000]) in mixed
    precision: per-replica forces against the oracle (a sample of replicas,
    always including the smallest and the largest); the FP64 batched forces
    of the smallest and largest replicas equal standalone runs bitwise."""
    ens = inputs.replica_ensemble(256, seed=777, jitter=0.1)
    sizes = np.diff(ens.offsets)
    kw = dict(r_cut=2.5, r_skin=0.3, dt=0.005)
    b = md.MDSystem(ens, precision="mixed", **kw)
    b.prepare()
    fb = b.forces().cpu().numpy()
    b.check_error()
    rng = np.random.default_rng(0)
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)),
                   *rng.choice(256, 14, replace=False).tolist()})
    for r in pick:
        sub = inputs.select_replica(ens, r)
        nl = oracle.neighbors(sub.pos, sub.box[0], 2.8, max_nb=256, method="cells")
        ref, _, absf = oracle.lj_forces(sub.pos, sub.box[0], 2.5, nlist=nl)
        o0, o1 = ens.offsets[r], ens.offsets[r + 1]
        rms, mx = mixed_force_stats(fb[o0:o1], ref, absf)
        assert rms <= 1e-5 and mx <= 1e-3, (r, rms, mx)
    b.close()
    b64 = md.MDSystem(ens, precision="fp64", **kw)
    b64.prepare()
    f64 = b64.forces().cpu().numpy()
    for r in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        sub = inputs.select_replica(ens, r)
        a = md.MDSystem(sub, precision="fp64", **kw)
        a.prepare()
        o0, o1 = ens.offsets[r], ens.offsets[r + 1]
        assert np.array_equal(a.forces().cpu().numpy(), f64[o0:o1]), r
        a.close()
    b64.close()


@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_bonds_after_sort_match_oracle(prec):
    st = inputs.diblock_melt(64, 32, 3.0, 1.0, seed=42)
    L = st.box[0]
    coeff = np.array([[[25.0, 4.5], [40.0, 4.5]], [[40.0, 4.5], [25.0, 4.5]]])
    step, seed = 11, 123
    ref, vref, absf = oracle.dpd_forces(st.pos, st.vel, L, 1.0, coeff, 1.0, 0.02, step, seed,
                                        type=st.type)
    ref, vref, absf = oracle.bond_forces(st.bonds, st.pos, L, 4.0, 0.0, ref, vref, absf)
    s = md.MDSystem(st, r_cut=1.0, r_skin=0.3, dt=0.02, pair="dpd", coeff=coeff, kT=1.0,
                    seed=seed, precision=prec, bond_K=4.0, bond_r0=0.0)
    s.set_step(step)
    s.build_cells()
    s.sort()
    s.prepare()
    s.compute_forces(want_virial=True)
    f = s.forces().cpu().numpy()
    s.check_error()
    tag = s.tag.cpu().numpy()
    assert not np.array_equal(tag, np.arange(st.n))
    if prec == "fp64":
        fp64_force_check(f, ref[tag], absf[tag])
        assert np.allclose(f[:, 3], ref[tag, 3], rtol=1e-12, atol=1e-12 * absf.max())
    else:
        rms, mx = mixed_force_stats(f, ref[tag], absf[tag])
        assert rms <= 1e-5 and mx <= 1e-3, (rms, mx)


def band_edge_state(seed, n_bg=500, n_pairs=64, L=20.0, r_cut=2.5, r_skin=0.3, d_min=0.9):
    """A dilute gas plus pairs whose squared separation lies within a few
    FP64 ulps (and, for some, across the FP32 error band) of r_list^2 or
    r_cut^2.  Each pair's first particle sits just inside a corner of a brick
    of 2 x 2 x 2 cells and its partner outside the brick along an outward
    diagonal, so the partner's brick-frame FP32 coordinates are the largest a
    stage holds.  Every other separation is at least d_min (no overlaps, so
    the mixed tolerance applies)."""
    rng = np.random.default_rng(seed)
    nc = math.floor(L / (r_cut + r_skin))
    h = L / nc
    nb = (nc + 1) // 2
    pts = np.zeros((0, 3))

    def far_from_all(x, skip=0):
        if len(pts) - skip <= 0:
            return True
        d = pts[:len(pts) - skip] - x
        d -= L * np.rint(d / L)
        return np.min(np.einsum("ij,ij->i", d, d)) >= d_min * d_min

    k = tries = 0
    while k < n_pairs and tries < 50 * n_pairs:
        tries += 1
        b = rng.integers(0, nb, 3)
        side = rng.integers(0, 2, 3)
        corner = np.minimum(2 * b + 2 * side, nc) * h
        sgn = np.where(side == 1, 1.0, -1.0)  # outward
        a = np.mod(corner - sgn * rng.uniform(0.005, 0.05, 3), L)
        u = sgn * rng.uniform(0.3, 1.0, 3)
        u /= np.linalg.norm(u)
        target = (r_cut + r_skin) if k % 2 == 0 else r_cut
        if k % 8 == 1:  # also spread across the FP32 band, not only FP64 ulps
            r = target * (1.0 + rng.uniform(-3e-6, 3e-6))
        else:
            r = target * (1.0 + int(rng.integers(-4, 5)) * 2.0 ** -52)
        c = np.mod(a + r * u, L)
        if far_from_all(a) and far_from_all(c):
            pts = np.concatenate([pts, a[None], c[None]])
            k += 1
    while len(pts) < 2 * n_pairs + n_bg:
        x = rng.uniform(0.0, L, 3)
        if far_from_all(x):
            pts = np.concatenate([pts, x[None]])
    n = len(pts)
    pos = np.zeros((n, 4))
    pos[:, :3] = pts
    return inputs.State(pos=pos, vel=np.zeros((n, 4)), image=np.zeros((n, 4), np.int32),
                        tag=np.arange(n, dtype=np.int32), type=np.zeros(n, np.int32),
                        box=np.array([[L, L, L]]), offsets=np.array([0, n], np.int64))


@pytest.mark.parametrize("w", (1, 2, 8))
def test_band_edge_pairs_rows_and_forces_exact(w):
    st = band_edge_state(seed=70 + w)
    L = st.box[0]
    cb, rb = oracle.neighbors(st.pos, L, 2.8, max_nb=128, method="brute")
    ref, _, absf = oracle.lj_forces(st.pos, L, 2.5)
    for prec in ("fp64", "mixed"):
        s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, precision=prec, max_nb=128)
        s.set_tuning(md.KERNEL_PAIR, 128, w)
        s.set_tuning(md.KERNEL_NLIST, 64, w)
        s.prepare()
        counts, rows = (x.cpu().numpy() for x in s.nlist())
        assert np.array_equal(counts, cb), prec
        for i in range(st.n):
            assert np.array_equal(np.sort(rows[i, :counts[i]]), rb[i, :cb[i]]), (prec, i)
        f = s.forces().cpu().numpy()
        s.check_error()
        if prec == "fp64":
            fp64_force_check(f, ref, absf, f"w={w}")
        else:
            # every pair inside r_cut is included exactly: a missing or extra
            # pair at r_cut changes a force by |F(r_cut)| ~ 0.04, far above the
            # mixed tolerance on these isolated pairs
            rms, mx = mixed_force_stats(f, ref, absf)
            assert rms <= 1e-5 and mx <= 1e-3, (rms, mx)
        s.close()


def test_dpd_fp64_trajectory_matches_oracle():
    st = inputs.dpd_fluid(3000, 3.0, 1.0, seed=33)
    L = st.box[0]
    kw = dict(r_cut=1.0, r_skin=0.3, dt=0.02)
    coeff = [[25.0, 4.5]]
    out = oracle.run(st.pos, st.vel, st.image, L, 50, pair="dpd", coeff=coeff, kT=1.0,
                     seed=9, thermo_period=10, **kw)
    s = md.MDSystem(st, pair="dpd", coeff=coeff, kT=1.0, seed=9, thermo_period=10,
                    graph_steps=50, sort_period=1, **kw)
    s.prepare()
    th = s.run_with_thermo(50).cpu().numpy()[:, 0, :]
    s.check_error()
    g = s.state_numpy()
    x0 = out["pos"][:, :3] + out["image"][:, :3] * L
    assert np.max(np.abs(unwrapped_by_tag(g, L) - x0)) < 1e-9
    assert np.max(np.abs(vel_by_tag(g) - out["vel"][:, :3])) < 1e-8
    assert np.allclose(th[:, [0, 4, 5, 6, 7]], out["thermo"][:, [0, 4, 5, 6, 7]], rtol=1e-9,
                       atol=1e-9)


@pytest.mark.parametrize("prec", ("fp64", "mixed"))
def test_dpd_thermostat_and_momentum_over_steps(prec):
    """600 steps at dt = 0.02 from uniform positions: the kinetic temperature
    after 100 steps averages to the oracle's own average over the same steps
    within 0.02 (the statistical error of either mean is ~0.003); total
    momentum stays zero to rounding (pairwise-symmetric noise and forces).
    For the mixed path the momentum bound comes from FP32 rounding of the pair
    forces: 20 x dt sqrt(steps) 2^-24 sqrt(N n_pairs) f_rms."""
    st = inputs.dpd_fluid(3000, 3.0, 1.0, seed=16)
    L = st.box[0]
    kw = dict(r_cut=1.0, r_skin=0.3, dt=0.02)
    coeff = [[25.0, 4.5]]
    out = oracle.run(st.pos, st.vel, st.image, L, 600, pair="dpd", coeff=coeff, kT=1.0, seed=5,
                     thermo_period=10, **kw)
    s = md.MDSystem(st, pair="dpd", coeff=coeff, kT=1.0, seed=5, thermo_period=10,
                    graph_steps=100, sort_period=1, precision=prec, **kw)
    s.prepare()
    th = s.run_with_thermo(600).cpu().numpy()[:, 0, :]
    s.check_error()
    assert abs(th[10:, 4].mean() - out["thermo"][10:, 4].mean()) < 0.02
    p = np.abs(th[:, 5:8]).max()
    if prec == "fp64":
        assert p < 1e-9, p
    else:
        f = s.forces().cpu().numpy()[:, :3]
        counts, _ = s.nlist()
        n_pairs = float(counts.sum().item()) / 2
        f_rms = math.sqrt(float(np.mean(np.sum(f * f, axis=1))))
        bound = 20 * 0.02 * math.sqrt(600) * U32 * math.sqrt(n_pairs) * f_rms
        assert p < bound, (p, bound)


def library_band(L, r_cut, r_skin):
    """The library's FP32 r^2 uncertainty band for a cubic box (the plan's
    formula, restated here only to aim test pairs at the band's ends)."""
    rl = r_cut + r_skin
    nc = math.floor(L / (rl * (1 + 1e-12)))
    h = L / nc
    g = 2.0 ** -40
    while True:
        hq = 2 * g * round(h / (2 * g))
        wq = g * round((L - nc * hq) / g)
        omax = 0.5 * h + 0.5 * r_skin + nc * abs(hq - h) + g
        if omax < g * 2 ** 22 and omax + 1.5 * hq + abs(wq) < g * 2 ** 24:
            break
        g *= 2
    err = 2 * rl * math.sqrt(3) * 1.5 * g + 3 * 2.0 ** -24 * rl * rl
    return max(64 * 2.0 ** -24 * (h + r_skin) ** 2, 4 * err)


def band_ends_state(seed, L=60.0, r_cut=2.5, r_skin=0.3, n_per=100, spread=1.2e-5):
    """Isolated pairs (every other particle farther than r_list + 0.5) whose
    squared separation lies near an end of the FP32 band around r_cut^2 and
    r_list^2: end + U(-spread, spread), with end = the FP32-rounded
    target -+ band.  Their FP32 r^2 scatters across the ends by the grid
    rounding of the offsets, so every way of landing near an end occurs."""
    rng = np.random.default_rng(seed)
    f32 = np.float32
    band = f32(library_band(L, r_cut, r_skin))
    ends = []
    for target in (r_cut * r_cut, (r_cut + r_skin) ** 2):
        t = f32(target)
        ends += [float(f32(t - band)), float(f32(t + band))]
    d_min = r_cut + r_skin + 0.5
    pts = []

    def free(x):
        if not pts:
            return True
        d = np.array(pts) - x
        d -= L * np.rint(d / L)
        return np.min(np.einsum("ij,ij->i", d, d)) > d_min * d_min

    for end in ends:
        made = 0
        while made < n_per:
            a = rng.uniform(0.0, L, 3)
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            r = math.sqrt(end + rng.uniform(-spread, spread))
            c = np.mod(a + r * u, L)
            if free(a) and free(c):
                pts += [a, c]
                made += 1
    n = len(pts)
    pos = np.zeros((n, 4))
    pos[:, :3] = pts
    return inputs.State(pos=pos, vel=np.zeros((n, 4)), image=np.zeros((n, 4), np.int32),
                        tag=np.arange(n, dtype=np.int32), type=np.zeros(n, np.int32),
                        box=np.array([[L, L, L]]), offsets=np.array([0, n], np.int64))


@pytest.mark.parametrize("w", (1, 2))
def test_pairs_at_the_fp32_band_ends(w):
    """Every pair inside r_list is listed and every pair inside r_cut feels
    its force, in both precisions, also where the FP32 r^2 falls within an
    ulp or two of the band's rounded ends (a threshold that left a sliver
    between the FP32 decision and the FP64 re-test dropped such pairs)."""
    st = band_ends_state(seed=80 + w)
    L = st.box[0]
    cb, rb = oracle.neighbors(st.pos, L, 2.8, max_nb=32, method="cells")
    ref, _, absf = oracle.lj_forces(st.pos, L, 2.5)
    assert 150 < np.sum(cb) // 2 < 400 and np.sum(absf > 0) > 100
    for prec in ("fp64", "mixed"):
        s = md.MDSystem(st, r_cut=2.5, r_skin=0.3, dt=0.005, precision=prec, max_nb=32)
        s.set_tuning(md.KERNEL_PAIR, 128, w)
        s.set_tuning(md.KERNEL_NLIST, 64, w)
        s.prepare()
        counts, rows = (x.cpu().numpy() for x in s.nlist())
        assert np.array_equal(counts, cb), prec
        for i in np.nonzero(cb)[0]:
            assert np.array_equal(np.sort(rows[i, :counts[i]]), rb[i, :cb[i]]), (prec, i)
        f = s.forces().cpu().numpy()
        s.check_error()
        # isolated pairs: a particle feels a force iff its partner is inside r_cut
        assert np.array_equal(np.linalg.norm(f[:, :3], axis=1) > 0, absf > 0), prec
        if prec == "fp64":
            fp64_force_check(f, ref, absf)
        else:
            rms, mx = mixed_force_stats(f, ref, absf)
            assert rms <= 1e-5 and mx <= 1e-3, (rms, mx)
        s.close()
