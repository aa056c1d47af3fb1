"""md_lj_forces_noalloc: the entry point for callers that cannot allocate
device memory (it keeps its cell-list scratch in a fixed array inside the
library instead of a caller workspace).

Its forces must match the regular path's (md_create_system + md_build_cells +
md_build_nlist + md_compute_pair) within the FP64 force tolerance used by the
parity tests, on two calls in a row with different systems, so that whatever
the first call left in the shared scratch cannot leak into the second.  This
file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_1412_3387_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3387_gb300 import build, md  # noqa: E402


def _regular_path_forces(st, r_cut):
    s = md.MDSystem(st, r_cut=r_cut, r_skin=0.3, dt=0.005, precision="fp64")
    s.build_cells()
    s.build_nlist()
    s.compute_pair(want_virial=True)
    f = s.forces().cpu().numpy()
    s.check_error()
    s.close()
    return f


def _check(f_new, f_ref):
    # same tolerance as the FP64 parity tests, with S estimated by the largest
    # force magnitude (the two sides sum the same pairs in different orders)
    d = np.linalg.norm(f_new[:, :3] - f_ref[:, :3], axis=1)
    F = np.linalg.norm(f_ref[:, :3], axis=1)
    scale = np.abs(f_ref[:, :3]).max()
    big = F >= 1e-2 * scale
    assert np.all(d[big] <= 1e-12 * F[big])
    assert np.all(d[~big] <= 1e-13 * scale)
    assert np.allclose(f_new[:, 3], f_ref[:, 3], rtol=1e-12, atol=1e-13 * scale)


def test_noalloc_matches_regular_path_on_two_calls():
    build.build()
    a = inputs.lj_fluid(4000, 0.8442, 1.2, seed=61, jitter=0.12)
    b = inputs.lj_fluid(1500, 0.70, 1.0, seed=62, jitter=0.15)
    ref_a = _regular_path_forces(a, 2.5)
    ref_b = _regular_path_forces(b, 2.2)
    pa = torch.as_tensor(a.pos, device="cuda")
    pb = torch.as_tensor(b.pos, device="cuda")
    fa = md.lj_forces_noalloc(pa, a.box[0], 2.5).cpu().numpy()
    fb = md.lj_forces_noalloc(pb, b.box[0], 2.2).cpu().numpy()
    _check(fa, ref_a)
    _check(fb, ref_b)
    # and the first system again, after the second one used the scratch
    fa2 = md.lj_forces_noalloc(pa, a.box[0], 2.5).cpu().numpy()
    _check(fa2, ref_a)


def test_noalloc_rejects_systems_beyond_its_scratch():
    st = inputs.lj_fluid(500_000, 0.8442, 1.2, seed=63)  # 3 n > 1,048,576 ints
    p = torch.as_tensor(st.pos, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.lj_forces_noalloc(p, st.box[0], 2.5)
    assert e.value.code == 3  # MD_ERR_WORKSPACE_TOO_SMALL
    small = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.lj_forces_noalloc(small, [5.0, 5.0, 5.0], 2.5)  # 2 cells per edge
    assert e.value.code == 5  # MD_ERR_CELL_GRID


def _check_vs_oracle(f_new, pos, box, r_cut, brute=None):
    """The FP64 parity rule of the other GPU tests against the oracle's
    forces: |dF| <= 1e-12 |F| where |F| >= 1e-2 S, else <= 1e-14 S, with S
    the oracle's sum of pair-force magnitudes (all-pairs oracle for small or
    unwrapped inputs, its cell list otherwise)."""
    if brute is None:
        brute = len(pos) < 5000
    nl = oracle.neighbors(pos, box, r_cut, max_nb=128, method="brute" if brute else "cells")
    ref, _, absf = oracle.lj_forces(pos, box, r_cut, nlist=nl)
    d = np.linalg.norm(f_new[:, :3] - ref[:, :3], axis=1)
    F = np.linalg.norm(ref[:, :3], axis=1)
    big = F >= 1e-2 * absf
    assert np.all(d[big] <= 1e-12 * F[big]), np.max(d[big] / F[big])
    assert np.all(d[~big] <= 1e-14 * absf[~big] + 1e-300)
    assert np.allclose(f_new[:, 3], ref[:, 3], rtol=1e-12, atol=1e-12 * absf.max())


def _lattice_state(counts, seed, jitter=0.1, vacancies=0, rho=0.8442):
    """Jittered simple-cubic lattice at density rho in an orthorhombic box of
    counts[d] lattice spacings per edge, with `vacancies` seeded empty sites."""
    rng = np.random.default_rng(seed)
    a = (1.0 / rho) ** (1.0 / 3.0)
    g = np.stack(np.meshgrid(*[np.arange(c) for c in counts], indexing="ij"), -1).reshape(-1, 3)
    if vacancies:
        g = g[np.sort(rng.permutation(len(g))[:len(g) - vacancies])]
    xyz = (g + 0.5 + rng.uniform(-jitter, jitter, g.shape)) * a
    n = len(g)
    box = np.array(counts, np.float64) * a
    pos = np.zeros((n, 4))
    pos[:, :3] = np.mod(xyz, box)
    return inputs.State(pos=pos, vel=np.zeros((n, 4)), image=np.zeros((n, 4), np.int32),
                        tag=np.arange(n, dtype=np.int32), type=np.zeros(n, np.int32),
                        box=box[None, :], offsets=np.array([0, n], np.int64))


def test_noalloc_accepts_exactly_its_scratch_and_refuses_one_more():
    # 69 x 69 x 70 sites less 4 vacancies: 333,266 particles in 29^3 cells of
    # r_cut = 2.5, i.e. 2 * 24,389 + 3 * 333,266 = 1,048,576 ints, the whole array
    st = _lattice_state((69, 69, 70), seed=64, vacancies=4)
    assert 2 * 29 ** 3 + 3 * st.n == 1 << 20
    p = torch.as_tensor(st.pos, device="cuda")
    _check_vs_oracle(md.lj_forces_noalloc(p, st.box[0], 2.5).cpu().numpy(), st.pos, st.box[0],
                     2.5)
    st1 = _lattice_state((69, 69, 70), seed=64, vacancies=3)  # one particle more
    p1 = torch.as_tensor(st1.pos, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.lj_forces_noalloc(p1, st1.box[0], 2.5)
    assert e.value.code == 3  # MD_ERR_WORKSPACE_TOO_SMALL


def test_noalloc_noncubic_box_and_unwrapped_positions():
    st = _lattice_state((20, 28, 36), seed=65)
    p = torch.as_tensor(st.pos, device="cuda")
    f = md.lj_forces_noalloc(p, st.box[0], 2.5).cpu().numpy()
    _check_vs_oracle(f, st.pos, st.box[0], 2.5)
    # the positions shifted by whole box lengths (callers need not wrap); the
    # shifted inputs are rounded (an ulp of ~4 L), so they are compared with
    # the oracle on the same shifted inputs
    shift = np.random.default_rng(5).integers(-3, 4, (st.n, 3)) * st.box[0]
    q = st.pos.copy()
    q[:, :3] += shift
    fq = md.lj_forces_noalloc(torch.as_tensor(q, device="cuda"), st.box[0], 2.5).cpu().numpy()
    _check_vs_oracle(fq, q, st.box[0], 2.5, brute=True)


def test_noalloc_box_an_exact_multiple_of_r_cut():
    # box 10 = 4 r_cut: cells are 10 / 3 wide (the 1e-12 margin), and pairs
    # straddling the planes x = k r_cut at r_cut (1 - 1e-14) still interact
    L, rc = 10.0, 2.5
    d = rc * (1 - 1e-14)
    yz = ((0.5, 0.5), (5.5, 0.5), (0.5, 5.5), (5.5, 5.5))  # pairs >= 5 apart
    pos = np.zeros((8, 4))
    for k, x0 in enumerate((2.5, 5.0, 7.5, 10.0)):
        pos[2 * k, :3] = [x0 - 0.5 * d, *yz[k]]
        pos[2 * k + 1, :3] = [x0 + 0.5 * d, *yz[k]]
    pos[:, :3] = np.mod(pos[:, :3], L)
    f = md.lj_forces_noalloc(torch.as_tensor(pos, device="cuda"), [L, L, L], rc).cpu().numpy()
    _, _, absf = oracle.lj_forces(pos, L, rc)
    assert np.all(absf > 0)  # each particle feels its partner, inside r_cut
    _check_vs_oracle(f, pos, np.array([L, L, L]), rc)


def test_noalloc_long_box_beyond_the_cell_cap():
    # 2600 / 2.5 = 1040 cells along x, capped at 1024 (cells 2.54 wide)
    rng = np.random.default_rng(67)
    n = 3000
    box = np.array([2600.0, 9.0, 9.0])
    pos = np.zeros((n, 4))
    pos[:, :3] = rng.uniform(0.0, 1.0, (n, 3)) * box
    st = inputs.State(pos=pos, vel=np.zeros((n, 4)), image=np.zeros((n, 4), np.int32),
                      tag=np.arange(n, dtype=np.int32), type=np.zeros(n, np.int32),
                      box=box[None, :], offsets=np.array([0, n], np.int64))
    f = md.lj_forces_noalloc(torch.as_tensor(pos, device="cuda"), box, 2.5).cpu().numpy()
    _check_vs_oracle(f, pos, box, 2.5)
