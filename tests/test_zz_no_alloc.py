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
