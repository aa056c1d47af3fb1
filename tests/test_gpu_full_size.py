"""Parity at the headline size: the 16,777,216-particle LJ fluid (density
0.8442, T = 1.2, r_cut = 2.5, skin = 0.4, dt = 0.005) in the launch
configuration the benchmark times (mixed precision; pair kernel w = 2 with
128 threads, list build w = 1 with 192 threads; space-filling-curve sort at
every rebuild; 100-step CUDA graphs).

The system starts as the benchmark does (the fcc lattice, seed 12345).
After a run with rebuilds and sorts, the list is rebuilt on the final
positions and the forces computed.  For a sample of particles the oracle
gives each one's exact neighbour row and force from a local system: the
particle and every particle of the 27 cells around it, in the same periodic
box.  The list radius is at most the cell width, so that set holds all of the
particle's neighbours and every pair within the cut-off.  Tolerances as in
test_gpu_parity: rows bit-exact; mixed forces RMS relative error <= 1e-5 and
max <= 1e-3; FP64 forces |dF| <= 1e-12 |F| (|F| >= 1e-2 S, else 1e-14 S).
"""
import time

import numpy as np
import pytest

import oracle
from paper_1412_3387_gb300 import inputs
from local_ref import local_reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_3387_gb300 import md  # noqa: E402

N = 16_777_216
R_CUT, R_SKIN = 2.5, 0.4
KW = dict(r_cut=R_CUT, r_skin=R_SKIN, dt=0.005, thermo_period=100, graph_steps=100,
          sort_period=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1412_3387_gb300 import build
    build.build()
    oracle.build()


def gpu_rows(s, samples):
    counts, rows = s.nlist()
    sel = torch.as_tensor(samples, device=counts.device)
    c = counts[sel].cpu().numpy()
    r = rows[sel].cpu().numpy()
    del counts, rows
    torch.cuda.empty_cache()
    return [np.sort(r[k, :c[k]]) for k in range(len(samples))]


def test_headline_fluid_sampled_rows_and_forces():
    st = inputs.lj_fluid(N, 0.8442, 1.2, seed=12345)
    L = st.box[0, 0]
    s = md.MDSystem(st, precision="mixed", **KW)
    s.set_tuning(md.KERNEL_PAIR, 128, 2)
    s.set_tuning(md.KERNEL_NLIST, 192, 1)
    s.prepare()
    t0 = time.perf_counter()
    s.run(200)
    s.check_error()
    assert time.perf_counter() - t0 < 60.0  # about 1.2 s on a GB300
    assert s.info()["n_builds"] > 1  # the run rebuilt (and sorted) the list
    s.build_cells(True)
    s.build_nlist(True)
    s.compute_pair(False)
    s.check_error()
    g = s.state_numpy()
    pos = np.ascontiguousarray(g["pos"])  # [N, 4], as the oracle takes it

    rng = np.random.default_rng(7)
    # random particles plus the ones closest to each face of the box
    edge = np.concatenate([np.argsort(pos[:, k])[:4] for k in range(3)] +
                          [np.argsort(pos[:, k])[-4:] for k in range(3)])
    samples = np.unique(np.concatenate([rng.choice(N, 1500, replace=False), edge]))

    rows_ref, f_ref, absf = local_reference(pos, L, samples, R_CUT, R_SKIN)
    rows_mixed = gpu_rows(s, samples)
    for k, i in enumerate(samples):
        assert np.array_equal(rows_mixed[k], rows_ref[k]), int(i)

    f = s.forces().cpu().numpy()[samples]
    d = np.linalg.norm(f[:, :3] - f_ref[:, :3], axis=1)
    F = np.linalg.norm(f_ref[:, :3], axis=1)
    big = F >= 1e-2 * absf
    rel = d[big] / F[big]
    assert big.sum() > 1000
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-5, np.sqrt(np.mean(rel ** 2))
    assert rel.max() <= 1e-3, rel.max()
    s.close()
    del s
    torch.cuda.empty_cache()

    # the plain FP64 path on the same positions
    st64 = st.copy()
    for k in ("pos", "vel", "image", "tag", "type"):
        setattr(st64, k, g[k])
    s64 = md.MDSystem(st64, precision="fp64", **KW)
    s64.set_tuning(md.KERNEL_PAIR, 128, 2)
    s64.set_tuning(md.KERNEL_NLIST, 192, 1)
    s64.prepare()
    s64.check_error()
    rows64 = gpu_rows(s64, samples)
    for k, i in enumerate(samples):
        assert np.array_equal(rows64[k], rows_ref[k]), int(i)
    f64 = s64.forces().cpu().numpy()[samples]
    d = np.linalg.norm(f64[:, :3] - f_ref[:, :3], axis=1)
    assert np.all(d[big] <= 1e-12 * F[big]), np.max(d[big] / F[big])
    assert np.all(d[~big] <= 1e-14 * absf[~big] + 1e-300)
    s64.close()
