"""The C-ABI library loads and exports every symbol include/md.h declares;
host-only entry points (no GPU needed) validate their arguments."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1412_3387_gb300 import build, md

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return md.load()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(md.SIGNATURES), set(md.SIGNATURES) ^ names


def test_abi_version_and_status_strings(lib):
    assert lib.md_abi_version() == 8
    for code in range(11):
        assert lib.md_status_string(code)


def _params(n=4000, L=16.8, r_cut=2.5, r_skin=0.3, R=1, **kw):
    off = np.linspace(0, n, R + 1).astype(np.int64)
    box = np.full((R, 3), L)
    coeff = np.array([1.0, 1.0])
    p = md.Params()
    p.n_total, p.n_replicas = n, R
    p.replica_offset, p.box = off.ctypes.data, box.ctypes.data
    p.r_cut, p.r_skin, p.dt, p.mass, p.kT = r_cut, r_skin, 0.005, 1.0, 1.0
    p.pair, p.n_types, p.pair_coeff = md.LJ, 1, coeff.ctypes.data
    p.precision, p.max_nb = md.FP64, 128
    for k, v in kw.items():
        setattr(p, k, v)
    return p, (off, box, coeff)


def _size(lib, p):
    s = C.c_size_t()
    code = lib.md_workspace_size(C.byref(p), C.byref(s))
    return code, s.value


def test_workspace_size_grows_with_n_and_max_nb(lib):
    p, keep = _params()
    code, s1 = _size(lib, p)
    assert code == md.MD_OK and s1 > 4000 * 128 * 4
    p.max_nb = 256
    assert _size(lib, p)[1] > s1
    p2, keep2 = _params(n=8000, L=21.2)
    assert _size(lib, p2)[1] > s1
    p3, keep3 = _params(precision=md.MIXED)
    assert _size(lib, p3)[1] < s1  # FP32 force and virial arrays


def test_workspace_size_rejects_bad_parameters(lib):
    for kw in (dict(r_cut=0.0), dict(r_skin=-1.0), dict(dt=0.0), dict(n_types=0),
               dict(pair=7), dict(precision=3), dict(max_nb=0), dict(sort_period=-1),
               dict(graph_steps=10, thermo_period=3), dict(n_total=2 ** 27 + 1)):
        p, keep = _params(**kw)
        assert _size(lib, p)[0] == 1, kw  # MD_ERR_INVALID_ARG
    p, keep = _params(L=7.0)  # 7 / 2.8 -> 2 cells per edge
    assert _size(lib, p)[0] == 5  # MD_ERR_CELL_GRID


def test_workspace_size_batched_replicas(lib):
    p, keep = _params(n=8000, R=4, L=16.8)
    code, s = _size(lib, p)
    assert code == md.MD_OK
    off = np.array([0, 10, 5, 8000], np.int64)  # non-monotone offsets
    p.replica_offset = off.ctypes.data
    p.n_replicas = 3
    assert _size(lib, p)[0] == 1


def test_null_handles_are_rejected(lib):
    assert lib.md_destroy_system(None) == 1
    assert lib.md_step(None, 0, None) == 1
    assert lib.md_poll_error(None, None) == 1
    assert lib.md_philox4x32_10(None, None, 5, None) == 1


def test_workspace_size_checks_potential_arguments(lib):
    """Host-side checks of the potentials' parameters: coefficient arrays must
    be finite (3 per type pair for Morse), a tabulated pair needs 2 .. 65536
    samples per type pair (and no coefficients), at most 64 angles per
    particle, and a DPD temperature must be non-negative."""
    morse = np.array([1.0, 2.0, 1.1])
    p, keep = _params(pair=md.MORSE)
    p.pair_coeff = morse.ctypes.data
    assert _size(lib, p)[0] == md.MD_OK
    bad = np.array([1.0, float("nan"), 1.1])
    p.pair_coeff = bad.ctypes.data
    assert _size(lib, p)[0] == 1
    for pts, want in ((1, 1), (2, md.MD_OK), (65536, md.MD_OK), (65537, 1)):
        p, keep = _params(pair=md.TABLE, table_points=pts)
        p.pair_coeff = None
        assert _size(lib, p)[0] == want, pts
    for na, want in ((64, md.MD_OK), (65, 1), (-1, 1)):
        p, keep = _params(max_angles=na)
        assert _size(lib, p)[0] == want, na
    p, keep = _params(pair=md.DPD, kT=-1.0)
    assert _size(lib, p)[0] == 1
