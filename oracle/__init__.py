"""CPU FP64 oracle for the short-range MD hot path (Python side).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path; its arithmetic lives in ``oracle.c`` (plain C, FP64,
compiled with -ffp-contract=off), and this module only marshals NumPy arrays.

Every function cites, in oracle.h / oracle.c, the section of Glaser et al.
(arXiv:1412.3387) or the textbook definition it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP, no FMA)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3), ("r_cut", C.c_double), ("r_skin", C.c_double),
        ("dt", C.c_double), ("mass", C.c_double), ("kT", C.c_double),
        ("seed", C.c_uint64), ("pair", C.c_int32), ("ntypes", C.c_int32),
        ("coeff", C.c_void_p), ("shift_energy", C.c_int32),
        ("thermo_period", C.c_int32), ("K", C.c_double), ("r0", C.c_double),
        ("n_bonds", C.c_int64), ("bonds", C.c_void_p), ("step0", C.c_int64),
        ("max_nb", C.c_int32), ("integrator", C.c_int32), ("t_kT", C.c_double),
        ("t_gamma", C.c_double), ("t_tau", C.c_double), ("t_seed", C.c_uint64),
        ("nh_state", C.c_void_p), ("bond_style", C.c_int32),
        ("n_angles", C.c_int64), ("angles", C.c_void_p), ("angle_K", C.c_double),
        ("angle_theta0", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = C.CDLL(so)
            P, I64, I32, D, U64, U32 = (C.c_void_p, C.c_int64, C.c_int32, C.c_double,
                                         C.c_uint64, C.c_uint32)
            sig = {
                "orc_cells_per_dim": (I32, [D, D]),
                "orc_cell_coords": (None, [I64, P, P, P, P]),
                "orc_neighbors_brute": (I32, [I64, P, P, D, P, P, I32]),
                "orc_neighbors_cells": (I32, [I64, P, P, D, P, P, I32]),
                "orc_lj_pair": (D, [D, D, D, P]),
                "orc_pair_ncoeff": (I32, [I32]),
                "orc_table_eval": (D, [D, P, I32, D, D, P]),
                "orc_table_forces_brute": (None, [I64, P, P, P, D, I32, P, I32, D, P, P, P]),
                "orc_pair_eval": (D, [I32, D, P, P]),
                "orc_pair_forces_brute": (None, [I32, I64, P, P, P, D, I32, P, I32, P, P, P]),
                "orc_pair_forces_nlist": (None, [I32, I64, P, P, P, D, I32, P, I32, P, P, I32, P, P, P]),
                "orc_lj_forces_brute": (None, [I64, P, P, P, D, I32, P, I32, P, P, P]),
                "orc_lj_forces_nlist": (None, [I64, P, P, P, D, I32, P, I32, P, P, I32, P, P, P]),
                "orc_philox4x32_10": (None, [P, P, P]),
                "orc_dpd_theta": (D, [I32, I32, U64, U64]),
                "orc_dpd_forces_brute": (None, [I64, P, P, P, P, P, D, I32, P, D, D, U64, U64, P, P, P]),
                "orc_dpd_forces_nlist": (None, [I64, P, P, P, P, P, D, I32, P, D, D, U64, U64, P, P, I32, P, P, P]),
                "orc_bond_forces": (None, [I64, P, P, P, D, D, P, P, P]),
                "orc_fene_bond_forces": (I64, [I64, P, P, P, D, D, P, P, P]),
                "orc_angle_forces": (None, [I64, P, P, P, D, D, P, P, P]),
                "orc_vv_first": (None, [I64, P, P, P, P, D, D, P]),
                "orc_vv_second": (None, [I64, P, P, D, D]),
                "orc_thermo": (None, [I64, P, P, P, D, P, P]),
                "orc_hilbert3": (U64, [U32, U32, U32, I32]),
                "orc_sfc_order": (None, [I64, P, P, D, P]),
                "orc_run": (I64, [I64, P, P, P, P, P, P, C.POINTER(Params), I64, P]),
                "orc_langevin_noise": (None, [I32, U64, U64, P]),
                "orc_baoab_first": (None, [I64, P, P, P, P, P, D, D, D, D, U64, U64, P]),
                "orc_nh_half": (D, [I64, P, D, D, D, D, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _box(L):
    L = np.asarray(L, np.float64).reshape(-1)
    if L.size == 1:
        L = np.repeat(L, 3)
    return np.ascontiguousarray(L[:3])


def cells_per_dim(L: float, r_list: float) -> int:
    return int(lib().orc_cells_per_dim(float(L), float(r_list)))


def cell_coords(pos, L, nc):
    pos = _f64(pos)
    nc = np.ascontiguousarray(nc, np.int32)
    out = np.zeros((pos.shape[0], 3), np.int32)
    lib().orc_cell_coords(pos.shape[0], _p(pos), _p(_box(L)), _p(nc), _p(out))
    return out


def neighbors(pos, L, r_list, max_nb=256, method="brute"):
    """Full neighbour rows: (counts[N], rows[N, max_nb]) with ascending j."""
    pos = _f64(pos)
    n = pos.shape[0]
    counts = np.zeros(n, np.int32)
    rows = np.full((n, max_nb), -1, np.int32)
    fn = lib().orc_neighbors_brute if method == "brute" else lib().orc_neighbors_cells
    longest = fn(n, _p(pos), _p(_box(L)), float(r_list), _p(counts), _p(rows), max_nb)
    if longest > max_nb:
        raise ValueError(f"neighbour row of {longest} exceeds max_nb={max_nb}")
    return counts, rows


def lj_pair(r2, eps=1.0, sigma=1.0):
    v = C.c_double()
    fr = lib().orc_lj_pair(float(r2), float(eps), float(sigma), C.byref(v))
    return fr, v.value


def _coeff(coeff, ntypes, k=2):
    c = np.ascontiguousarray(coeff, np.float64).reshape(ntypes, ntypes, k)
    return c


# pair kinds (oracle.h): coefficients per ordered type pair
PAIR_KINDS = {"lj": 0, "dpd": 1, "gauss": 2, "morse": 3, "yukawa": 4}


def pair_ncoeff(pair):
    return int(lib().orc_pair_ncoeff(PAIR_KINDS[pair]))


def pair_eval(pair, r2, c):
    """(-dV/dr / r, V) of one pair at r^2 (kinds lj, gauss, morse, yukawa)."""
    v = C.c_double()
    cc = np.ascontiguousarray(c, np.float64)
    fr = lib().orc_pair_eval(PAIR_KINDS[pair], float(r2), _p(cc), C.byref(v))
    return fr, v.value


def pair_forces(pair, pos, L, r_cut, coeff, type=None, shift_energy=False, nlist=None):
    """(force[N,4], virial[N,6], absf[N]) of kind lj, gauss, morse or yukawa,
    from brute force or given rows."""
    kind = PAIR_KINDS[pair]
    k = pair_ncoeff(pair)
    pos = _f64(pos)
    n = pos.shape[0]
    ntypes = int(round(np.sqrt(np.asarray(coeff, np.float64).size / k)))
    c = _coeff(coeff, ntypes, k)
    t = _i32(np.zeros(n) if type is None else type)
    force = np.zeros((n, 4))
    virial = np.zeros((n, 6))
    absf = np.zeros(n)
    if nlist is None:
        lib().orc_pair_forces_brute(kind, n, _p(pos), _p(t), _p(_box(L)), float(r_cut), ntypes,
                                    _p(c), int(shift_energy), _p(force), _p(virial), _p(absf))
    else:
        counts, rows = nlist
        counts, rows = _i32(counts), _i32(rows)
        lib().orc_pair_forces_nlist(kind, n, _p(pos), _p(t), _p(_box(L)), float(r_cut), ntypes,
                                    _p(c), int(shift_energy), _p(counts), _p(rows),
                                    rows.shape[1], _p(force), _p(virial), _p(absf))
    return force, virial, absf


def lj_forces(pos, L, r_cut, coeff=((1.0, 1.0),), type=None, shift_energy=False,
              nlist=None):
    """(force[N,4], virial[N,6], absf[N]) from brute force or given rows."""
    pos = _f64(pos)
    n = pos.shape[0]
    ntypes = int(round(np.sqrt(np.asarray(coeff, np.float64).size / 2)))
    c = _coeff(coeff, ntypes)
    t = _i32(np.zeros(n) if type is None else type)
    force = np.zeros((n, 4))
    virial = np.zeros((n, 6))
    absf = np.zeros(n)
    if nlist is None:
        lib().orc_lj_forces_brute(n, _p(pos), _p(t), _p(_box(L)), float(r_cut), ntypes,
                                  _p(c), int(shift_energy), _p(force), _p(virial), _p(absf))
    else:
        counts, rows = nlist
        counts, rows = _i32(counts), _i32(rows)
        lib().orc_lj_forces_nlist(n, _p(pos), _p(t), _p(_box(L)), float(r_cut), ntypes,
                                  _p(c), int(shift_energy), _p(counts), _p(rows),
                                  rows.shape[1], _p(force), _p(virial), _p(absf))
    return force, virial, absf


def table_eval(r2, tab, r_min, r_cut):
    """(F(r)/r, V) of a tabulated pair ([n_points][2] samples of V, F)."""
    t = np.ascontiguousarray(tab, np.float64).reshape(-1, 2)
    v = C.c_double()
    fr = lib().orc_table_eval(float(r2), _p(t), t.shape[0], float(r_min), float(r_cut),
                              C.byref(v))
    return fr, v.value


def table_forces(pos, L, r_cut, table, r_min, type=None):
    """(force, virial, absf) of a tabulated pair potential, brute force;
    table [ntypes][ntypes][n_points][2]."""
    pos = _f64(pos)
    n = pos.shape[0]
    tab = np.ascontiguousarray(table, np.float64)
    ntypes = tab.shape[0]
    t = _i32(np.zeros(n) if type is None else type)
    force = np.zeros((n, 4))
    virial = np.zeros((n, 6))
    absf = np.zeros(n)
    lib().orc_table_forces_brute(n, _p(pos), _p(t), _p(_box(L)), float(r_cut), ntypes, _p(tab),
                                 tab.shape[2], float(r_min), _p(force), _p(virial), _p(absf))
    return force, virial, absf


def philox4x32_10(ctr, key):
    ctr = np.ascontiguousarray(ctr, np.uint32)
    key = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(ctr), _p(key), _p(out))
    return out


def dpd_theta(tag_i, tag_j, step, seed):
    return lib().orc_dpd_theta(int(tag_i), int(tag_j), int(step), int(seed))


def dpd_forces(pos, vel, L, r_cut, coeff, kT, dt, step, seed, type=None, tag=None,
               nlist=None):
    pos, vel = _f64(pos), _f64(vel)
    n = pos.shape[0]
    ntypes = int(round(np.sqrt(np.asarray(coeff, np.float64).size / 2)))
    c = _coeff(coeff, ntypes)
    t = _i32(np.zeros(n) if type is None else type)
    g = _i32(np.arange(n) if tag is None else tag)
    force = np.zeros((n, 4))
    virial = np.zeros((n, 6))
    absf = np.zeros(n)
    if nlist is None:
        lib().orc_dpd_forces_brute(n, _p(pos), _p(vel), _p(t), _p(g), _p(_box(L)),
                                   float(r_cut), ntypes, _p(c), float(kT), float(dt),
                                   int(step), int(seed), _p(force), _p(virial), _p(absf))
    else:
        counts, rows = nlist
        counts, rows = _i32(counts), _i32(rows)
        lib().orc_dpd_forces_nlist(n, _p(pos), _p(vel), _p(t), _p(g), _p(_box(L)),
                                   float(r_cut), ntypes, _p(c), float(kT), float(dt),
                                   int(step), int(seed), _p(counts), _p(rows),
                                   rows.shape[1], _p(force), _p(virial), _p(absf))
    return force, virial, absf


def bond_forces(bonds, pos, L, K, r0, force=None, virial=None, absf=None):
    """Adds harmonic-bond forces to (force, virial, absf); returns them."""
    pos = _f64(pos)
    n = pos.shape[0]
    bonds = _i32(bonds).reshape(-1, 2)
    force = np.zeros((n, 4)) if force is None else _f64(force).copy()
    virial = np.zeros((n, 6)) if virial is None else _f64(virial).copy()
    absf = np.zeros(n) if absf is None else _f64(absf).copy()
    lib().orc_bond_forces(bonds.shape[0], _p(bonds), _p(pos), _p(_box(L)), float(K),
                          float(r0), _p(force), _p(virial), _p(absf))
    return force, virial, absf


def fene_bond_forces(bonds, pos, L, K, R0, force=None, virial=None, absf=None):
    """Adds FENE-bond forces to (force, virial, absf); returns them and the
    number of bonds stretched to R0 or beyond (skipped)."""
    pos = _f64(pos)
    n = pos.shape[0]
    bonds = _i32(bonds).reshape(-1, 2)
    force = np.zeros((n, 4)) if force is None else _f64(force).copy()
    virial = np.zeros((n, 6)) if virial is None else _f64(virial).copy()
    absf = np.zeros(n) if absf is None else _f64(absf).copy()
    broken = lib().orc_fene_bond_forces(bonds.shape[0], _p(bonds), _p(pos), _p(_box(L)),
                                        float(K), float(R0), _p(force), _p(virial), _p(absf))
    return force, virial, absf, int(broken)


def angle_forces(angles, pos, L, K, theta0, force=None, virial=None, absf=None):
    """Adds harmonic-angle forces (index triplets, vertex in the middle) to
    (force, virial, absf); returns them."""
    pos = _f64(pos)
    n = pos.shape[0]
    tri = _i32(angles).reshape(-1, 3)
    force = np.zeros((n, 4)) if force is None else _f64(force).copy()
    virial = np.zeros((n, 6)) if virial is None else _f64(virial).copy()
    absf = np.zeros(n) if absf is None else _f64(absf).copy()
    lib().orc_angle_forces(tri.shape[0], _p(tri), _p(pos), _p(_box(L)), float(K), float(theta0),
                           _p(force), _p(virial), _p(absf))
    return force, virial, absf


def vv_first(pos, vel, image, force, dt, L, mass=1.0):
    pos, vel, force = _f64(pos).copy(), _f64(vel).copy(), _f64(force)
    image = _i32(image).copy()
    lib().orc_vv_first(pos.shape[0], _p(pos), _p(vel), _p(image), _p(force), float(dt),
                       float(mass), _p(_box(L)))
    return pos, vel, image


def vv_second(vel, force, dt, mass=1.0):
    vel, force = _f64(vel).copy(), _f64(force)
    lib().orc_vv_second(vel.shape[0], _p(vel), _p(force), float(dt), float(mass))
    return vel


THERMO_FIELDS = ("ke", "pe", "virial", "pressure", "temperature", "px", "py", "pz")


def thermo(vel, force, virial, L, mass=1.0):
    vel, force = _f64(vel), _f64(force)
    vir = None if virial is None else _f64(virial)
    out = np.zeros(8)
    lib().orc_thermo(vel.shape[0], _p(vel), _p(force), _p(vir), float(mass),
                     _p(_box(L)), _p(out))
    return dict(zip(THERMO_FIELDS, out.tolist()))


def hilbert3(x, y, z, bits):
    return int(lib().orc_hilbert3(int(x), int(y), int(z), int(bits)))


def sfc_order(pos, L, r_list):
    pos = _f64(pos)
    order = np.zeros(pos.shape[0], np.int32)
    lib().orc_sfc_order(pos.shape[0], _p(pos), _p(_box(L)), float(r_list), _p(order))
    return order


def langevin_noise(tag, step, seed):
    out = np.zeros(3)
    lib().orc_langevin_noise(int(tag), int(step), int(seed), _p(out))
    return out


def baoab_first(pos, vel, image, force, tag, dt, gamma, kT, step, seed, L, mass=1.0):
    pos, vel, force = _f64(pos).copy(), _f64(vel).copy(), _f64(force)
    image, tag = _i32(image).copy(), _i32(tag)
    lib().orc_baoab_first(pos.shape[0], _p(pos), _p(vel), _p(image), _p(force), _p(tag),
                          float(dt), float(mass), float(gamma), float(kT), int(step), int(seed),
                          _p(_box(L)))
    return pos, vel, image


def nh_half(vel, kT, tau, dt, state, mass=1.0):
    """One Nose-Hoover half step on a copy of vel; state = [xi, eta] is
    updated in place.  Returns (vel, scale)."""
    vel = _f64(vel).copy()
    st = np.ascontiguousarray(state, np.float64)
    s = lib().orc_nh_half(vel.shape[0], _p(vel), float(mass), float(kT), float(tau), float(dt),
                          _p(st))
    state[:] = st
    return vel, s


INTEGRATORS = {"nve": 0, "langevin": 1, "nose-hoover": 2}


def run(pos, vel, image, L, n_steps, *, r_cut, r_skin, dt, pair="lj", type=None,
        tag=None, coeff=((1.0, 1.0),), kT=1.0, seed=0, mass=1.0, shift_energy=False,
        thermo_period=0, bonds=None, K=0.0, r0=0.0, step0=0, max_nb=256,
        integrator="nve", t_kT=1.0, gamma=1.0, tau=1.0, t_seed=0, nh_state=None,
        bond_style="harmonic", angles=None, angle_K=0.0, angle_theta0=0.0):
    """Full MD loop on copies of the inputs; returns a dict with the final
    state, forces, thermo rows, the number of list builds and (Nose-Hoover)
    the thermostat state [xi, eta] (nh_state gives its initial value)."""
    pos, vel = _f64(pos).copy(), _f64(vel).copy()
    image = _i32(image).copy()
    n = pos.shape[0]
    k = pair_ncoeff(pair)
    ntypes = int(round(np.sqrt(np.asarray(coeff, np.float64).size / k)))
    c = _coeff(coeff, ntypes, k)
    t = _i32(np.zeros(n) if type is None else type)
    g = _i32(np.arange(n) if tag is None else tag)
    b = _i32(np.zeros((0, 2)) if bonds is None else bonds).reshape(-1, 2)
    force = np.zeros((n, 4))
    p = Params()
    p.L = (C.c_double * 3)(*_box(L).tolist())
    p.r_cut, p.r_skin, p.dt, p.mass, p.kT = r_cut, r_skin, dt, mass, kT
    p.seed = int(seed)
    p.pair = PAIR_KINDS[pair]
    p.ntypes = ntypes
    p.coeff = c.ctypes.data
    p.shift_energy = int(shift_energy)
    p.thermo_period = int(thermo_period)
    p.K, p.r0 = K, r0
    p.n_bonds = b.shape[0]
    p.bonds = b.ctypes.data if b.shape[0] else None
    p.step0 = int(step0)
    p.max_nb = int(max_nb)
    p.integrator = INTEGRATORS[integrator]
    p.t_kT, p.t_gamma, p.t_tau, p.t_seed = float(t_kT), float(gamma), float(tau), int(t_seed)
    nh = np.ascontiguousarray(np.zeros(2) if nh_state is None else nh_state, np.float64).copy()
    p.nh_state = nh.ctypes.data
    p.bond_style = {"harmonic": 0, "fene": 1}[bond_style]
    tri = _i32(np.zeros((0, 3)) if angles is None else angles).reshape(-1, 3)
    p.n_angles = tri.shape[0]
    p.angles = tri.ctypes.data if tri.shape[0] else None
    p.angle_K, p.angle_theta0 = float(angle_K), float(angle_theta0)
    n_th = (n_steps // thermo_period + 1) if thermo_period else 0
    th = np.zeros((max(n_th, 1), 8))
    builds = lib().orc_run(n, _p(pos), _p(vel), _p(image), _p(t), _p(g), _p(force),
                           C.byref(p), int(n_steps), _p(th))
    if builds < 0:
        raise ValueError("neighbour row overflow in oracle run; raise max_nb")
    rows = th[: (sum(1 for s in range(step0 + 1, step0 + n_steps + 1)
                     if thermo_period and s % thermo_period == 0))]
    return dict(pos=pos, vel=vel, image=image, force=force, thermo=rows,
                builds=int(builds), nh_state=nh)
