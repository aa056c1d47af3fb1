"""Thin Python binding of the libmdgb C ABI (include/md.h).

Argument marshalling only: every step of the MD path runs in the library's
CUDA kernels.  PyTorch provides device memory (particle arrays and the
workspace) and streams.  If the compiled library is missing the import of
this module's functions fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

MD_OK = 0
STATUS = {
    0: "MD_OK", 1: "MD_ERR_INVALID_ARG", 2: "MD_ERR_CUDA", 3: "MD_ERR_WORKSPACE_TOO_SMALL",
    4: "MD_ERR_NLIST_OVERFLOW", 5: "MD_ERR_CELL_GRID", 6: "MD_ERR_NONFINITE",
    7: "MD_ERR_CELL_OVERFLOW", 8: "MD_ERR_STATE", 9: "MD_ERR_TIMEOUT",
}
FP64, MIXED = 0, 1
LJ, DPD, GAUSS, MORSE, YUKAWA, TABLE = 0, 1, 2, 3, 4, 5
# pair kinds by name, and their coefficients per ordered type pair (md.h)
PAIRS = {"lj": LJ, "dpd": DPD, "gauss": GAUSS, "morse": MORSE, "yukawa": YUKAWA, "table": TABLE}
PAIR_NCOEFF = {LJ: 2, DPD: 2, GAUSS: 2, MORSE: 3, YUKAWA: 2, TABLE: 0}
KERNEL_NLIST, KERNEL_PAIR = 0, 1
THERMO_FIELDS = ("ke", "pe", "virial", "pressure", "temperature", "px", "py", "pz")

# Every entry point declared in include/md.h, with its ctypes signature.
_P, _I32, _I64, _D, _SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t


class Particles(C.Structure):
    _fields_ = [("pos", _P), ("vel", _P), ("image", _P), ("tag", _P), ("type", _P)]


class Params(C.Structure):
    _fields_ = [
        ("n_total", _I64), ("n_replicas", _I32), ("replica_offset", _P), ("box", _P),
        ("r_cut", _D), ("r_skin", _D), ("dt", _D), ("mass", _D), ("kT", _D),
        ("seed", C.c_uint64), ("pair", _I32), ("n_types", _I32), ("pair_coeff", _P),
        ("precision", _I32), ("shift_energy", _I32), ("max_nb", _I32),
        ("sort_period", _I32), ("thermo_period", _I32), ("graph_steps", _I32),
        ("max_bonds", _I32), ("max_angles", _I32), ("table_points", _I32),
    ]


SIGNATURES = {
    "md_abi_version": (_I32, []),
    "md_status_string": (C.c_char_p, [C.c_int]),
    "md_workspace_size": (C.c_int, [C.POINTER(Params), C.POINTER(_SZ)]),
    "md_create_system": (C.c_int, [C.POINTER(Params), C.POINTER(Particles), _P, _SZ, _P,
                                   C.POINTER(_P)]),
    "md_destroy_system": (C.c_int, [_P]),
    "md_set_bonds": (C.c_int, [_P, _P, _I64, _D, _D, _P]),
    "md_sort_particles": (C.c_int, [_P, _I32, _P]),
    "md_build_cells": (C.c_int, [_P, _I32, _P]),
    "md_build_nlist": (C.c_int, [_P, _I32, _P]),
    "md_compute_pair": (C.c_int, [_P, _I32, _P]),
    "md_compute_bonds": (C.c_int, [_P, _I32, _P]),
    "md_integrate": (C.c_int, [_P, _I32, _P]),
    "md_step": (C.c_int, [_P, _I32, _P]),
    "md_reduce_thermo": (C.c_int, [_P, _P, _P]),
    "md_run": (C.c_int, [_P, _I64, _P, _P]),
    "md_autotune": (C.c_int, [_P, _I32, _I32, _P]),
    "md_set_tuning": (C.c_int, [_P, _I32, _I32, _I32]),
    "md_get_tuning": (C.c_int, [_P, _I32, C.POINTER(_I32), C.POINTER(_I32)]),
    "md_set_step": (C.c_int, [_P, _I64, _P]),
    "md_get_step": (C.c_int, [_P, C.POINTER(_I64)]),
    "md_poll_error": (C.c_int, [_P, C.POINTER(_I64)]),
    "md_get_forces": (C.c_int, [_P, _P, _P, _P]),
    "md_get_nlist": (C.c_int, [_P, _P, _P, _P]),
    "md_get_cells": (C.c_int, [_P, _P, _P, _P, _P]),
    "md_get_info": (C.c_int, [_P, C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I64)]),
    "md_philox4x32_10": (C.c_int, [_P, _P, _I64, _P]),
    "md_lj_forces_noalloc": (C.c_int, [_P, _I64, _P, _D, _D, _D, _P, _P]),
    "md_set_integrator": (C.c_int, [_P, _I32, _D, _D, C.c_uint64]),
    "md_set_newton": (C.c_int, [_P, _I32]),
    "md_set_bond_style": (C.c_int, [_P, _I32]),
    "md_set_pair_table": (C.c_int, [_P, _P, _D, _P]),
    "md_set_angles": (C.c_int, [_P, _P, _I64, _D, _D, _P]),
    "md_get_thermostat": (C.c_int, [_P, _P]),
}
INTEGRATORS = {"nve": 0, "langevin": 1, "nose-hoover": 2}

_lib = None


def load(path: str | None = None):
    """Loads libmdgb.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libmdgb.so not built ({p}); run __graft_entry__.build()")
        lib = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class MDError(RuntimeError):
    def __init__(self, code, where, detail=None):
        self.code = code
        self.detail = detail
        msg = f"{where}: {STATUS.get(code, code)}"
        if detail is not None:
            msg += f" (detail {detail})"
        super().__init__(msg)


def check(code, where, detail=None):
    if code != MD_OK:
        raise MDError(code, where, detail)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class MDSystem:
    """A GPU-resident MD system (one or more replicas) over torch device
    tensors.  State arrays follow include/md.h: pos/vel float64 [N, 4],
    image int32 [N, 4], tag/type int32 [N]."""

    def __init__(self, state, *, r_cut, r_skin, dt, pair="lj", coeff=((1.0, 1.0),),
                 precision="fp64", kT=1.0, seed=0, mass=1.0, shift_energy=False,
                 max_nb=None, sort_period=0, thermo_period=0, graph_steps=0,
                 max_bonds=None, bond_K=0.0, bond_r0=0.0, max_angles=0, table_points=0,
                 n_types=None, device="cuda:0", stream=None):
        import torch
        self.lib = load()
        self.device = torch.device(device)
        self.R = state.n_replicas
        self.n = state.n
        t = lambda a, dt_: torch.as_tensor(np.ascontiguousarray(a), dtype=dt_).to(self.device)
        self.pos = t(state.pos, torch.float64)
        self.vel = t(state.vel, torch.float64)
        self.image = t(state.image, torch.int32)
        self.tag = t(state.tag, torch.int32)
        self.type = t(state.type, torch.int32)
        if pair not in PAIRS:
            raise ValueError(f"unknown pair kind {pair!r}")
        nk = PAIR_NCOEFF[PAIRS[pair]]
        if nk == 0:  # tabulated: the table comes with set_pair_table
            n_types = int(n_types or (int(np.max(state.type)) + 1 if state.n else 1))
            coeff = np.zeros((n_types, n_types, 0))
        else:
            coeff = np.ascontiguousarray(coeff, np.float64)
            n_types = int(round(np.sqrt(coeff.size / nk)))
            if n_types * n_types * nk != coeff.size:
                raise ValueError(f"{pair} needs {nk} coefficients per ordered type pair")
        self._off = np.ascontiguousarray(state.offsets, np.int64)
        self._box = np.ascontiguousarray(state.box, np.float64).reshape(-1, 3)
        self._coeff = coeff.reshape(n_types, n_types, nk).copy()
        bonds = getattr(state, "bonds", None)
        if max_bonds is None:
            if bonds is not None and len(bonds):
                deg = np.bincount(np.asarray(bonds).reshape(-1), minlength=self.n)
                max_bonds = int(deg.max())
            else:
                max_bonds = 0
        if max_nb is None:
            max_nb = default_max_nb(state, r_cut + r_skin)
        p = Params()
        p.n_total = self.n
        p.n_replicas = self.R
        p.replica_offset = self._off.ctypes.data
        p.box = self._box.ctypes.data
        p.r_cut, p.r_skin, p.dt, p.mass, p.kT = r_cut, r_skin, dt, mass, kT
        p.seed = int(seed)
        p.pair = PAIRS[pair]
        p.n_types = n_types
        p.pair_coeff = self._coeff.ctypes.data if nk else None
        p.table_points = int(table_points)
        p.precision = FP64 if precision == "fp64" else MIXED
        p.shift_energy = int(bool(shift_energy))
        p.max_nb = int(max_nb)
        p.sort_period = int(sort_period)
        p.thermo_period = int(thermo_period)
        p.graph_steps = int(graph_steps)
        p.max_bonds = int(max_bonds)
        p.max_angles = int(max_angles)
        self.params = p
        self.precision = precision
        size = _SZ()
        check(self.lib.md_workspace_size(C.byref(p), C.byref(size)), "md_workspace_size")
        self.workspace = torch.empty(int(size.value), dtype=torch.uint8, device=self.device)
        parts = Particles(self.pos.data_ptr(), self.vel.data_ptr(), self.image.data_ptr(),
                          self.tag.data_ptr(), self.type.data_ptr())
        self._parts = parts
        h = C.c_void_p()
        check(self.lib.md_create_system(C.byref(p), C.byref(parts), _ptr(self.workspace),
                                        size.value, _stream(stream), C.byref(h)),
              "md_create_system")
        self.handle = h
        self.max_nb = self.info()["max_nb"]
        if bonds is not None and len(bonds):
            b = np.ascontiguousarray(bonds, np.int32)
            self._bonds = b
            self.set_bonds(b, bond_K, bond_r0, stream)

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            self.lib.md_destroy_system(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI calls ---------------------------------------------------------
    def set_bonds(self, bond_tags, K, r0, stream=None):
        b = np.ascontiguousarray(bond_tags, np.int32).reshape(-1, 2)
        self._bonds = b
        check(self.lib.md_set_bonds(self.handle, b.ctypes.data_as(C.c_void_p), b.shape[0],
                                    float(K), float(r0), _stream(stream)), "md_set_bonds")

    def build_cells(self, force=True, stream=None):
        check(self.lib.md_build_cells(self.handle, int(force), _stream(stream)), "md_build_cells")

    def build_nlist(self, force=True, stream=None):
        check(self.lib.md_build_nlist(self.handle, int(force), _stream(stream)), "md_build_nlist")

    def sort(self, force=True, stream=None):
        check(self.lib.md_sort_particles(self.handle, int(force), _stream(stream)),
              "md_sort_particles")

    def compute_pair(self, want_virial=False, stream=None):
        check(self.lib.md_compute_pair(self.handle, int(want_virial), _stream(stream)),
              "md_compute_pair")

    def compute_bonds(self, want_virial=False, stream=None):
        check(self.lib.md_compute_bonds(self.handle, int(want_virial), _stream(stream)),
              "md_compute_bonds")

    def compute_forces(self, want_virial=False, stream=None):
        self.compute_pair(want_virial, stream)
        self.compute_bonds(want_virial, stream)

    def integrate(self, half, stream=None):
        check(self.lib.md_integrate(self.handle, int(half), _stream(stream)), "md_integrate")

    def step(self, n=1, want_virial=False, stream=None):
        for _ in range(n):
            check(self.lib.md_step(self.handle, int(want_virial), _stream(stream)), "md_step")

    def run(self, n_steps, thermo_out=None, stream=None):
        check(self.lib.md_run(self.handle, int(n_steps), _ptr(thermo_out), _stream(stream)),
              "md_run")

    def run_with_thermo(self, n_steps, stream=None):
        import torch
        period = self.params.thermo_period
        t0 = self.get_step() if period else 0
        rows = ((t0 + n_steps) // period - t0 // period) if period else 0
        out = torch.zeros((max(rows, 1), self.R, 8), dtype=torch.float64, device=self.device)
        self.run(n_steps, out if rows else None, stream)
        return out[:rows]

    def thermo(self, stream=None):
        import torch
        out = torch.zeros((self.R, 8), dtype=torch.float64, device=self.device)
        check(self.lib.md_reduce_thermo(self.handle, _ptr(out), _stream(stream)),
              "md_reduce_thermo")
        return out

    def set_angles(self, angle_tags, K, theta0, stream=None):
        """Harmonic angles over tag triplets (a, b, c), b the vertex; see
        md_set_angles."""
        t = np.ascontiguousarray(angle_tags, np.int32).reshape(-1, 3)
        self._angles = t
        check(self.lib.md_set_angles(self.handle, t.ctypes.data_as(C.c_void_p), t.shape[0],
                                     float(K), float(theta0), _stream(stream)), "md_set_angles")

    def set_pair_table(self, table, r_min, stream=None):
        """Tabulated pair (pair="table"): table [n_types][n_types][points][2]
        samples (V, F) from r_min to r_cut; see md_set_pair_table."""
        t = np.ascontiguousarray(table, np.float64)
        self._table = t
        check(self.lib.md_set_pair_table(self.handle, t.ctypes.data_as(C.c_void_p), float(r_min),
                                         _stream(stream)), "md_set_pair_table")

    def set_bond_style(self, style="harmonic"):
        """"harmonic" or "fene" (the r0 of set_bonds is then R0); see
        md_set_bond_style."""
        check(self.lib.md_set_bond_style(self.handle, {"harmonic": 0, "fene": 1}[style]),
              "md_set_bond_style")

    def set_newton(self, enable=True):
        """Half neighbour list with Newton's third law (FP64 systems); see
        md_set_newton."""
        check(self.lib.md_set_newton(self.handle, int(bool(enable))), "md_set_newton")

    def set_integrator(self, kind="nve", kT=1.0, param=1.0, seed=0):
        """kind: "nve", "langevin" (param = friction gamma) or "nose-hoover"
        (param = thermostat period tau); see md_set_integrator."""
        check(self.lib.md_set_integrator(self.handle, INTEGRATORS[kind], float(kT), float(param),
                                         int(seed)), "md_set_integrator")

    def thermostat(self):
        """Nose-Hoover (xi, eta) per replica, float64 numpy [R, 2]."""
        out = np.zeros((self.R, 2))
        check(self.lib.md_get_thermostat(self.handle, out.ctypes.data_as(C.c_void_p)),
              "md_get_thermostat")
        return out

    def autotune(self, n_samples=5, block_stride=1, stream=None):
        check(self.lib.md_autotune(self.handle, int(n_samples), int(block_stride),
                                   _stream(stream)), "md_autotune")
        return self.tuning()

    def set_tuning(self, kernel, block, w):
        check(self.lib.md_set_tuning(self.handle, int(kernel), int(block), int(w)),
              "md_set_tuning")

    def tuning(self):
        out = {}
        for k, name in ((KERNEL_NLIST, "nlist"), (KERNEL_PAIR, "pair")):
            b, w = _I32(), _I32()
            check(self.lib.md_get_tuning(self.handle, k, C.byref(b), C.byref(w)), "md_get_tuning")
            out[name] = (b.value, w.value)
        return out

    def set_step(self, step, stream=None):
        check(self.lib.md_set_step(self.handle, int(step), _stream(stream)), "md_set_step")

    def get_step(self):
        v = _I64()
        check(self.lib.md_get_step(self.handle, C.byref(v)), "md_get_step")
        return v.value

    def poll_error(self):
        d = _I64()
        code = self.lib.md_poll_error(self.handle, C.byref(d))
        return code, d.value

    def check_error(self):
        code, d = self.poll_error()
        check(code, "device error", d)

    def forces(self, virial=False, stream=None):
        import torch
        f = torch.empty((self.n, 4), dtype=torch.float64, device=self.device)
        v = torch.empty((self.n, 6), dtype=torch.float64, device=self.device) if virial else None
        check(self.lib.md_get_forces(self.handle, _ptr(f), _ptr(v), _stream(stream)),
              "md_get_forces")
        return (f, v) if virial else f

    def nlist(self, stream=None):
        import torch
        counts = torch.empty(self.n, dtype=torch.int32, device=self.device)
        rows = torch.empty((self.n, self.max_nb), dtype=torch.int32, device=self.device)
        check(self.lib.md_get_nlist(self.handle, _ptr(counts), _ptr(rows), _stream(stream)),
              "md_get_nlist")
        return counts, rows

    def cells(self, stream=None):
        import torch
        nc = self.info()["n_cells"]
        start = torch.empty(nc, dtype=torch.int32, device=self.device)
        count = torch.empty(nc, dtype=torch.int32, device=self.device)
        idx = torch.empty(self.n, dtype=torch.int32, device=self.device)
        check(self.lib.md_get_cells(self.handle, _ptr(start), _ptr(count), _ptr(idx),
                                    _stream(stream)), "md_get_cells")
        return start, count, idx

    def info(self):
        nc, mb, nb = _I64(), _I32(), _I64()
        check(self.lib.md_get_info(self.handle, C.byref(nc), C.byref(mb), C.byref(nb)),
              "md_get_info")
        return dict(n_cells=nc.value, max_nb=mb.value, n_builds=nb.value)

    def prepare(self, stream=None):
        """Bins, builds the list (forced) and computes the initial forces."""
        self.build_cells(True, stream)
        self.build_nlist(True, stream)
        self.compute_forces(False, stream)

    def state_numpy(self):
        import torch
        torch.cuda.synchronize(self.device)
        return dict(pos=self.pos.cpu().numpy(), vel=self.vel.cpu().numpy(),
                    image=self.image.cpu().numpy(), tag=self.tag.cpu().numpy(),
                    type=self.type.cpu().numpy())


def philox4x32_10(inp, stream=None):
    """Device Philox-4x32-10 on rows (ctr0..3, key0..1); returns uint32 [n, 4]."""
    import torch
    lib = load()
    a = np.ascontiguousarray(inp, np.uint32).reshape(-1, 6)
    dev_in = torch.from_numpy(a.view(np.int32)).to("cuda")
    dev_out = torch.empty((a.shape[0], 4), dtype=torch.int32, device="cuda")
    check(lib.md_philox4x32_10(_ptr(dev_in), _ptr(dev_out), a.shape[0], _stream(stream)),
          "md_philox4x32_10")
    return dev_out.cpu().numpy().view(np.uint32)


def lj_forces_noalloc(pos, box, r_cut, epsilon=1.0, sigma=1.0, stream=None):
    """FP64 LJ forces of one system through md_lj_forces_noalloc, the entry
    point for callers that cannot allocate device memory (it uses a fixed
    4 MiB scratch array inside the library).  pos: contiguous float64 CUDA
    tensor [n, 4]; returns a float64 CUDA tensor [n, 4] (F, per-particle
    energy) on the same device.  The C entry point sees only a raw pointer,
    so the tensor's dtype, shape, layout and device are checked here, before
    anything is launched (ValueError)."""
    import torch
    if not isinstance(pos, torch.Tensor):
        raise ValueError("pos must be a torch tensor")
    if pos.dtype != torch.float64:
        raise ValueError(f"pos must be float64, not {pos.dtype}")
    if pos.dim() != 2 or pos.shape[1] != 4:
        raise ValueError(f"pos must have shape [n, 4], not {tuple(pos.shape)}")
    if not pos.is_contiguous():
        raise ValueError("pos must be contiguous")
    if not pos.is_cuda:
        raise ValueError("pos must be a CUDA tensor")
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64).reshape(-1), (3,)))
    lib = load()
    n = int(pos.shape[0])
    with torch.cuda.device(pos.device):
        st = stream if stream is not None else torch.cuda.current_stream(pos.device)
        out = torch.empty((n, 4), dtype=torch.float64, device=pos.device)
        check(lib.md_lj_forces_noalloc(_ptr(pos), n, b.ctypes.data_as(C.c_void_p), float(r_cut),
                                       float(epsilon), float(sigma), _ptr(out),
                                       C.c_void_p(st.cuda_stream)),
              "md_lj_forces_noalloc")
    return out


def default_max_nb(state, r_list: float) -> int:
    """Row capacity from the densest replica: 1.4x the mean neighbour count
    of a uniform fluid plus 32, rounded to a multiple of 32."""
    vol = np.prod(state.box, axis=1)
    counts = np.diff(state.offsets)
    rho = float(np.max(counts / vol)) if len(vol) else 1.0
    mean = 4.0 / 3.0 * np.pi * r_list ** 3 * rho
    return int(np.ceil((1.4 * mean + 32) / 32.0) * 32)
