"""Seeded synthetic inputs for the short-range MD hot path.

This module holds no force, neighbour-list or integration arithmetic: it only
draws initial states (positions, velocities, types, tags, bonds) from seeded
NumPy generators.  Both the CUDA path and the CPU oracle are fed from the
arrays it returns, so neither side depends on the other.

Workload shapes follow the benchmarks the paper describes:
  * LJ fluids started from an fcc lattice and Maxwell-Boltzmann velocities
    (the LAMMPS-Kokkos comparison in Sec. 8.3: fcc start, T = 1.44, rho 0.8442);
  * DPD fluids at number density 3 with uniform random positions (Sec. 9);
  * a diblock-copolymer melt of linear chains (harmonic bonds, Sec. 3 lists
    harmonic bonds among the supported potentials);
  * an ensemble of independent small LJ replicas (the small-N regime of Sec. 5).

Arrays use the layouts of the C ABI: positions and velocities are float64
[N, 4] (x, y, z, w) with w unused; image counters int32 [N, 4].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FCC_BASIS = np.array(
    [[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]]
)


@dataclass
class State:
    """A periodic particle system (one or more independent replicas)."""

    pos: np.ndarray  # float64 [N, 4]
    vel: np.ndarray  # float64 [N, 4]
    image: np.ndarray  # int32 [N, 4]
    tag: np.ndarray  # int32 [N]
    type: np.ndarray  # int32 [N]
    box: np.ndarray  # float64 [R, 3] edge lengths per replica
    offsets: np.ndarray  # int64 [R + 1] replica particle ranges
    bonds: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_replicas(self) -> int:
        return int(self.box.shape[0])

    def copy(self) -> "State":
        return State(
            self.pos.copy(), self.vel.copy(), self.image.copy(), self.tag.copy(),
            self.type.copy(), self.box.copy(), self.offsets.copy(),
            self.bonds.copy(), dict(self.meta),
        )


def _pack4(xyz: np.ndarray) -> np.ndarray:
    out = np.zeros((xyz.shape[0], 4), np.float64)
    out[:, :3] = xyz
    return out


def _wrap(xyz: np.ndarray, L: float) -> np.ndarray:
    xyz = np.mod(xyz, L)
    # np.mod can return L for tiny negative inputs; fold those onto 0.
    xyz[xyz >= L] = 0.0
    return xyz


def fcc_positions(n: int, rho: float, rng: np.random.Generator,
                  jitter: float = 0.0) -> tuple[np.ndarray, float]:
    """n particles on an fcc lattice at number density rho.

    The box edge is L = (n / rho)^(1/3).  The lattice has m^3 cubic cells with
    m = ceil((n / 4)^(1/3)); when 4 m^3 > n the surplus sites are removed at
    random (seeded vacancies), which keeps the density exactly rho.  `jitter`
    adds uniform displacements in [-jitter, jitter) * a per coordinate, where
    a = L / m is the lattice constant.
    """
    m = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
    while 4 * m ** 3 < n:
        m += 1
    L = (n / rho) ** (1.0 / 3.0)
    a = L / m
    cells = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m),
                                 indexing="ij"), -1).reshape(-1, 3)
    sites = (cells[:, None, :] + FCC_BASIS[None, :, :]).reshape(-1, 3)
    sites = (sites + 0.25) * a
    n_sites = sites.shape[0]
    if n_sites > n:
        keep = np.sort(rng.permutation(n_sites)[:n])
        sites = sites[keep]
    if jitter > 0.0:
        sites = sites + rng.uniform(-jitter, jitter, sites.shape) * a
    return _wrap(sites, L), L


def maxwell_boltzmann(n: int, T: float, rng: np.random.Generator,
                      mass: float = 1.0) -> np.ndarray:
    """Gaussian velocities with zero total momentum, rescaled so that the
    kinetic energy equals (3n - 3) T / 2 exactly (k_B = 1)."""
    v = rng.standard_normal((n, 3)) * math.sqrt(T / mass)
    v -= v.mean(axis=0, keepdims=True)
    ke = 0.5 * mass * float(np.sum(v * v))
    target = 0.5 * (3 * n - 3) * T
    if ke > 0.0:
        v *= math.sqrt(target / ke)
    return v


def lj_fluid(n: int, rho: float, T: float, seed: int, jitter: float = 0.0) -> State:
    """LJ fluid: fcc start (optionally jittered) + Maxwell-Boltzmann velocities."""
    rng = np.random.default_rng(seed)
    xyz, L = fcc_positions(n, rho, rng, jitter)
    v = maxwell_boltzmann(n, T, rng)
    return State(
        pos=_pack4(xyz), vel=_pack4(v), image=np.zeros((n, 4), np.int32),
        tag=np.arange(n, dtype=np.int32), type=np.zeros(n, np.int32),
        box=np.array([[L, L, L]]), offsets=np.array([0, n], np.int64),
        meta=dict(kind="lj", rho=rho, T=T, seed=seed, jitter=jitter),
    )


def dpd_fluid(n: int, rho: float, kT: float, seed: int) -> State:
    """DPD fluid: uniform random positions, Maxwell-Boltzmann velocities."""
    rng = np.random.default_rng(seed)
    L = (n / rho) ** (1.0 / 3.0)
    xyz = _wrap(rng.uniform(0.0, L, (n, 3)), L)
    v = maxwell_boltzmann(n, kT, rng)
    return State(
        pos=_pack4(xyz), vel=_pack4(v), image=np.zeros((n, 4), np.int32),
        tag=np.arange(n, dtype=np.int32), type=np.zeros(n, np.int32),
        box=np.array([[L, L, L]]), offsets=np.array([0, n], np.int64),
        meta=dict(kind="dpd", rho=rho, kT=kT, seed=seed),
    )


def diblock_melt(n_chains: int, n_beads: int, rho: float, kT: float, seed: int,
                 bond_length: float = 0.9, frac_a: float = 0.5) -> State:
    """Linear A-B diblock chains as seeded random walks.

    Each chain starts at a uniform random point; every further bead sits at
    bond_length times a uniform random unit vector from the previous one.
    The first round(frac_a * n_beads) beads are type 0 (A), the rest type 1 (B).
    Bonds join consecutive beads of a chain and are given by tag.
    """
    rng = np.random.default_rng(seed)
    n = n_chains * n_beads
    L = (n / rho) ** (1.0 / 3.0)
    start = rng.uniform(0.0, L, (n_chains, 1, 3))
    u = rng.standard_normal((n_chains, n_beads - 1, 3))
    u /= np.linalg.norm(u, axis=-1, keepdims=True)
    steps = np.concatenate([np.zeros((n_chains, 1, 3)), bond_length * u], axis=1)
    xyz = (start + np.cumsum(steps, axis=1)).reshape(-1, 3)
    image = np.zeros((n, 4), np.int32)
    image[:, :3] = np.floor(xyz / L).astype(np.int32)
    xyz = _wrap(xyz, L)
    n_a = int(round(frac_a * n_beads))
    types = np.tile((np.arange(n_beads) >= n_a).astype(np.int32), n_chains)
    base = (np.arange(n_chains) * n_beads)[:, None]
    a = (base + np.arange(n_beads - 1)[None, :]).reshape(-1)
    bonds = np.stack([a, a + 1], axis=1).astype(np.int32)
    v = maxwell_boltzmann(n, kT, rng)
    return State(
        pos=_pack4(xyz), vel=_pack4(v), image=image,
        tag=np.arange(n, dtype=np.int32), type=types,
        box=np.array([[L, L, L]]), offsets=np.array([0, n], np.int64), bonds=bonds,
        meta=dict(kind="diblock", rho=rho, kT=kT, seed=seed, n_chains=n_chains,
                  n_beads=n_beads),
    )


def replica_ensemble(n_replicas: int, seed: int, n_min: int = 2000,
                     n_max: int = 64000, rho_range=(0.70, 0.90),
                     T_range=(0.8, 1.5), jitter: float = 0.0) -> State:
    """Independent LJ replicas of uneven size, concatenated.

    N_r = round(exp(U[ln n_min, ln n_max])), rho_r ~ U[rho_range],
    T_r ~ U[T_range], all drawn from one seeded stream; each replica is an fcc
    start in its own cubic box with Maxwell-Boltzmann velocities at T_r.
    """
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max),
                                       n_replicas))).astype(np.int64)
    rhos = rng.uniform(*rho_range, n_replicas)
    temps = rng.uniform(*T_range, n_replicas)
    pos, vel, box = [], [], []
    for r in range(n_replicas):
        sub = np.random.default_rng([seed, r])
        xyz, L = fcc_positions(int(sizes[r]), float(rhos[r]), sub, jitter)
        pos.append(_pack4(xyz))
        vel.append(_pack4(maxwell_boltzmann(int(sizes[r]), float(temps[r]), sub)))
        box.append([L, L, L])
    n = int(sizes.sum())
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return State(
        pos=np.concatenate(pos), vel=np.concatenate(vel),
        image=np.zeros((n, 4), np.int32), tag=np.arange(n, dtype=np.int32),
        type=np.zeros(n, np.int32), box=np.array(box), offsets=offsets,
        meta=dict(kind="lj-ensemble", seed=seed, rho=rhos.tolist(), T=temps.tolist()),
    )


def select_replica(state: State, r: int) -> State:
    """Copy of replica r of a concatenated ensemble as a standalone system."""
    a, b = int(state.offsets[r]), int(state.offsets[r + 1])
    return State(
        pos=state.pos[a:b].copy(), vel=state.vel[a:b].copy(),
        image=state.image[a:b].copy(), tag=np.arange(b - a, dtype=np.int32),
        type=state.type[a:b].copy(), box=state.box[r:r + 1].copy(),
        offsets=np.array([0, b - a], np.int64), meta=dict(state.meta, replica=r),
    )


# Named workloads.  Sizes and parameters are those of the benchmark
# configurations; `small` variants keep the same densities and temperatures.
WORKLOADS = {
    "lj-4000": dict(kind="lj", n=4000, rho=0.8442, T=1.44, r_cut=2.5, r_skin=0.3,
                    dt=0.005, steps=100),
    "lj-16.7M": dict(kind="lj", n=16_777_216, rho=0.8442, T=1.2, r_cut=2.5,
                     r_skin=0.4, dt=0.005, steps=1000),
    "lj-64k": dict(kind="lj", n=65_536, rho=0.8442, T=1.2, r_cut=2.5, r_skin=0.4,
                   dt=0.005, steps=1000),
    "dpd-8M": dict(kind="dpd", n=8_000_000, rho=3.0, kT=1.0, r_cut=1.0, r_skin=0.3,
                   dt=0.02, A=25.0, gamma=4.5, steps=1000),
    "diblock-4.2M": dict(kind="diblock", n_chains=131_072, n_beads=32, rho=3.0,
                         kT=1.0, r_cut=1.0, r_skin=0.3, dt=0.02, A_same=25.0,
                         A_diff=40.0, gamma=4.5, K=4.0, r0=0.0, steps=2000),
    "lj-ensemble-256": dict(kind="ensemble", n_replicas=256, r_cut=2.5, r_skin=0.3,
                            dt=0.005, steps=100),
}
