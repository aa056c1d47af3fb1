"""Writes nve_drift_oracle.txt: the CPU oracle's own NVE energy drift on the
seeded trajectories that tests/test_gpu_parity.py::test_nve_energy_drift runs
on the GPU (calls only oracle/ and the seeded input generators).

Workload: LJ fluid, N = 4000 (fcc 10^3 start), density 0.8442, T = 1.44,
r_cut = 2.5, r_skin = 0.3, dt = 0.005, energy shifted by V(r_cut); 1000
equilibration steps, then 10^4 steps with a thermo row every 10 steps.
Drift = |least-squares slope of E/N against t| x (10^4 dt); also the largest
|E(t)/N - E(0)/N|.

  python tests/golden/make_nve_drift_oracle.py [seeds...]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1412_3387_gb300 import inputs  # noqa: E402

N, RHO, T, RC, SKIN, DT = 4000, 0.8442, 1.44, 2.5, 0.3, 0.005
EQUIL, STEPS, PERIOD = 1000, 10_000, 10


def drift_of(seed):
    st = inputs.lj_fluid(N, RHO, T, seed=seed)
    kw = dict(r_cut=RC, r_skin=SKIN, dt=DT, shift_energy=True)
    eq = oracle.run(st.pos, st.vel, st.image, st.box[0], EQUIL, **kw)
    out = oracle.run(eq["pos"], eq["vel"], eq["image"], st.box[0], STEPS, thermo_period=PERIOD,
                     step0=EQUIL, **kw)
    th = out["thermo"]
    e = (th[:, 0] + th[:, 1]) / N
    t = np.arange(e.size) * PERIOD * DT
    slope = np.polyfit(t, e, 1)[0]
    return abs(slope) * STEPS * DT, float(np.max(np.abs(e - e[0])))


def main():
    seeds = [int(s) for s in sys.argv[1:]] or list(range(14, 22))
    lines = ["# CPU FP64 oracle NVE drift, LJ N=4000 rho=0.8442 T=1.44 rc=2.5 skin=0.3 dt=0.005,",
             "# shifted energy, 1000 equilibration steps then 1e4 steps (thermo every 10).",
             "# Written by tests/golden/make_nve_drift_oracle.py (calls only oracle/).",
             "# seed  drift_per_particle_over_1e4_steps  max_abs_dev_per_particle"]
    for s in seeds:
        d, m = drift_of(s)
        lines.append(f"{s} {d:.6e} {m:.6e}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "nve_drift_oracle.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
