"""Per-particle oracle answers from a local neighbourhood (test helper).

For a sampled particle the oracle's exact neighbour row and force follow from
the particle and every particle of the 27 cells around it (cells of width at
least the list radius), in the same periodic box: that set holds all of its
neighbours and every pair within the cut-off.  This lets tests check single
particles of systems far too large for a whole-system oracle run.
"""
import numpy as np

import oracle


def local_reference(pos, L, samples, r_cut=2.5, r_skin=0.4):
    """For each sampled particle: its oracle row (global indices, ascending)
    and oracle force, from the particle and the members of its 27 cells."""
    r_list = r_cut + r_skin
    nc = oracle.cells_per_dim(L, r_list)
    cc = oracle.cell_coords(pos, L, [nc] * 3).astype(np.int64)
    cid = cc[:, 0] + nc * (cc[:, 1] + nc * cc[:, 2])
    order = np.argsort(cid, kind="stable")
    starts = np.searchsorted(cid[order], np.arange(nc ** 3 + 1))
    rows, forces, absf = [], [], []
    for i in samples:
        cx, cy, cz = cc[i]
        parts = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    c = ((cx + dx) % nc) + nc * (((cy + dy) % nc) + nc * ((cz + dz) % nc))
                    parts.append(order[starts[c]:starts[c + 1]])
        idx = np.unique(np.concatenate(parts))  # small boxes repeat cells
        loc = int(np.searchsorted(idx, i))
        sub = pos[idx]
        cnt, rw = oracle.neighbors(sub, L, r_list, max_nb=256, method="brute")
        rows.append(np.sort(idx[rw[loc, :cnt[loc]]]))
        f, _, af = oracle.lj_forces(sub, L, r_cut)
        forces.append(f[loc])
        absf.append(af[loc])
    return rows, np.array(forces), np.array(absf)
