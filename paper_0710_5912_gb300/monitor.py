"""Run a grid for many steps and log the paper's observables as JSON lines.

Every ``every`` steps one row is appended: the step n, time t, strain s and
wrap count K (Section V), the compensated mean of phi, the domain sizes L_1
(first moment of S(k)) and L_s (Eq. L_structure), the principal lengths of
Eq. L_matrix, and the wall time and point updates per second of the chunk.
Everything is computed by the library's kernels; this module only schedules
the calls and writes the rows.
"""
from __future__ import annotations

import json
import time


def run_logged(grid, nsteps, every, path=None, append=False):
    """Advance ``grid`` (a Grid or an ensemble Member's owner is not supported)
    by ``nsteps`` in chunks of ``every`` steps and return the list of rows;
    with ``path`` the rows are also written there as JSON lines."""
    if every <= 0 or nsteps < 0:
        raise ValueError("every must be positive and nsteps non-negative")
    rows = []
    fh = open(path, "a" if append else "w") if path else None
    try:
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            t0 = time.perf_counter()
            grid.step(k)
            grid.sync()
            wall = time.perf_counter() - t0
            done += k
            n, t, s, K = grid.get_time()
            moments, _ = grid.structure_factor()
            _, (Lpar, Lperp) = grid.gradient_tensor()
            row = {"n": n, "t": t, "s": s, "K": K, "mean_phi": grid.mass(),
                   "L1": moments[3], "Ls": moments[4], "L_par": Lpar, "L_perp": Lperp,
                   "wall_s": wall, "pts_per_s": grid.nx * grid.ny * k / wall}
            rows.append(row)
            if fh:
                fh.write(json.dumps(row) + "\n")
                fh.flush()
    finally:
        if fh:
            fh.close()
    return rows
