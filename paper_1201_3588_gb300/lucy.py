"""Lucy (1999) iteration: transport with re-emission from the previous iteration's
temperatures (the frozen-temperature mode), temperatures from the path-length
tallies, repeat. The first iteration starts from the counts of a Bjorkman-Wood pass."""
from __future__ import annotations

import numpy as np

from . import rt


def iterate(grid: "rt.Grid", n_packages: int, iterations: int = 4, seed: int = 0,
            T0=None, stream=None):
    """Returns the final temperatures [S][N] and the largest relative change of T
    (over cells with T > 0) at each iteration."""
    if T0 is None:
        grid.reset(stream)
        grid.transport(n_packages, seed=seed, stream=stream)
        T = grid.temperatures(stream=stream)
    else:
        T = np.asarray(T0, dtype=np.float32)
    changes = []
    for it in range(iterations):
        grid.set_frozen_temperatures(T, stream=stream)
        grid.reset(stream)
        grid.transport(n_packages, seed=seed + 1 + it, mode=rt.REEMIT_FROZEN,
                       estimators=rt.EST_PATHLENGTH, stream=stream)
        T_new = grid.temperatures_pathlength(stream=stream)
        pos = (T > 0) & (T_new > 0)
        changes.append(float(np.abs(T_new[pos] / T[pos] - 1).max()) if pos.any() else 0.0)
        T = T_new
    return T, changes
