"""Iterated PAH coupling: the first transport re-emits the packages PAHs absorb from
each PAH's template spectrum; every further pass re-emits them from the emission
spectrum of the PAHs in that very cell, computed (exactly, or by the surrogate with
exact fallback) from the absorbed spectra of the pass before."""
from __future__ import annotations

import numpy as np

from . import rt


def set_cell_spectra(grid: "rt.Grid", mode: int = rt.PAH_EXACT, surrogate=None,
                     tol: float = 0.05, chunk: int = 1 << 18, out=None, stream=None):
    """Per-cell spectra of every PAH from the grid's current absorbed spectra.
    `out` is a [chunk][B] float32 buffer (host or device) reused per chunk."""
    N, B = grid.N, grid.B
    chunk = min(chunk, N)
    if out is None:
        out = np.zeros((chunk, B), dtype=np.float32)
    for p in range(grid.n_pah):
        for c0 in range(0, N, chunk):
            nc = min(chunk, N - c0)
            grid.pah_emission(first=c0, n=nc, mode=mode, surrogate=surrogate, tol=tol,
                              out=out[:nc], pah=p, stream=stream, count_fallback=False)
            grid.set_pah_spectra(p, out[:nc], first=c0, stream=stream)


def iterate(grid: "rt.Grid", n_packages: int, passes: int = 3, seed: int = 0,
            mode: int = rt.PAH_EXACT, surrogate=None, tol: float = 0.05, stream=None):
    """Runs `passes` transports (Bjorkman-Wood re-emission for grains) with the PAH
    spectra updated in between. Returns the escaped spectra (counts [2][n_dir][B]) of
    every pass and the relative L1 change of the escaped spectrum from pass to pass."""
    grid.set_pah_spectra(0, None, stream=stream)  # start from the templates
    seds, changes = [], []
    for k in range(passes):
        grid.reset(stream)
        grid.transport(n_packages, seed=seed + k, stream=stream)
        sed, _ = grid.sed(stream=stream)
        sed = sed.astype(np.float64)
        if seds:
            prev = seds[-1][0].sum(axis=0)
            cur = sed[0].sum(axis=0)
            changes.append(float(np.abs(cur - prev).sum() / max(prev.sum(), 1.0)))
        seds.append(sed)
        if k + 1 < passes:
            set_cell_spectra(grid, mode=mode, surrogate=surrogate, tol=tol, stream=stream)
    return seds, changes
