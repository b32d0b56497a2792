"""Pins of the oracle's Lucy path-length tallies: their first-flight expectation in a
thin grey box by quadrature (per cell), and their agreement in expectation with the
absorption counts."""
import math

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import workloads as w
from test_oracle_transport import _cell_integral, _corner_cell_integral


def test_first_flight_tally_matches_quadrature():
    """Stopped at their first interaction, packages from the centre of a thin grey box
    leave a tally whose expectation in each cell is N rho kappa (1/4 pi) int_cell
    e^{-rho kappa r} / r^2 dV: checked with batch means of 16 independent runs."""
    H = w.AU
    n_base, B = 6, 4
    sp = [w.grey_species(B, 1.0)]
    m = w.uniform_box_model(n_base, B, 0.3, sp, half_size_cm=H)
    om = oracle.OracleModel(m)
    N, R = 20_000, 16
    runs = np.array([oracle.transport(om, N, seed=100 + k, max_events=0).pathabs[0]
                     for k in range(R)])
    d0 = 2 * H / n_base
    rho = m.rho[0, 0]
    lo, hi = w.leaf_bounds_cm(m.tree, H)
    E = []
    for c in range(m.tree.n_leaves):
        corner = np.all(np.isclose(np.minimum(np.abs(lo[c]), np.abs(hi[c])), 0.0))
        I = _corner_cell_integral(rho, d0) if corner else _cell_integral(rho, lo[c], hi[c])
        E.append(N * rho * 1.0 * I)
    E = np.array(E)
    z = (runs.mean(axis=0) - E) / (runs.std(axis=0, ddof=1) / math.sqrt(R))
    assert np.abs(z).max() < 4.5, np.abs(z).max()
    assert abs(z.mean()) < 4.0 / math.sqrt(len(z))
    assert abs(runs.sum() / (R * E.sum()) - 1) < 0.01


def test_tally_equals_counts_in_expectation():
    m = w.sphere_model(n_base=8, n_bins=16, tau_v=2.0)
    t = oracle.transport(m, 20_000, seed=3, n_total=20_000)
    a, b = t.pathabs.sum(), float(t.count.sum())
    assert abs(a - b) < 4 * math.sqrt(b), (a, b)
