"""Pins of the oracle's per-cell PAH re-emission spectra (the iterated PAH coupling):
a PAH absorption in a cell re-emits from that cell's spectrum, the template where a
cell has none.

The set-up makes the result an exact integer identity: a pure PAH absorber that is
transparent at two bins b1, b2; cells with x < 0 re-emit only at b1, cells with
x > 0 only at b2. A re-emitted package then escapes without further interaction, so
the collided escapes at b1 (b2) equal the PAH absorptions in the x < 0 (x > 0) cells.
"""
import numpy as np

import oracle
from paper_1201_3588_gb300 import workloads as w


def _pah_box(B=16, n_base=6, tau=0.8):
    nu = w.frequency_edges(B)
    sp = w.pah_species(nu, 50)
    b1, b2 = B - 3, B - 1
    sp.kabs = sp.kabs.copy()
    sp.kabs[[b1, b2]] = 0.0
    sp.ksca = np.zeros(B)
    m = w.uniform_box_model(n_base, B, tau, [sp], half_size_cm=w.AU)
    return m, b1, b2


def _halves(m):
    lo, hi = w.leaf_bounds_cm(m.tree, m.half_size)
    return (lo[:, 0] + hi[:, 0]) / 2 < 0


def test_cell_spectra_route_reemission_by_cell():
    m, b1, b2 = _pah_box()
    B, N = m.n_bins, m.tree.n_leaves
    left = _halves(m)
    J = np.zeros((1, N, B))
    J[0, left, b1] = 1.0
    J[0, ~left, b2] = 2.5                      # any positive weight: rows are normalised
    template = np.ones((1, B))
    om = oracle.OracleModel(m, pah_template=template, pah_cell_spectra=J)
    n = 20000
    t = oracle.transport(om, n, seed=7, n_total=n)
    assert t.emitted == n == t.escaped and t.errors == 0
    pah = t.pahabs[0].sum(axis=1).astype(np.int64)          # per cell
    collided = t.sed[0].sum(axis=0).astype(np.int64) - t.sed[1].sum(axis=0).astype(np.int64)
    assert collided[b1] == pah[left].sum() > 0
    assert collided[b2] == pah[~left].sum() > 0
    others = np.ones(B, bool)
    others[[b1, b2]] = False
    assert collided[others].sum() == 0
    assert t.absorptions == pah.sum()


def test_empty_rows_fall_back_to_the_template():
    """Rows of zeros re-emit from the template, bit for bit the same run; a partial
    set of rows changes only the packages absorbed in those cells."""
    m, b1, b2 = _pah_box(B=12, n_base=4)
    B, N = m.n_bins, m.tree.n_leaves
    template = np.linspace(1.0, 2.0, B)[None, :]
    n = 5000
    a = oracle.transport(oracle.OracleModel(m, pah_template=template), n, seed=3, n_total=n)
    z = oracle.transport(oracle.OracleModel(m, pah_template=template,
                                            pah_cell_spectra=np.zeros((1, N, B))),
                         n, seed=3, n_total=n)
    for f in ("count", "sed", "pahabs"):
        assert np.array_equal(getattr(a, f), getattr(z, f)), f
    # the template's own rows in every cell: identical histories as well
    same = oracle.transport(oracle.OracleModel(m, pah_template=template,
                                               pah_cell_spectra=np.repeat(
                                                   template[:, None, :], N, axis=1)),
                            n, seed=3, n_total=n)
    assert np.array_equal(a.sed, same.sed) and np.array_equal(a.pahabs, same.pahabs)
