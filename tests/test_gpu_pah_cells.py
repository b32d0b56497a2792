"""Per-cell PAH re-emission spectra on the GPU (the iterated PAH coupling).

* An exact integer identity at large N: a pure PAH absorber transparent at two bins
  whose x < 0 cells re-emit only at b1 and x > 0 cells only at b2 -- the collided
  escapes at b1 (b2) equal the PAH absorptions in those cells.
* Rows with nothing positive keep the template: bit-identical runs.
* Against the oracle: random per-cell spectra, the same packages replayed.
* The iteration: template pass, then passes with the cells' exact PAH spectra.
"""
import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import pah_iteration, rt, workloads as w
from _helpers import frozen_field, trace_agreement

pytestmark = pytest.mark.gpu


def _pah_box(B=16, n_base=6, tau=0.8):
    nu = w.frequency_edges(B)
    sp = w.pah_species(nu, 50)
    b1, b2 = B - 3, B - 1
    sp.kabs = sp.kabs.copy()
    sp.kabs[[b1, b2]] = 0.0
    sp.ksca = np.zeros(B)
    m = w.uniform_box_model(n_base, B, tau, [sp], half_size_cm=w.AU)
    return m, b1, b2


def _left(m):
    lo, hi = w.leaf_bounds_cm(m.tree, m.half_size)
    return (lo[:, 0] + hi[:, 0]) / 2 < 0


def test_routing_identity_large_n():
    m, b1, b2 = _pah_box()
    B, N = m.n_bins, m.tree.n_leaves
    left = _left(m)
    J = np.zeros((N, B), np.float32)
    J[left, b1] = 3.0
    J[~left, b2] = 1e-20          # any positive row works, however small
    n = 4_000_000
    with rt.Grid(m) as g:
        g.emit_star(n)
        g.set_pah_spectra(0, J[:100])                  # host rows, two pieces
        g.set_pah_spectra(0, J[100:], first=100)
        g.transport(n, seed=1)
        c = g.counters()
        sed, _ = g.sed()
        tal = g.pah_absorbed().astype(np.int64)
    assert c["emitted"] == n == c["escaped"] and c["errors"] == 0
    pah = tal[0].sum(axis=1)
    coll = sed[0].sum(axis=0).astype(np.int64) - sed[1].sum(axis=0).astype(np.int64)
    assert coll[b1] == pah[left].sum() > 0
    assert coll[b2] == pah[~left].sum() > 0
    others = np.ones(B, bool)
    others[[b1, b2]] = False
    assert coll[others].sum() == 0


def test_empty_rows_keep_the_template():
    m, _, _ = _pah_box(B=12, n_base=4)
    B, N = m.n_bins, m.tree.n_leaves
    n = 500_000
    out = []
    for rows in (None, np.zeros((N, B), np.float32), -np.ones((N, B), np.float32)):
        with rt.Grid(m) as g:
            g.emit_star(n)
            if rows is not None:
                g.set_pah_spectra(0, rows)
            g.transport(n, seed=8)
            out.append((g.sed()[0], g.pah_absorbed()))
    for sed, tal in out[1:]:
        assert np.array_equal(sed, out[0][0]) and np.array_equal(tal, out[0][1])


def test_cell_spectra_match_oracle():
    """Grains (frozen temperatures) and a PAH with random per-cell spectra: the
    same packages on both sides."""
    B = 24
    nu = w.frequency_edges(B)
    sp = w.two_species(nu) + [w.pah_species(nu, 60)]
    m = w.sphere_model(n_base=8, n_bins=B, tau_v=2.0, species=sp, fractions=[0.7, 0.25, 0.05])
    N = m.tree.n_leaves
    rng = np.random.default_rng(3)
    J = rng.dirichlet(np.full(B, 0.3), size=N).astype(np.float32)
    J[rng.random(N) < 0.2] = 0.0                       # some cells keep the template
    Tf = frozen_field(m)
    n = 20000
    with rt.Grid(m) as g:
        g.emit_star(n)
        g.set_frozen_temperatures(Tf)
        import torch
        Jd = torch.from_numpy(J).cuda()
        g.set_pah_spectra(0, Jd)                        # device rows
        torch.cuda.synchronize()
        g.transport(n, seed=6, mode=rt.REEMIT_FROZEN)
        sed, _ = g.sed()
        tal = g.pah_absorbed().astype(np.int64)
        ids = np.arange(3000, dtype=np.uint64) * 5 + 1
        rec = g.trace(ids, seed=6)
    # the oracle's template is its own; cells with rows never use it, the others
    # differ from the library's only by FP32 rounding of the same solution
    om = oracle.OracleModel(m, pah_cell_spectra=J[None].astype(np.float64))
    t = oracle.transport(om, n, seed=6, n_total=n, mode=oracle.MODE_FROZEN,
                         T_frozen=Tf.astype(np.float64))
    orc = oracle.trace(om, ids, Tf.astype(np.float64), seed=6, n_total=n)
    frac, _ = trace_agreement(rec, orc)
    print("replay agreement with per-cell PAH spectra", frac)
    assert frac >= 0.97
    assert np.abs(sed.astype(np.int64) - t.sed.astype(np.int64)).sum() <= 0.03 * n
    assert np.abs(tal - t.pahabs.astype(np.int64)).sum() <= 0.03 * t.pahabs.sum() + 5


def test_iteration_moves_then_settles():
    B = 48
    nu = w.frequency_edges(B)
    sp = w.two_species(nu) + [w.pah_species(nu, 30)]
    m = w.sphere_model(n_base=8, n_bins=B, tau_v=3.0, species=sp, fractions=[0.6, 0.2, 0.2])
    n = 16_000_000
    with rt.Grid(m) as g:
        g.emit_star(n)
        seds, changes = pah_iteration.iterate(g, n, passes=4, seed=10)
        c = g.counters()
    print("escaped-spectrum change per pass", changes)
    assert c["errors"] == 0 and c["emitted"] == n
    # the first update (template -> each cell's own spectrum) moves the spectrum more
    # than the later ones, which only carry the Monte Carlo noise of the passes
    assert changes[0] > 2 * max(changes[1:]), changes
