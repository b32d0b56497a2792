"""The two pool walks -- face links, and the package's own path of blocks -- find the
same neighbours with the same geometry, so in the frozen mode (histories independent
of arrival order) they give identical counts, spectra, PAH tallies and counters, for
two species, four species with PAHs, and the generic species count; the automatic
choice keeps the links on grids deeper than the path walk serves."""
import numpy as np
import pytest

from paper_1201_3588_gb300 import rt, workloads as w
from _helpers import frozen_field

pytestmark = pytest.mark.gpu


def _models():
    nu = w.frequency_edges(48)
    return {
        "disk, 2 species": w.disk_model(n_base=32, max_level=2, n_bins=48, tau_v_mid=30.0),
        "PAH disk, 4 species": w.disk_pah_model(n_base=32, max_level=2, n_bins=64),
        "box, 3 species": w.uniform_box_model(
            8, 48, 3.0, w.two_species(nu) + [w.grey_species(48, 0.6, 0.4, 0.3)], max_level=3,
            refine=w.sphere_refine_fn(8, 0.4)),
    }


@pytest.mark.parametrize("name", list(_models()))
def test_path_and_linked_walks_agree_exactly(name):
    m = _models()[name]
    N = 300_000
    Tf = frozen_field(m)
    out = {}
    for walk in (rt.WALK_LINKED, rt.WALK_PATH):
        with rt.Grid(m) as g:
            g.emit_star(N)
            g.set_frozen_temperatures(Tf)
            g.transport(N, seed=17, mode=rt.REEMIT_FROZEN, walk=walk)
            c = g.counters()
            out[walk] = (g.counts(), g.sed()[0], g.pah_absorbed() if g.n_pah else None, c)
    (a, sa, pa, ca), (b, sb, pb, cb) = out[rt.WALK_LINKED], out[rt.WALK_PATH]
    assert ca["errors"] == cb["errors"] == 0 and ca["emitted"] == N
    for f in ("emitted", "escaped", "capped", "absorptions", "scatters", "crossings", "clamped"):
        assert ca[f] == cb[f], (name, f, ca[f], cb[f])
    assert np.array_equal(a, b)
    assert np.array_equal(sa, sb)
    if pa is not None:
        assert np.array_equal(pa, pb)


def test_path_walk_in_bw_mode_and_deep_grids():
    m = _models()["PAH disk, 4 species"]
    with rt.Grid(m) as g:
        g.emit_star(10 ** 6)
        g.transport(10 ** 6, seed=3, walk=rt.WALK_PATH)
        c = g.counters()
        assert c["errors"] == 0 and c["emitted"] == c["escaped"] == 10 ** 6
    # five levels: deeper than the path walk serves; it falls back to the links
    deep = w.uniform_box_model(4, 16, 2.0, [w.grey_species(16, 0.8, 0.2)], max_level=5,
                               refine=w.sphere_refine_fn(4, 0.2))
    assert deep.tree.max_level == 5 and (deep.tree.leaf_level == 5).any()
    with rt.Grid(deep) as g:
        g.emit_star(10 ** 5)
        g.transport(10 ** 5, seed=3, walk=rt.WALK_PATH)
        c = g.counters()
        assert c["errors"] == 0 and c["emitted"] == c["escaped"] == 10 ** 5
