"""Host logic of bench.py (no GPU): the per-unit byte counts behind the roofline, the
walk the library runs for a grid, the grid's resident bytes, and the source hash that
keys the ncu figures."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1201_3588_gb300 import workloads as w  # noqa: E402


def _counters(**kw):
    c = dict(emitted=0, escaped=0, capped=0, absorptions=0, scatters=0, crossings=0,
             errors=0, clamped=0, levels=0, peel_events=0, peel_crossings=0)
    c.update(kw)
    return c


def test_algorithmic_bytes_follow_the_per_unit_counts():
    # base id + L child ids + S densities per crossing, one 8-byte count RMW per absorption
    c = _counters(crossings=1000, absorptions=10)
    assert bench.crossing_bytes(c, 4, 3) == 1000 * 32 + 10 * 16
    assert bench.crossing_bytes(c, 2, 2) == 1000 * 20 + 10 * 16


def test_walk_bytes_of_each_walk():
    c = _counters(crossings=1000, absorptions=10, scatters=5, levels=70)
    # path walk: one row of S words per crossing and per level descended, the leaf id
    # and densities at each interaction, the count RMW
    assert bench.walk_bytes(c, 4, path=True) == 16 * 1070 + 20 * 15 + 16 * 10
    # linked walk: link + densities per cell entered, a child id per level read
    assert bench.walk_bytes(c, 2, path=False) == 1015 * 12 + 4 * 70 + 16 * 10
    c["peel_crossings"], c["peel_events"] = 100, 3
    assert bench.walk_bytes(c, 2) == 1015 * 12 + 4 * 70 + 16 * 10 + 100 * 12 + 16 * 3


@pytest.mark.parametrize("walk,S,N,L,expect", [
    (0, 4, 10 ** 6, 2, True),          # automatic: four species take the path walk
    (0, 2, 10 ** 6, 2, False),         # two species on a small grid keep the links
    (0, 2, 2 * 10 ** 8, 3, True),      # link records over 4 GB
    (0, 4, 10 ** 6, 5, False),         # deeper than the path walk serves
    (1, 4, 10 ** 6, 2, False),
    (2, 2, 10 ** 6, 2, True),
    (2, 2, 10 ** 6, 5, False),
])
def test_path_walk_rule(walk, S, N, L, expect):
    slots = 64 ** 3 + 8 * 10 ** 5
    assert bench.path_walk_runs(walk, N, S, L, slots) is expect
    assert bench.path_walk_runs(walk, N, S, L, slots, images=True) is False
    assert bench.path_walk_runs(walk, N, S, L, 2 ** 31) is False


def test_grid_bytes_count_the_walks_own_array():
    m = w.disk_model(n_base=16, max_level=2, n_bins=16)
    t = m.tree
    N, S = t.n_leaves, m.n_species
    slots = t.n_base ** 3 + 8 * t.n_blocks
    common = 4 * N * S + N + 4 * slots + 8 * N * S
    assert bench.grid_bytes(m, True) == common + 4 * S * slots
    assert bench.grid_bytes(m, False) == common + 32 * N


def test_source_hash_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    a = tmp_path / "a.cu"
    a.write_text("int f() {  // one\n  return 1;\n}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.source_code_hash(["a.cu"])
    a.write_text("/* header */\nint f() {\n\n  return 1;   \n}\n")
    assert bench.source_code_hash(["a.cu"]) == h
    a.write_text("int f() {\n  return 2;\n}\n")
    assert bench.source_code_hash(["a.cu"]) != h


def test_autotuner_tries_each_distinct_launch_once():
    from paper_1201_3588_gb300 import autotune, rt
    c = list(autotune.single_grid_candidates())
    keys = [tuple(sorted(o.items())) for o in c]
    assert len(keys) == len(set(keys))
    assert all(set(o) == set(autotune.CANDIDATES) for o in c)
    # both walks, every interaction batch and refill period
    for k, vals in autotune.CANDIDATES.items():
        assert {o[k] for o in c} == set(vals)
    # the path walk has no five-block build for 256 threads: that cap is its occupancy
    assert not any(o["walk"] == rt.WALK_PATH and o["blocks_per_sm"] == 5 and o["threads"] == 256
                   for o in c)
    assert any(o["walk"] == rt.WALK_LINKED and o["blocks_per_sm"] == 5 for o in c)
