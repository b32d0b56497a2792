"""Pins of the oracle's phase-function sampler, direction rotation, leaf location and
cell walk: closed-form moments and CDF of Henyey-Greenstein, hand-computed crossing
lists, and a brute-force ray/box intersection over every leaf."""
import math

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import workloads as w


def _xi_grid(n):
    return (np.arange(n) + 0.5) / n


@pytest.mark.parametrize("g", [0.0, 0.3, 0.5, 0.9, -0.4])
def test_hg_moments_and_cdf(g):
    xi = _xi_grid(200_000)
    mu = np.array([oracle.hg_mu(g, x) for x in xi])
    # <mu> = g and <mu^2> = (1 + 2 g^2)/3 for Henyey-Greenstein
    assert mu.mean() == pytest.approx(g, abs=2e-6)
    assert (mu ** 2).mean() == pytest.approx((1 + 2 * g * g) / 3, abs=2e-6)
    # cumulative distribution F(mu) = (1-g^2)/(2g) [1/sqrt(1+g^2-2g mu) - 1/(1+g)]
    for m0 in (-0.9, -0.2, 0.4, 0.95):
        if abs(g) < 1e-6:
            F = (m0 + 1) / 2
        else:
            F = (1 - g * g) / (2 * g) * (1 / math.sqrt(1 + g * g - 2 * g * m0) - 1 / (1 + g))
        assert (mu <= m0).mean() == pytest.approx(F, abs=1e-4)


def test_rotation_preserves_angle_and_spreads_azimuth():
    rng = np.random.default_rng(3)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if _ == 0:
            d = np.array([0.0, 0.0, 1.0])
        if _ == 1:
            d = np.array([0.0, 0.0, -1.0])
        mu = rng.uniform(-1, 1)
        outs = np.array([oracle.rotate(d, mu, ph) for ph in 2 * math.pi * _xi_grid(64)])
        assert np.allclose(np.linalg.norm(outs, axis=1), 1.0, atol=1e-14)
        assert np.allclose(outs @ d, mu, atol=1e-12)
        # over a uniform azimuth the mean of the new directions is mu * d
        assert np.allclose(outs.mean(axis=0), mu * d, atol=1e-12)


def _tree_2x2x2_refined():
    # 2^3 base cubes, the cube at the origin corner split once
    return w.build_tree(2, 1, lambda l, lo, hi: (lo == 0).all(axis=1))


def _model(tree, half=1.0):
    sp = [w.grey_species(4, 1.0)]
    return w.explicit_model(tree, np.ones(tree.n_leaves), 4, sp, half_size_cm=half)


def _box(tree, leaf):
    lo, hi = tree.leaf_bounds()
    return lo[leaf], hi[leaf]


def test_hand_computed_crossings_uniform():
    t = w.build_tree(2, 0)
    m = oracle.OracleModel(_model(t))
    # from inside cube (0,0,0) along +x: 0.5 in (0,0,0), then 1.0 in (1,0,0)
    leaves, lens = oracle.ray_cells(m, [0.5, 0.25, 0.25], [1.0, 0.0, 0.0])
    assert [tuple(t.leaf_ijk[l]) for l in leaves] == [(0, 0, 0), (1, 0, 0)]
    assert lens.tolist() == [0.5, 1.0]
    # diagonal through the cube corner (1,1,1): all three faces at once
    d = np.ones(3) / math.sqrt(3)
    leaves, lens = oracle.ray_cells(m, [0.5, 0.5, 0.5], d)
    assert [tuple(t.leaf_ijk[l]) for l in leaves] == [(0, 0, 0), (1, 1, 1)]
    assert lens == pytest.approx([0.5 * math.sqrt(3), math.sqrt(3)])


def test_hand_computed_crossings_refined():
    t = _tree_2x2x2_refined()
    m = oracle.OracleModel(_model(t))
    leaves, lens = oracle.ray_cells(m, [0.1, 0.3, 0.3], [1.0, 0.0, 0.0])
    got = [(int(t.leaf_level[l]),) + tuple(t.leaf_ijk[l]) for l in leaves]
    assert got == [(1, 0, 0, 0), (1, 1, 0, 0), (0, 1, 0, 0)]
    assert lens == pytest.approx([0.4, 0.5, 1.0], abs=1e-15)
    # coming back along -x from the coarse cube into the fine ones
    leaves, lens = oracle.ray_cells(m, [1.7, 0.8, 0.2], [-1.0, 0.0, 0.0])
    got = [(int(t.leaf_level[l]),) + tuple(t.leaf_ijk[l]) for l in leaves]
    assert got == [(0, 1, 0, 0), (1, 1, 1, 0), (1, 0, 1, 0)]
    assert lens == pytest.approx([0.7, 0.5, 0.5], abs=1e-15)


def _brute_segments(tree, p, d):
    """Ray/box slab intersection with every leaf, independent of the walk."""
    lo, hi = tree.leaf_bounds()
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - p) / d
        t1 = (hi - p) / d
    tmin = np.where(d != 0, np.minimum(t0, t1), np.where((p >= lo) & (p <= hi), -np.inf, np.inf))
    tmax = np.where(d != 0, np.maximum(t0, t1), np.where((p >= lo) & (p <= hi), np.inf, -np.inf))
    a = np.maximum(tmin.max(axis=1), 0.0)
    b = tmax.min(axis=1)
    L = b - a
    keep = L > 1e-12
    order = np.argsort(a[keep], kind="stable")
    return np.nonzero(keep)[0][order], L[keep][order]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_walk_matches_brute_force_intersection(seed):
    rng = np.random.default_rng(seed)
    n = 4
    t = w.build_tree(n, 2, lambda l, lo, hi: rng.random(lo.shape[0]) < 0.35)
    m = oracle.OracleModel(_model(t))
    for _ in range(200):
        p = rng.uniform(0, n, size=3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        leaves, lens = oracle.ray_cells(m, p, d)
        bl, bL = _brute_segments(t, p, d)
        assert leaves.tolist() == bl.tolist()
        assert lens == pytest.approx(bL, abs=1e-12)


def test_locate_brute_force_and_face_rule():
    rng = np.random.default_rng(5)
    n = 4
    t = w.build_tree(n, 2, lambda l, lo, hi: rng.random(lo.shape[0]) < 0.4)
    m = oracle.OracleModel(_model(t))
    lo, hi = t.leaf_bounds()
    for _ in range(500):
        p = rng.uniform(0, n, size=3)
        d = rng.normal(size=3)
        rc, out = oracle.locate(m, p, d)
        assert rc == 0
        inside = np.nonzero(((lo <= p) & (p < hi)).all(axis=1))[0]
        assert inside.tolist() == [out[0]]
        assert int(t.leaf_level[out[0]]) == out[1]
        assert tuple(t.leaf_ijk[out[0]]) == tuple(out[2:])
    # a point on a face belongs to the cell ahead of the direction of motion
    for _ in range(200):
        p = rng.uniform(0, n, size=3)
        ax = rng.integers(3)
        p[ax] = rng.integers(1, 4 * n) / 4.0
        p[ax] = min(p[ax], n - 0.25)
        d = rng.normal(size=3)
        rc, out = oracle.locate(m, p, d)
        ahead = p + 1e-9 * d
        inside = np.nonzero(((lo <= ahead) & (ahead < hi)).all(axis=1))[0]
        assert rc == 0 and inside.tolist() == [out[0]]
    # outside the domain
    assert oracle.locate(m, [n + 0.1, 1, 1], [1, 0, 0])[0] == 1
    assert oracle.locate(m, [n, 1, 1], [1, 0, 0])[0] == 1
    assert oracle.locate(m, [0, 1, 1], [-1, 0, 0])[0] == 1
    assert oracle.locate(m, [0, 1, 1], [1, 0, 0])[0] == 0
