"""Pins of the oracle's peel-off images: line-of-sight optical depths against the
geometry of a uniform box, the direct stellar image against L/(4 pi) e^{-tau}, the
image axes against a displaced source, and the peel-off flux against the count of
escaping packages (two independent estimators of the same intensity)."""
import math

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import workloads as w


def _grey_box(n_base=6, B=4, tau_half=0.7, albedo=0.0, g=0.0, star=None, n_dir=1):
    sp = [w.grey_species(B, 1.0 - albedo, albedo, g)]
    return w.uniform_box_model(n_base, B, tau_half, sp, half_size_cm=w.AU, star=star,
                               n_sed_dirs=n_dir)


def _one_plane(B, obs, nx=1, half=None):
    return oracle.Peel(np.asarray(obs, float), np.zeros(B, np.int32), nx, nx,
                       half if half is not None else 2.0 * w.AU)


@pytest.mark.parametrize("d,frac", [((1, 0, 0), 1.0), ((0, 0, -1), 1.0),
                                    ((1, 1, 1), math.sqrt(3.0)), ((1, 2, 0), math.sqrt(5) / 2)])
def test_optical_depth_uniform_box(d, frac):
    """From the centre of a uniform box the line of sight leaves through a face at
    distance H / max|d_a| (d normalised): tau = rho kappa_ext H |d| / max|d_a|."""
    m = _grey_box(tau_half=1.3)
    dd = np.asarray(d, float)
    tau = oracle.optical_depth(m, (0.0, 0.0, 0.0), dd / np.linalg.norm(dd), 2)
    assert tau == pytest.approx(1.3 * frac, rel=1e-10)


def test_optical_depth_off_centre_and_empty_cells():
    """A sight line through the box's dust-free half picks up only the other half."""
    m = _grey_box(n_base=8, tau_half=1.0)
    lo, hi = w.leaf_bounds_cm(m.tree, m.half_size)
    m.rho[:, (lo[:, 0] + hi[:, 0]) / 2 < 0] = 0.0      # clear x < 0
    x0 = -0.5 * m.half_size
    tau = oracle.optical_depth(m, (x0, 0.1 * m.half_size, 0.0), (1.0, 0.0, 0.0), 0)
    assert tau == pytest.approx(1.0, rel=1e-10)        # only the x > 0 half counts
    tau_back = oracle.optical_depth(m, (x0, 0.0, 0.0), (-1.0, 0.0, 0.0), 0)
    assert tau_back == 0.0


@pytest.mark.parametrize("obs", [(0, 0, 1), (1, 0, 0), (0.3, -0.4, 0.866)])
def test_direct_star_image(obs):
    """Packages stopped at their first interaction contribute only their emission:
    the image holds L_in/(4 pi) e^{-tau} in the star's pixel and nothing else (L_in:
    the luminosity inside the frequency grid)."""
    B, nx = 4, 5
    m = _grey_box(B=B, tau_half=0.8)
    o = np.asarray(obs, float)
    o /= np.linalg.norm(o)
    peel = _one_plane(B, o, nx=nx, half=1.5 * w.AU)
    n = 3000
    t = oracle.transport(m, n, seed=5, n_total=n, max_events=0, peel=peel)
    tau = oracle.optical_depth(m, (0, 0, 0), o, 0)
    # the packages carry the star's luminosity inside the frequency grid
    L_in = oracle.package_energy(m, n) * n
    assert L_in == pytest.approx(m.star.L, rel=1e-6)
    want = L_in / (4 * math.pi) * math.exp(-tau)
    img = t.image[0]
    # the star sits on the pixel grid's centre (odd nx): the centre pixel
    assert img[nx // 2, nx // 2] == pytest.approx(want, rel=1e-9)
    img[nx // 2, nx // 2] = 0.0
    assert not img.any()


def test_image_axes():
    """Axis convention: u along normalise(z x o) (x when o is along z), v = o x u.
    Seen along +z a source at +x lands right of centre; seen along +y it lands left
    (u = -x); seen along +z a source at +y lands above centre."""
    B, nx, H = 2, 8, w.AU
    for pos, obs, (ix, iy) in [((0.3 * H, 0, 0), (0, 0, 1), (5, 4)),
                               ((0.3 * H, 0, 0), (0, 1, 0), (2, 4)),
                               ((0, 0.3 * H, 0), (0, 0, 1), (4, 5)),
                               ((0, 0, 0.3 * H), (0, 1, 0), (4, 5))]:
        star = w.Star(pos_cm=pos)
        m = _grey_box(n_base=4, B=B, tau_half=0.0 + 1e-9, star=star)
        t = oracle.transport(m, 10, seed=1, n_total=10, max_events=0,
                             peel=_one_plane(B, obs, nx=nx, half=H))
        iy_, ix_ = np.unravel_index(np.argmax(t.image[0]), t.image[0].shape)
        assert (ix_, iy_) == (ix, iy), (pos, obs)


def _band_direction(rng, mu_lo, mu_hi, stratum, n_strata):
    """Uniform over the band, stratified in mu (still unbiased over the strata)."""
    mu = mu_lo + (mu_hi - mu_lo) * (stratum + rng.uniform()) / n_strata
    phi = rng.uniform(0, 2 * math.pi)
    s = math.sqrt(max(0.0, 1 - mu * mu))
    return np.array([s * math.cos(phi), s * math.sin(phi), mu])


@pytest.mark.parametrize("case", ["star_scatter", "beam_forward", "frozen_reemit"])
def test_peel_matches_escape_counts(case):
    """For an observer direction drawn uniformly over a band of polar angle, the
    peel-off flux is an unbiased estimate of the mean intensity over the band, as is
    eps (escaped packages in the band) / (band solid angle). Run by run, from the same
    packages; their difference must average to zero (batch means over the runs).
    The beam case compares only scattered light (the beam itself has no intensity off
    its own direction); the forward-peaked phase function makes the result depend on
    the sign of the scattering angle."""
    B, n_dir = 3, 4
    mode, T_frozen, max_ev = oracle.MODE_BW, None, 10_000_000
    R, n = 200, 1000
    if case == "star_scatter":
        m = _grey_box(n_base=6, B=B, tau_half=1.0, albedo=1.0, g=0.6, n_dir=n_dir)
        band = 2
    elif case == "beam_forward":
        star = w.Star(pos_cm=(0.0, 0.0, -0.9 * w.AU), kind=w.SOURCE_BEAM,
                      beam_dir=(0.0, 0.0, 1.0))
        m = _grey_box(n_base=6, B=B, tau_half=0.5, albedo=1.0, g=0.85, star=star,
                      n_dir=n_dir)
        band = 3                                           # mu in [0.5, 1]
    else:
        sp = [w.powerlaw_species("dust", w.frequency_edges(B), 1.0e4, 0.4, 1.5, g=0.3)]
        m = w.uniform_box_model(6, B, 1.5, sp, half_size_cm=w.AU, n_sed_dirs=n_dir)
        mode = oracle.MODE_FROZEN
        T_frozen = np.full((1, m.tree.n_leaves), 300.0)
        band = 1
        R, n = 100, 200                    # exact re-emission draws are slow
    om = oracle.OracleModel(m)
    mu_lo, mu_hi = -1 + 2 * band / n_dir, -1 + 2 * (band + 1) / n_dir
    omega = 2 * math.pi * (mu_hi - mu_lo)
    rng = np.random.default_rng(11)
    eps = oracle.package_energy(om, n)
    diffs, peels = [], []
    for r in range(R):
        o = _band_direction(rng, mu_lo, mu_hi, r, R)
        peel = oracle.Peel(o, np.zeros(B, np.int32), 1, 1, 2.0 * w.AU)
        t = oracle.transport(om, n, seed=40 + r, n_total=n, mode=mode, T_frozen=T_frozen,
                             max_events=max_ev, peel=peel)
        counted = t.sed[0, band].sum()
        if case == "beam_forward":
            counted -= t.sed[1, band].sum()
        F_count = eps * counted / omega
        peels.append(t.image.sum())
        diffs.append(t.image.sum() - F_count)
    diffs, peels = np.array(diffs), np.array(peels)
    # standard error of a stratified mean, one sample per stratum: collapse
    # neighbouring strata in pairs
    se = math.sqrt(((diffs[0::2] - diffs[1::2]) ** 2).sum()) / R
    assert abs(diffs.mean()) < 4.0 * se, (diffs.mean(), se, peels.mean())
    # and the test has power: a 12 % error in the peel-off flux would show
    assert se < 0.03 * peels.mean(), (se, peels.mean())
