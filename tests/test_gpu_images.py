"""Peel-off images on the GPU (through the C ABI) against the FP64 oracle.

* Emission only (packages stopped at their first interaction): the stellar image,
  bin by bin, equals the oracle's to FP32 sight-line rounding.
* Pure scattering (no absorption: histories do not depend on arrival order) and the
  frozen-temperature mode: GPU and oracle follow the same packages, so their images
  agree pixel by pixel up to the few histories that FP32 rounding (and the tabulated
  re-emission spectra) make diverge.
* Large N on the GPU alone: the peel-off flux of an observer band against the count
  of escaping packages in that band (two estimators of the same mean intensity).
* The profile entry point against the images it reads, and argument errors.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import rt, workloads as w
from _helpers import frozen_field, grey_box

pytestmark = pytest.mark.gpu


def _inclined(deg):
    a = math.radians(deg)
    return np.array([0.0, math.sin(a), math.cos(a)])


def _gpu_images(model, N, peel, seed, mode=rt.REEMIT_BW, T_frozen=None, max_events=0,
                tau_max=1e30):
    with rt.Grid(model) as g:
        g.emit_star(N)
        if T_frozen is not None:
            g.set_frozen_temperatures(T_frozen)
        g.set_images(peel.obs_dir, peel.plane_of_bin, peel.nx, peel.ny, peel.half_width,
                     tau_max=tau_max)
        g.transport(N, seed=seed, mode=mode, max_events=max_events)
        img = g.images()
        c = g.counters()
    return img, c


def _planes(B, bins):
    pob = np.full(B, -1, np.int32)
    for p, b in enumerate(bins):
        pob[b] = p
    return pob


def test_direct_stellar_image_matches_oracle():
    """A pure absorber frozen at 5 K re-emits only far-infrared photons, so image
    planes at optical and near-infrared bins hold the attenuated star alone."""
    B = 16
    nu = w.frequency_edges(B)
    sp = [w.powerlaw_species("absorber", nu, 1.0e4, 0.0, 1.5)]
    m = w.sphere_model(n_base=8, n_bins=B, tau_v=2.0, species=sp)
    lam = w.bin_centre_wavelength(nu) / w.MICRON
    bins = [b for b in range(B) if lam[b] < 3.0]
    Tf = np.full((1, m.tree.n_leaves), 5.0, np.float32)
    N = 50000
    peel = oracle.Peel(_inclined(35.0), _planes(B, bins), 9, 9, 1.1 * m.half_size)
    img, c = _gpu_images(m, N, peel, seed=4, mode=rt.REEMIT_FROZEN, T_frozen=Tf)
    t = oracle.transport(m, N, seed=4, n_total=N, mode=oracle.MODE_FROZEN,
                         T_frozen=Tf.astype(np.float64), peel=peel)
    assert c["peel_events"] == 0 and c["absorptions"] > 0
    np.testing.assert_allclose(img, t.image, rtol=2e-5, atol=0)
    # only the star's pixel is lit, in every plane
    assert (np.count_nonzero(img, axis=(1, 2)) == 1).all()


@pytest.mark.parametrize("g_hg", [0.0, 0.7])
def test_scattering_images_match_oracle(g_hg):
    """Nearly pure scattering (albedo 0.999, frozen re-emission for the rare
    absorption): histories replay, images agree pixel by pixel."""
    B = 4
    m = grey_box(8, 1.5, albedo=0.999, B=B, g=g_hg)
    Tf = np.full((1, m.tree.n_leaves), 300.0, np.float32)
    N = 40000
    peel = oracle.Peel(_inclined(60.0), np.array([0, -1, 1, 0], np.int32), 17, 13,
                       1.2 * m.half_size)
    img, c = _gpu_images(m, N, peel, seed=9, mode=rt.REEMIT_FROZEN, T_frozen=Tf)
    t = oracle.transport(m, N, seed=9, n_total=N, mode=oracle.MODE_FROZEN,
                         T_frozen=Tf.astype(np.float64), peel=peel)
    assert c["errors"] == 0 and c["emitted"] == N
    assert 0 < c["peel_events"] <= c["scatters"]
    for p in range(2):
        tot_g, tot_o = img[p].sum(), t.image[p].sum()
        assert tot_g == pytest.approx(tot_o, rel=2e-3), (p, tot_g, tot_o)
        l1 = np.abs(img[p] - t.image[p]).sum() / tot_o
        assert l1 < 5e-3, (p, l1)


def test_frozen_reemission_images_match_oracle():
    m = w.sphere_model(n_base=8, n_bins=32, tau_v=3.0)
    Tf = frozen_field(m, T0=120.0)
    N = 20000
    lam = w.bin_centre_wavelength(m.nu_edges) / w.MICRON
    bins = [int(np.argmin(np.abs(lam - x))) for x in (0.55, 10.0, 11.3, 60.0)]
    peel = oracle.Peel(_inclined(50.0), _planes(32, sorted(set(bins))), 21, 21,
                       1.05 * m.half_size)
    img, c = _gpu_images(m, N, peel, seed=21, mode=rt.REEMIT_FROZEN, T_frozen=Tf)
    t = oracle.transport(m, N, seed=21, n_total=N, mode=oracle.MODE_FROZEN,
                         T_frozen=Tf.astype(np.float64), peel=peel)
    assert c["errors"] == 0
    for p in range(img.shape[0]):
        tot_o = t.image[p].sum()
        assert tot_o > 0
        rel = abs(img[p].sum() / tot_o - 1)
        l1 = np.abs(img[p] - t.image[p]).sum() / tot_o
        print(f"plane {p}: total rel diff {rel:.2e}, pixel L1 {l1:.2e}")
        assert rel < 0.03 and l1 < 0.06, (p, rel, l1)


def test_peel_flux_matches_escape_counts_large_n():
    """Observer directions stratified over the whole sphere around a cube with a
    central star (albedo 0.8, g 0.6, BW re-emission): the mean peel-off flux over all
    bins equals eps (escaped packages) / (4 pi)."""
    B, n_dir = 8, 1
    m = w.uniform_box_model(8, B, 1.0, [w.grey_species(B, 0.2, 0.8, 0.6)],
                            half_size_cm=w.AU, n_sed_dirs=n_dir)
    R, N = 32, 2_000_000
    band = 0
    mu_lo, mu_hi = -1.0, 1.0
    omega = 2 * math.pi * (mu_hi - mu_lo)
    rng = np.random.default_rng(5)
    diffs, peels = [], []
    with rt.Grid(m) as g:
        g.emit_star(N)
        for r in range(R):
            mu = mu_lo + (mu_hi - mu_lo) * (r + rng.uniform()) / R
            phi = rng.uniform(0, 2 * math.pi)
            s = math.sqrt(1 - mu * mu)
            o = (s * math.cos(phi), s * math.sin(phi), mu)
            g.set_images(o, np.zeros(B, np.int32), 1, 1, 2.0 * w.AU, tau_max=1e30)
            g.reset()
            g.transport(N, seed=100 + r)
            sed, eps = g.sed()
            F_count = eps * float(sed[0, band].sum()) / omega
            F_peel = float(g.images().sum())
            diffs.append(F_peel - F_count)
            peels.append(F_peel)
    diffs, peels = np.array(diffs), np.array(peels)
    se = math.sqrt(((diffs[0::2] - diffs[1::2]) ** 2).sum()) / R
    print("peel", peels.mean(), "diff", diffs.mean(), "se", se)
    assert abs(diffs.mean()) < 4 * se
    assert se < 0.01 * peels.mean()


def test_profile_and_dual_band():
    m = w.sphere_model(n_base=8, n_bins=16, tau_v=1.0)
    N = 100000
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.set_images(_inclined(60.0), _planes(16, [3, 4]), 12, 10, 1.0 * m.half_size)
        g.transport(N, seed=2)
        img = g.images()
        for a, b, h in [(0, 1, 1), (1, 0, 3), (1, -1, 20), (0, -1, 2)]:
            prof = g.image_profile(a, b, h)
            rows = [py for py in range(10) if abs(py + 0.5 - 5.0) <= h]
            ref = img[a][rows].mean(axis=0) - (img[b][rows].mean(axis=0) if b >= 0 else 0)
            np.testing.assert_allclose(prof, ref, rtol=1e-12, atol=1e-300)
        # h = 0 with an even row count selects no row: the profile is zero
        assert not g.image_profile(0, -1, 0).any()
        # reset clears the images
        g.reset()
        assert not g.images().any()


def test_image_arguments_and_states():
    m = grey_box(4, 0.5, albedo=0.5)
    with rt.Grid(m) as g:
        g.emit_star(1000)
        with pytest.raises(rt.RTError) as e:
            g.images()
        assert e.value.code == 5                               # no images set
        for bad in [dict(nx=0), dict(ny=20000), dict(half_width_cm=0.0),
                    dict(tau_max=-1.0), dict(obs_dir=(0, 0, 0))]:
            kw = dict(obs_dir=(0, 0, 1), plane_of_bin=np.zeros(4, np.int32), nx=4, ny=4,
                      half_width_cm=w.AU)
            kw.update(bad)
            with pytest.raises(rt.RTError) as e:
                g.set_images(**kw)
            assert e.value.code == 1, bad
        with pytest.raises(rt.RTError) as e:
            g.set_images((0, 0, 1), np.full(4, -1, np.int32), 4, 4, w.AU)
        assert e.value.code == 1                               # no plane at all
        with pytest.raises(rt.RTError) as e:
            g.set_images((0, 0, 1), np.array([0, 7, 0, 0], np.int32), 4, 4, w.AU)
        assert e.value.code == 1                               # plane beyond the bins
        with pytest.raises(rt.RTError) as e:
            g.set_images((0, 0, 1), np.array([0, 1, 0, 0], np.int32), 16384, 16384, w.AU)
        assert e.value.code == 8                               # 2^29 pixels in all
        with pytest.raises(rt.RTError) as e:
            g.set_images((0, 0, 1), np.zeros(4, np.int32), 4, 4, w.AU,
                         event_capacity=2 ** 31 + 1)
        assert e.value.code == 8                               # event buffer too large
        g.set_images((0, 0, 1), np.zeros(4, np.int32), 4, 4, w.AU)
        with pytest.raises(rt.RTError) as e:
            g.transport(100, kernel=rt.KERNEL_PLAIN_F32)
        assert e.value.code == 5                               # images need the pool
        with pytest.raises(rt.RTError) as e:
            rt.Batch([g], [100])
        assert e.value.code == 5
        with pytest.raises(rt.RTError) as e:
            g.image_profile(1)
        assert e.value.code == 1
        g.set_images(None, None, 0, 0, 0.0)                    # images off
        g.transport(100, kernel=rt.KERNEL_PLAIN_F32)
        assert g.counters()["emitted"] == 100
