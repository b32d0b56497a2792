"""Shared helpers of the test-suite: small models and statistical comparisons."""
import math

import numpy as np

from paper_1201_3588_gb300 import workloads as w


def grey_box(n_base, tau_half, albedo=0.0, B=4, star=None, g=0.0):
    sp = [w.grey_species(B, 1.0 - albedo, albedo, g)]
    return w.uniform_box_model(n_base, B, tau_half, sp, half_size_cm=w.AU, star=star)


def binom_ok(k, n, p, z=4.0):
    p = min(max(p, 0.0), 1.0)
    return abs(k - n * p) <= z * math.sqrt(max(n * p * (1 - p), 1e-300)) + 1e-9


def escape_fraction_cube(tau_face):
    """Uncollided escape of isotropic packages from the centre of a uniform cube with
    centre-to-face optical depth tau_face (angular quadrature over one face)."""
    x, wt = np.polynomial.legendre.leggauss(200)
    X, Y = np.meshgrid(x, x)
    W = np.outer(wt, wt)
    r2 = 1 + X ** 2 + Y ** 2
    return 6 / (4 * math.pi) * float((W * np.exp(-tau_face * np.sqrt(r2)) / r2 ** 1.5).sum())


def frozen_field(model, T0=40.0, r0_frac=0.1, slope=-0.4):
    """A smooth per-cell temperature field for frozen-mode replays."""
    lo, hi = w.leaf_bounds_cm(model.tree, model.half_size)
    r = np.linalg.norm((lo + hi) / 2, axis=1) / (r0_frac * model.half_size)
    T = np.clip(T0 * np.maximum(r, 1e-3) ** slope, 5.0, 800.0)
    return np.repeat(T[None, :], model.n_species, axis=0).astype(np.float32)


def trace_agreement(gpu_rec, orc_rec):
    """Fraction of packages whose whole integer history agrees."""
    fields = ("events", "absorptions", "scatters", "crossings", "escaped", "capped",
              "final_bin", "dir_bin", "last_leaf")
    same = np.ones(gpu_rec.shape[0], dtype=bool)
    for j, f in enumerate(fields):
        same &= gpu_rec[:, j] == orc_rec[f].astype(np.int64)
    return same.mean(), same


def runs_z(o_runs, g_runs):
    """z of the mean over oracle runs against the mean over GPU runs, per cell; the
    per-run variance pooled from both sets, floored at the Poisson value and at one
    count. Returns (z, compared) with compared = cells where either mean is > 0."""
    mo, mg = o_runs.mean(axis=0), g_runs.mean(axis=0)
    ko, kg = o_runs.shape[0], g_runs.shape[0]
    ov = o_runs.var(axis=0, ddof=1) if ko > 1 else 0.0   # one oracle run: GPU spread only
    pooled = ((ko - 1) * ov + (kg - 1) * g_runs.var(axis=0, ddof=1)) / (ko + kg - 2)
    var = np.maximum(np.maximum(pooled, 0.5 * (mo + mg)), 1.0)
    return (mo - mg) / np.sqrt(var * (1.0 / ko + 1.0 / kg)), mo + mg > 0


def t_tail(z, dof):
    """P(|t| > z) for Student's t with `dof` degrees of freedom."""
    try:
        from scipy import stats
        return float(2 * stats.t.sf(z, dof))
    except Exception:
        return math.erfc(z / math.sqrt(2))


def assert_runs_agree(o_runs, g_runs, label=""):
    """Per-cell means of independent oracle and GPU runs agree within 4 sigma: no
    more cells beyond 4 sigma than chance allows for the number compared (Poisson
    tail of the expected count at about a one-in-a-million false alarm), none beyond
    6.5 sigma, and the mean square z of cells with > 20 counts near its expectation
    dof / (dof - 2)."""
    o = o_runs.reshape(o_runs.shape[0], -1)
    g = g_runs.reshape(g_runs.shape[0], -1)
    z, ok = runs_z(o, g)
    well = (o.mean(axis=0) + g.mean(axis=0) > 40)[ok]
    z = z[ok]
    dof = o.shape[0] + g.shape[0] - 2
    n_out = int((np.abs(z) > 4.0).sum())
    chance = t_tail(4.0, dof) * z.size
    msq = float((z[well] ** 2).mean()) if well.any() else 1.0
    print(f"{label}: {z.size} cells compared ({int(well.sum())} with > 20 counts), "
          f"max |z| {np.abs(z).max():.2f}, {n_out} beyond 4 sigma (chance {chance:.2f}), "
          f"mean z^2 of the well-measured {msq:.3f}")
    assert n_out <= chance + 5.0 * math.sqrt(chance) + 5.0, (label, n_out, chance)
    assert np.abs(z).max() < 6.5, label
    if well.sum() >= 10:
        assert abs(msq - dof / (dof - 2)) < 0.15 + 3 * math.sqrt(2.0 / well.sum()), (label, msq)
    return z
