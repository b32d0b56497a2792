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
