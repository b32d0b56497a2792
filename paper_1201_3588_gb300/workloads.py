"""Seeded synthetic model builders: grids of cubes and subcubes, densities, dust, star.

This module is shared by the CUDA path and by the CPU oracle; it prepares *inputs*
only and contains none of the transport arithmetic (no Planck function, no optical
depth sampling, no temperature inversion).

Every builder returns plain numpy arrays in the layout both sides consume:

* ``base``   int32 ``[n^3]`` indexed ``ix + n*(iy + n*iz)``: ``>= 0`` a leaf id,
  ``< 0`` a child block ``-(block+1)``.
* ``child``  int32 ``[n_blocks*8]``: entry ``8*block + (ox | oy<<1 | oz<<2)`` with
  the same encoding (Sec. 2: cubes are divided into subcubes where a finer grid is
  needed; the factor 2 per axis and level is this library's choice).
* ``leaf_level`` / ``leaf_ijk``: refinement level and integer lower corner of each
  leaf at its own level (grid units of ``2^-level`` base cells).
* ``rho``    float64 ``[S][n_leaves]`` in g/cm^3.

Leaves are numbered in Morton (Z) order of their lower corner at the finest level,
so every 2x2x2 block of siblings is contiguous and spatial neighbours are close in
memory.

Physical constants here are only the unit conversions and the stellar parameters
the workloads are quoted with.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

AU = 1.495978707e13          # cm
RSUN = 6.957e10              # cm
C_LIGHT = 2.99792458e10      # cm/s
SIGMA_SB = 5.670374419e-5    # erg cm^-2 s^-1 K^-4
MICRON = 1e-4                # cm
LAMBDA_V = 0.55 * MICRON     # V band reference wavelength

# Source kinds understood by both sides.
SOURCE_POINT = 0
SOURCE_BEAM = 1


# --------------------------------------------------------------------------- grid

@dataclasses.dataclass
class Tree:
    n_base: int
    max_level: int
    base: np.ndarray        # int32 [n^3]
    child: np.ndarray       # int32 [n_blocks*8]
    leaf_level: np.ndarray  # int32 [N]
    leaf_ijk: np.ndarray    # int64 [N,3] lower corner at the leaf's level

    @property
    def n_leaves(self) -> int:
        return int(self.leaf_level.shape[0])

    @property
    def n_blocks(self) -> int:
        return int(self.child.shape[0] // 8)

    def leaf_bounds(self):
        """Lower/upper corners of every leaf in base-cell units, float64 [N,3]."""
        size = np.ldexp(1.0, -self.leaf_level.astype(np.int64))[:, None]
        lo = self.leaf_ijk.astype(np.float64) * size
        return lo, lo + size


def _morton3(ix: np.ndarray, iy: np.ndarray, iz: np.ndarray, bits: int) -> np.ndarray:
    """Interleave the low ``bits`` bits of three int64 arrays (x lowest)."""
    key = np.zeros(ix.shape, dtype=np.int64)
    for b in range(bits):
        key |= ((ix >> b) & 1) << (3 * b)
        key |= ((iy >> b) & 1) << (3 * b + 1)
        key |= ((iz >> b) & 1) << (3 * b + 2)
    return key


def build_tree(n_base: int, max_level: int,
               refine: Optional[Callable[[int, np.ndarray, np.ndarray], np.ndarray]] = None
               ) -> Tree:
    """Build a cube/subcube tree.

    ``refine(level, lo, hi)`` gets the corners (base-cell units, float64 [M,3]) of the
    M nodes at ``level`` and returns a bool [M]: which of them to split into 2x2x2
    children. Nodes at ``max_level`` are never split.
    """
    if n_base < 1 or max_level < 0:
        raise ValueError("n_base >= 1 and max_level >= 0 required")
    n = n_base
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ijk = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.int64)
    # nodes per level: (ijk at that level, slot) where slot identifies where the id goes:
    # level 0 slot = base index, deeper slot = 8*block + octant
    levels_ijk: List[np.ndarray] = [ijk]
    levels_slot: List[np.ndarray] = [np.arange(n ** 3, dtype=np.int64)]
    levels_split: List[np.ndarray] = []
    for lev in range(max_level + 1):
        cur = levels_ijk[lev]
        if lev < max_level and refine is not None and cur.shape[0] > 0:
            size = math.ldexp(1.0, -lev)
            lo = cur.astype(np.float64) * size
            split = np.asarray(refine(lev, lo, lo + size), dtype=bool)
            if split.shape != (cur.shape[0],):
                raise ValueError("refine() must return one bool per node")
        else:
            split = np.zeros(cur.shape[0], dtype=bool)
        levels_split.append(split)
        if lev < max_level:
            par = cur[split]
            nb = par.shape[0]
            oct_ = np.arange(8, dtype=np.int64)
            off = np.stack([oct_ & 1, (oct_ >> 1) & 1, (oct_ >> 2) & 1], axis=1)
            kids = (2 * par[:, None, :] + off[None, :, :]).reshape(-1, 3)
            levels_ijk.append(kids)
            # block ids are assigned after ordering; store parent position for now
            levels_slot.append(np.repeat(np.arange(nb, dtype=np.int64), 8) * 8
                               + np.tile(oct_, nb))
    # Morton key of every node's lower corner at the finest level, for ordering.
    bits = max(1, int(math.ceil(math.log2(max(2, n)))) + max_level)
    base = np.empty(n ** 3, dtype=np.int32)
    # order blocks by the Morton key of their parent, per level
    n_blocks_before = 0
    block_of_level: List[np.ndarray] = []
    for lev in range(max_level):
        par = levels_ijk[lev][levels_split[lev]]
        shift = max_level - lev
        key = _morton3(par[:, 0] << shift, par[:, 1] << shift, par[:, 2] << shift, bits)
        order = np.argsort(key, kind="stable")
        bid = np.empty(par.shape[0], dtype=np.int64)
        bid[order] = np.arange(par.shape[0], dtype=np.int64) + n_blocks_before
        block_of_level.append(bid)
        n_blocks_before += par.shape[0]
    n_blocks = n_blocks_before
    child = np.full(n_blocks * 8, np.iinfo(np.int32).min, dtype=np.int32)
    # leaves
    leaf_ijk_l, leaf_lev_l, leaf_key_l = [], [], []
    for lev in range(max_level + 1):
        cur = levels_ijk[lev]
        leaf = ~levels_split[lev]
        shift = max_level - lev
        li = cur[leaf]
        leaf_ijk_l.append(li)
        leaf_lev_l.append(np.full(li.shape[0], lev, dtype=np.int32))
        leaf_key_l.append(_morton3(li[:, 0] << shift, li[:, 1] << shift, li[:, 2] << shift,
                                   bits))
    all_ijk = np.concatenate(leaf_ijk_l)
    all_lev = np.concatenate(leaf_lev_l)
    all_key = np.concatenate(leaf_key_l)
    order = np.argsort(all_key, kind="stable")
    leaf_id = np.empty(order.shape[0], dtype=np.int64)
    leaf_id[order] = np.arange(order.shape[0], dtype=np.int64)
    # write ids into base/child
    start = 0
    for lev in range(max_level + 1):
        cur = levels_ijk[lev]
        split = levels_split[lev]
        nl = int((~split).sum())
        ids = leaf_id[start:start + nl]
        start += nl
        slot = levels_slot[lev]
        if lev > 0:
            # remap the parent index (slot//8 is the parent's index among the split
            # nodes of level lev-1) to its ordered block id
            bid = block_of_level[lev - 1][slot // 8]
            slot = bid * 8 + (slot % 8)
        enc = np.empty(cur.shape[0], dtype=np.int64)
        enc[~split] = ids
        if lev < max_level and split.any():
            enc[split] = -(block_of_level[lev] + 1)
        if lev == 0:
            base[slot] = enc.astype(np.int32)
        else:
            child[slot] = enc.astype(np.int32)
    leaf_ijk = all_ijk[order]
    leaf_lev = all_lev[order]
    return Tree(n_base=n, max_level=max_level, base=base, child=child,
                leaf_level=leaf_lev.astype(np.int32), leaf_ijk=leaf_ijk)


# --------------------------------------------------------------------------- bins & dust

def frequency_edges(n_bins: int, lam_min_um: float = 0.1, lam_max_um: float = 1000.0
                    ) -> np.ndarray:
    """``n_bins+1`` bin edges in Hz, ascending, log-spaced in wavelength."""
    lam = np.logspace(math.log10(lam_max_um), math.log10(lam_min_um), n_bins + 1) * MICRON
    return C_LIGHT / lam


def bin_centre_wavelength(nu_edges: np.ndarray) -> np.ndarray:
    """Wavelength (cm) at the logarithmic centre of each frequency bin."""
    return C_LIGHT / np.sqrt(nu_edges[:-1] * nu_edges[1:])


@dataclasses.dataclass
class Species:
    name: str
    kabs: np.ndarray        # cm^2/g per bin
    ksca: np.ndarray        # cm^2/g per bin
    g: np.ndarray           # HG asymmetry per bin
    kappa_v_ext: float      # extinction opacity at 0.55 micron, cm^2/g
    is_pah: int = 0
    n_carbon: int = 0
    n_hydrogen: int = 0
    mol_mass: float = 0.0   # g per molecule (PAH)
    modes: tuple = ()       # ((count, theta_K), ...) vibrational modes (PAH)


def powerlaw_species(name: str, nu_edges: np.ndarray, kappa_v_ext: float,
                     albedo_v: float, beta_abs: float, beta_sca: float = 2.0,
                     g: float = 0.5, albedo_cap: float = 0.95) -> Species:
    """Smooth synthetic grain: kappa_abs ~ lambda^-beta_abs, kappa_sca ~ lambda^-beta_sca,
    normalised at V to ``kappa_v_ext`` and ``albedo_v``; albedo capped at ``albedo_cap``.
    Values are taken at each bin's logarithmic centre."""
    lam = bin_centre_wavelength(nu_edges)
    x = lam / LAMBDA_V
    kabs = kappa_v_ext * (1.0 - albedo_v) * x ** (-beta_abs)
    ksca = kappa_v_ext * albedo_v * x ** (-beta_sca)
    cap = albedo_cap / (1.0 - albedo_cap)
    ksca = np.minimum(ksca, cap * kabs)
    return Species(name, kabs, ksca, np.full(lam.shape, g), float(kappa_v_ext))


def grey_species(n_bins: int, kappa_abs: float, kappa_sca: float = 0.0,
                 g: float = 0.0, name: str = "grey") -> Species:
    return Species(name, np.full(n_bins, float(kappa_abs)), np.full(n_bins, float(kappa_sca)),
                   np.full(n_bins, float(g)), float(kappa_abs + kappa_sca))


AMU = 1.66053906660e-24     # g
H_PLANCK = 6.62607015e-27   # erg s (only for the band-centre conversion below)

# Synthetic PAH material data. The real cross sections and band parameters the
# paper uses are not available; these stand in for them with the same structure:
# a far-UV-rising continuum with a long-wavelength cut-off that moves redwards with
# size, plus 17 Lorentzian infrared bands, per carbon atom.
PAH_N_BANDS = 17
PAH_BAND_LAMBDA_UM = np.geomspace(3.0, 17.0, PAH_N_BANDS)     # band centres
PAH_BAND_FWHM_FRAC = 0.03                                      # FWHM / centre (frequency)
PAH_BAND_PEAK = 4.0e-20                                        # cm^2 per C atom at a peak
PAH_UV_SIGMA = 7.0e-18                                         # cm^2 per C at 0.1 micron


def pah_hydrogens(n_carbon: int) -> int:
    """Hydrogen count of a compact PAH, N_H ~ sqrt(6 N_C)."""
    return int(round(math.sqrt(6.0 * n_carbon)))


def pah_cross_section_per_carbon(nu_edges: np.ndarray, n_carbon: int) -> np.ndarray:
    """Bin-averaged absorption cross section per C atom (cm^2): continuum
    (lambda/0.1um)^-1 / (1 + (lambda/lambda_c)^6) with lambda_c = 0.5 um (N_C/50)^(1/4),
    taken at the bin centre, plus the Lorentzian bands averaged over each bin in
    closed form (arctan)."""
    lam_um = bin_centre_wavelength(nu_edges) / MICRON
    lam_c = 0.5 * (n_carbon / 50.0) ** 0.25
    cont = PAH_UV_SIGMA * (lam_um / 0.1) ** -1.0 / (1.0 + (lam_um / lam_c) ** 6)
    nu0, nu1 = nu_edges[:-1], nu_edges[1:]
    bands = np.zeros_like(cont)
    for lc in PAH_BAND_LAMBDA_UM:
        nuc = C_LIGHT / (lc * MICRON)
        hw = 0.5 * PAH_BAND_FWHM_FRAC * nuc
        # Lorentzian with peak PAH_BAND_PEAK: sigma(nu) = peak hw^2 / ((nu-nuc)^2 + hw^2)
        integral = PAH_BAND_PEAK * hw * (np.arctan((nu1 - nuc) / hw) - np.arctan((nu0 - nuc) / hw))
        bands += integral / (nu1 - nu0)
    return cont + bands


def pah_modes(n_carbon: int, n_hydrogen: int) -> tuple:
    """Einstein-type vibrational modes (count, characteristic temperature K):
    3 N_C - 6 skeletal C-C modes at 900 K, 2 N_H C-H bends at 1600 K and N_H C-H
    stretches at 4360 K -- 3 (N_C + N_H) - 6 modes in all."""
    return ((3 * n_carbon - 6, 900.0), (2 * n_hydrogen, 1600.0), (n_hydrogen, 4360.0))


def pah_species(nu_edges: np.ndarray, n_carbon: int) -> Species:
    """A PAH species: absorption only (no scattering), opacity per gram of PAH."""
    nh = pah_hydrogens(n_carbon)
    m = (12.011 * n_carbon + 1.008 * nh) * AMU
    sigma = n_carbon * pah_cross_section_per_carbon(nu_edges, n_carbon)
    kabs = sigma / m
    lam = bin_centre_wavelength(nu_edges)
    kv = float(np.interp(math.log(LAMBDA_V), np.log(lam[::-1]), kabs[::-1]))
    return Species(f"pah{n_carbon}", kabs, np.zeros_like(kabs), np.zeros_like(kabs), kv,
                   is_pah=1, n_carbon=n_carbon, n_hydrogen=nh, mol_mass=m,
                   modes=pah_modes(n_carbon, nh))


# Mass split between the two large-grain species, from the abundances [Si] = 31 ppm
# and [amorphous C] = 150 ppm (Sec. 1) weighted by a representative grain mass per
# key atom: olivine MgFeSiO4 172 amu per Si, amorphous carbon 12 amu per C.
SIL_MASS_PER_SI = 172.0
CARB_MASS_PER_C = 12.0
MASS_FRACTION = np.array([31.0 * SIL_MASS_PER_SI, 150.0 * CARB_MASS_PER_C])
MASS_FRACTION = MASS_FRACTION / MASS_FRACTION.sum()


def two_species(nu_edges: np.ndarray) -> List[Species]:
    """Silicate (beta 1.5, albedo_V 0.5) and amorphous carbon (beta 1.0, albedo_V 0.3)."""
    return [powerlaw_species("silicate", nu_edges, 1.0e4, 0.5, 1.5),
            powerlaw_species("amorphous_carbon", nu_edges, 2.0e4, 0.3, 1.0)]


# --------------------------------------------------------------------------- star

@dataclasses.dataclass
class Star:
    T: float = 5800.0
    R: float = RSUN
    pos_cm: tuple = (0.0, 0.0, 0.0)
    kind: int = SOURCE_POINT
    beam_dir: tuple = (0.0, 0.0, 1.0)

    @property
    def L(self) -> float:
        return 4.0 * math.pi * self.R ** 2 * SIGMA_SB * self.T ** 4


# --------------------------------------------------------------------------- model

@dataclasses.dataclass
class Model:
    name: str
    half_size: float             # cm
    tree: Tree
    rho: np.ndarray              # float64 [S][N]
    nu_edges: np.ndarray         # float64 [B+1]
    species: List[Species]
    star: Star
    n_sed_dirs: int = 1
    recipe: dict = dataclasses.field(default_factory=dict)

    @property
    def n_bins(self) -> int:
        return int(self.nu_edges.shape[0] - 1)

    @property
    def n_species(self) -> int:
        return len(self.species)

    def opacity_arrays(self):
        kabs = np.stack([s.kabs for s in self.species]).astype(np.float64)
        ksca = np.stack([s.ksca for s in self.species]).astype(np.float64)
        g = np.stack([s.g for s in self.species]).astype(np.float64)
        return kabs, ksca, g

    def cell_size_cm(self) -> float:
        return 2.0 * self.half_size / self.tree.n_base


# --------------------------------------------------------------------------- helpers

def _split_species(rho_total: np.ndarray, fractions: Sequence[float]) -> np.ndarray:
    f = np.asarray(fractions, dtype=np.float64)
    return (f[:, None] * rho_total[None, :]).astype(np.float64)


def leaf_bounds_cm(tree: Tree, half_size: float):
    """Leaf corners in cm (origin at the domain centre)."""
    lo, hi = tree.leaf_bounds()
    d0 = 2.0 * half_size / tree.n_base
    return lo * d0 - half_size, hi * d0 - half_size


def tau_v_along_plus_x(tree: Tree, rho: np.ndarray, species: Sequence[Species],
                       half_size: float) -> float:
    """V-band optical depth from the domain centre to the +x boundary, summed over the
    row of leaves whose lower y and z faces lie on the x axis (the centre is a cube
    corner, so the axis runs along cell edges; the builders here are symmetric in y and
    z, so all four rows around the axis agree)."""
    lo, hi = tree.leaf_bounds()
    c = tree.n_base / 2.0
    row = (lo[:, 1] == c) & (lo[:, 2] == c) & (lo[:, 0] >= c)
    d0 = 2.0 * half_size / tree.n_base
    kv = np.array([s.kappa_v_ext for s in species])
    dens = (kv[:, None] * rho[:, row]).sum(axis=0)
    return float((dens * (hi[row, 0] - lo[row, 0]) * d0).sum())


def normalise_tau(model_rho: np.ndarray, tree: Tree, species, half_size: float,
                  tau_v: float) -> np.ndarray:
    t = tau_v_along_plus_x(tree, model_rho, species, half_size)
    if not t > 0:
        raise ValueError("the +x row from the centre holds no dust")
    return model_rho * (tau_v / t)


# --------------------------------------------------------------------------- workloads

def sphere_model(n_base: int = 16, n_bins: int = 64, radius_au: float = 1.0e3,
                 tau_v: float = 1.0, species: Optional[List[Species]] = None,
                 fractions: Optional[Sequence[float]] = None, n_sed_dirs: int = 1
                 ) -> Model:
    """Homogeneous dust sphere of ``radius_au`` in a cube of the same half-size, central
    5800 K star, density uniform in every cube whose centre lies inside the radius
    ("staircased"), scaled so that the V-band optical depth from the centre along +x
    equals ``tau_v`` (the Fig. 1 set-up of Sec. 2 with smooth synthetic grains)."""
    H = radius_au * AU
    nu = frequency_edges(n_bins)
    sp = species if species is not None else two_species(nu)
    fr = fractions if fractions is not None else (MASS_FRACTION if len(sp) == 2 else
                                                  np.full(len(sp), 1.0 / len(sp)))
    tree = build_tree(n_base, 0)
    lo, hi = leaf_bounds_cm(tree, H)
    ctr = 0.5 * (lo + hi)
    inside = np.sqrt((ctr ** 2).sum(axis=1)) <= H
    rho = _split_species(inside.astype(np.float64), fr)
    rho = normalise_tau(rho, tree, sp, H, tau_v)
    return Model("sphere", H, tree, rho, nu, list(sp), Star(), n_sed_dirs,
                 recipe=dict(n_base=n_base, n_bins=n_bins, radius_au=radius_au,
                             tau_v=tau_v, fractions=list(map(float, fr))))


DISK_R_IN_AU = 0.1
DISK_R_OUT_AU = 100.0
DISK_H0_OVER_RIN = 0.05
DISK_FLARE = 1.125


def _disk_scale_height(r_cm, r_in):
    return DISK_H0_OVER_RIN * r_in * (np.maximum(r_cm, 1e-30) / r_in) ** DISK_FLARE


def disk_perturbation(r_cm: np.ndarray, phi: np.ndarray, gap_r_au: float = 10.0,
                      gap_depth: float = 0.1, gap_w_au: float = 1.0,
                      spiral_amp: float = 0.3, pitch_deg: float = 15.0,
                      spiral_r0_au: float = 10.0) -> np.ndarray:
    """Planet perturbation: Gaussian gap whose centre density is ``gap_depth`` of the
    unperturbed value, times a two-arm logarithmic spiral of relative amplitude
    ``spiral_amp``."""
    r_au = r_cm / AU
    gap = 1.0 - (1.0 - gap_depth) * np.exp(-(r_au - gap_r_au) ** 2 / (2.0 * gap_w_au ** 2))
    lnr = np.log(np.maximum(r_au, 1e-30) / spiral_r0_au)
    spiral = 1.0 + spiral_amp * np.cos(2.0 * (phi - lnr / math.tan(math.radians(pitch_deg))))
    return gap * spiral


def _disk_cell_average(lo: np.ndarray, hi: np.ndarray, r_in: float, r_out: float,
                       perturb: bool, ns: int = 2) -> np.ndarray:
    """Cell-averaged r^-1 exp(-z^2/2h^2): ns x ns midpoint samples in (x, y), the z
    average of the Gaussian taken in closed form (erf)."""
    from scipy.special import erf
    acc = np.zeros(lo.shape[0])
    dz = hi[:, 2] - lo[:, 2]
    for a in (np.arange(ns) + 0.5) / ns:
        x = lo[:, 0] + a * (hi[:, 0] - lo[:, 0])
        for b in (np.arange(ns) + 0.5) / ns:
            y = lo[:, 1] + b * (hi[:, 1] - lo[:, 1])
            r = np.hypot(x, y)
            h = _disk_scale_height(r, r_in)
            s = h * math.sqrt(2.0)
            zavg = h * math.sqrt(math.pi / 2.0) * (erf(hi[:, 2] / s) - erf(lo[:, 2] / s)) / dz
            val = (r_in / np.maximum(r, 1e-30)) * zavg
            if perturb:
                val = val * disk_perturbation(r, np.arctan2(y, x))
            acc += np.where((r >= r_in) & (r <= r_out), val, 0.0)
    return acc / (ns * ns)


def disk_refine_fn(n_base: int, half_size: float, r_in: float, r_out: float,
                   zfac: Sequence[float] = (2.0,)):
    """Refine a node if it comes within 2 r_in of the star, or if it reaches below
    zfac[level] times the local scale height, |z| < zfac h(r), inside the disk's radial
    range (the last entry of zfac holds for deeper levels)."""
    d0 = 2.0 * half_size / n_base

    def refine(level, lo, hi):
        lo_cm = lo * d0 - half_size
        hi_cm = hi * d0 - half_size
        # nearest/farthest cylindrical radius over the box
        nx = np.clip(0.0, lo_cm[:, 0], hi_cm[:, 0])
        ny = np.clip(0.0, lo_cm[:, 1], hi_cm[:, 1])
        rmin = np.hypot(nx, ny)
        fx = np.maximum(np.abs(lo_cm[:, 0]), np.abs(hi_cm[:, 0]))
        fy = np.maximum(np.abs(lo_cm[:, 1]), np.abs(hi_cm[:, 1]))
        rmax = np.hypot(fx, fy)
        zmin = np.where((lo_cm[:, 2] <= 0) & (hi_cm[:, 2] >= 0), 0.0,
                        np.minimum(np.abs(lo_cm[:, 2]), np.abs(hi_cm[:, 2])))
        near_star = np.hypot(rmin, zmin) < 2.0 * r_in
        c = zfac[level] if level < len(zfac) else zfac[-1]
        in_disk = (zmin < c * _disk_scale_height(rmax, r_in)) & (rmin <= r_out) & \
                  (rmax >= r_in)
        return near_star | in_disk

    return refine


def disk_model(n_base: int = 128, max_level: int = 2, n_bins: int = 200,
               tau_v_mid: float = 1.0e3, half_size_au: float = 100.0,
               perturbed: bool = False, species: Optional[List[Species]] = None,
               fractions: Optional[Sequence[float]] = None, n_sed_dirs: int = 1,
               refine_zfac: Sequence[float] = (2.0,)) -> Model:
    """Flared disk rho ~ r^-1 exp(-z^2/2h^2), h = 0.05 r_in (r/r_in)^1.125 over
    0.1-100 AU, in a cube of half-size ``half_size_au`` with ``max_level`` levels of
    2x2x2 refinement near the inner rim and the midplane; the density is scaled so that
    the V-band optical depth along the midplane (+x from the star) equals
    ``tau_v_mid``. ``perturbed`` adds the gap at 10 AU and the two-arm spiral."""
    H = half_size_au * AU
    r_in, r_out = DISK_R_IN_AU * AU, DISK_R_OUT_AU * AU
    nu = frequency_edges(n_bins)
    sp = species if species is not None else two_species(nu)
    fr = fractions if fractions is not None else (MASS_FRACTION if len(sp) == 2 else
                                                  np.full(len(sp), 1.0 / len(sp)))
    tree = build_tree(n_base, max_level, disk_refine_fn(n_base, H, r_in, r_out, refine_zfac))
    lo, hi = leaf_bounds_cm(tree, H)
    dens = _disk_cell_average(lo, hi, r_in, r_out, perturbed)
    rho = _split_species(dens, fr)
    rho = normalise_tau(rho, tree, sp, H, tau_v_mid)
    return Model("disk_perturbed" if perturbed else "disk", H, tree, rho, nu, list(sp),
                 Star(), n_sed_dirs,
                 recipe=dict(n_base=n_base, max_level=max_level, n_bins=n_bins,
                             tau_v_mid=tau_v_mid, half_size_au=half_size_au,
                             r_in_au=DISK_R_IN_AU, r_out_au=DISK_R_OUT_AU,
                             h0_over_rin=DISK_H0_OVER_RIN, flare=DISK_FLARE,
                             perturbed=perturbed, fractions=list(map(float, fr)),
                             refine_zfac=list(map(float, refine_zfac))))


PAH_MASS_FRACTION = 0.05   # of the dust mass, split equally between the two PAH sizes


def disk_pah_model(n_base: int = 128, max_level: int = 2, n_bins: int = 200,
                   tau_v_mid: float = 1.0e3, perturbed: bool = True,
                   pah_sizes: Sequence[int] = (30, 200),
                   refine_zfac: Sequence[float] = (2.0,)) -> Model:
    """The disk with the planet's gap and spiral and four species: silicate, amorphous
    carbon and two PAH sizes (30 and 200 C atoms) carrying PAH_MASS_FRACTION of the
    dust mass."""
    nu = frequency_edges(n_bins)
    sp = two_species(nu) + [pah_species(nu, n) for n in pah_sizes]
    fr = list(MASS_FRACTION * (1.0 - PAH_MASS_FRACTION)) + \
        [PAH_MASS_FRACTION / len(pah_sizes)] * len(pah_sizes)
    m = disk_model(n_base=n_base, max_level=max_level, n_bins=n_bins, tau_v_mid=tau_v_mid,
                   perturbed=perturbed, species=sp, fractions=fr, refine_zfac=refine_zfac)
    m.name = "disk_pah"
    m.recipe["pah_mass_fraction"] = PAH_MASS_FRACTION
    m.recipe["pah_sizes"] = list(pah_sizes)
    return m


def large_disk_model() -> Model:
    """The large disk: gap, spiral and the four species of disk_pah_model on 256^3 base
    cubes with three levels of refinement (|z| below 1, 0.5 and 0.25 scale heights for
    the first, second and third split; 1.73e8 leaves) and 400 frequency bins."""
    m = disk_pah_model(n_base=256, max_level=3, n_bins=400, refine_zfac=(1.0, 0.5, 0.25))
    m.name = "large_disk"
    return m


def disk4_model(n_base: int = 128, max_level: int = 2, n_bins: int = 400) -> Model:
    """The PAH disk's geometry and four species' opacities, all four treated as
    ordinary dust (no PAH tallies): the four-species walk with about 2.5 GB on the
    device at 128^3 base cubes and two levels, for profiling the transport."""
    m = disk_pah_model(n_base=n_base, max_level=max_level, n_bins=n_bins)
    m.species = [dataclasses.replace(sp, is_pah=0, n_carbon=0, n_hydrogen=0, mol_mass=0.0,
                                     modes=()) for sp in m.species]
    m.name = "disk4"
    return m


def uniform_box_model(n_base: int, n_bins: int, tau_half: float, species: List[Species],
                      half_size_cm: float = AU, star: Optional[Star] = None,
                      max_level: int = 0, refine=None, n_sed_dirs: int = 1) -> Model:
    """Dust of uniform density filling the whole cube (every leaf), scaled so that the
    V-band optical depth from the centre to a face along +x is ``tau_half``."""
    tree = build_tree(n_base, max_level, refine)
    rho = _split_species(np.ones(tree.n_leaves), np.full(len(species), 1.0 / len(species)))
    rho = normalise_tau(rho, tree, species, half_size_cm, tau_half)
    return Model("box", half_size_cm, tree, rho, frequency_edges(n_bins), list(species),
                 star if star is not None else Star(), n_sed_dirs,
                 recipe=dict(n_base=n_base, tau_half=tau_half))


def explicit_model(tree: Tree, rho: np.ndarray, n_bins: int, species: List[Species],
                   half_size_cm: float = AU, star: Optional[Star] = None,
                   n_sed_dirs: int = 1, name: str = "explicit") -> Model:
    """Model from a caller-given tree and per-leaf species densities."""
    rho = np.asarray(rho, dtype=np.float64).reshape(len(species), tree.n_leaves)
    return Model(name, half_size_cm, tree, rho, frequency_edges(n_bins), list(species),
                 star if star is not None else Star(), n_sed_dirs)


def sphere_refine_fn(n_base: int, frac: float = 0.25):
    """Refine nodes reaching within frac * half-size of the centre (the star)."""
    c = n_base / 2.0
    r0 = frac * c

    def refine(level, lo, hi):
        near = np.clip(c, lo, hi)
        return np.sqrt(((near - c) ** 2).sum(axis=1)) < r0

    return refine


def batch_models(n_models: int = 256, seed: int = 0, n_bins: int = 100, sizes=None):
    """The uneven batch: models from random_model_list, each a sphere (radius = half
    size 1e3 AU, refined near the star) or a flared disk, with its optical depth and
    package count. Trees and unscaled densities are shared between models of the same
    kind and shape (optical depth only rescales the density)."""
    specs = random_model_list(n_models, seed, n_bins)
    if sizes is not None:
        for sp in specs:
            sp["n_base"] = sizes[sp["index"] % len(sizes)]
    cache = {}
    out = []
    for sp in specs:
        key = (sp["kind"], sp["n_base"], sp["max_level"])
        if key not in cache:
            if sp["kind"] == "disk":
                base = disk_model(n_base=sp["n_base"], max_level=sp["max_level"], n_bins=n_bins,
                                  tau_v_mid=1.0)
            else:
                H = 1.0e3 * AU
                nu = frequency_edges(n_bins)
                spc = two_species(nu)
                tree = build_tree(sp["n_base"], sp["max_level"], sphere_refine_fn(sp["n_base"]))
                lo, hi = leaf_bounds_cm(tree, H)
                inside = np.sqrt((((lo + hi) / 2) ** 2).sum(axis=1)) <= H
                rho = _split_species(inside.astype(np.float64), MASS_FRACTION)
                rho = normalise_tau(rho, tree, spc, H, 1.0)
                base = Model("sphere", H, tree, rho, nu, spc, Star(), 1,
                             recipe=dict(n_base=sp["n_base"], max_level=sp["max_level"]))
            cache[key] = base
        b = cache[key]
        m = dataclasses.replace(b, rho=b.rho * sp["tau_v"], recipe=dict(b.recipe, **sp))
        out.append((m, sp["n_packages"]))
    return out


def random_model_list(n_models: int = 256, seed: int = 0, n_bins: int = 100):
    """Parameters of a batch of uneven sphere/disk models: base grid in
    {32,48,64,96,128}^3, 1-2 levels, optical depth log-uniform in [0.1, 1e3],
    packages log-uniform in [1e5, 1e7], sphere or disk with equal odds."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_models):
        out.append(dict(
            index=i,
            kind="sphere" if rng.random() < 0.5 else "disk",
            n_base=int(rng.choice([32, 48, 64, 96, 128])),
            max_level=int(rng.integers(1, 3)),
            tau_v=float(10.0 ** rng.uniform(-1.0, 3.0)),
            n_packages=int(10.0 ** rng.uniform(5.0, 7.0)),
            n_bins=n_bins))
    return out
