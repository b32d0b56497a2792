"""CPU oracle: plain FP64 Monte Carlo of the photon-package transport (Sec. 2 of
Siebenmorgen, Heymann & Kruegel), in C (``rt_oracle.c``) behind ctypes.

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the library (``paper_1201_3588_gb300``)
never does, and the two share no code. Inputs come from
``paper_1201_3588_gb300.workloads`` (model builders only).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_BW, MODE_NOCORR, MODE_FROZEN = 0, 1, 2
T_MIN_DEFAULT = 1.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no tuning)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    srcs = [_SRC, os.path.join(_HERE, "rt_oracle.h")]
    if not force and os.path.exists(_LIB) and \
            os.path.getmtime(_LIB) >= max(os.path.getmtime(s) for s in srcs):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                           "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("half_size", C.c_double), ("n_base", C.c_int32), ("max_level", C.c_int32),
                ("base", C.c_void_p), ("child", C.c_void_p), ("n_blocks", C.c_int64),
                ("n_leaves", C.c_int64), ("n_species", C.c_int32), ("n_bins", C.c_int32),
                ("rho", C.c_void_p), ("kabs", C.c_void_p), ("ksca", C.c_void_p),
                ("g", C.c_void_p), ("nu_edges", C.c_void_p), ("star_T", C.c_double),
                ("star_L", C.c_double), ("star_pos", C.c_double * 3),
                ("source_kind", C.c_int32), ("n_sed_dirs", C.c_int32),
                ("beam_dir", C.c_double * 3), ("pah_index", C.c_void_p),
                ("pah_template", C.c_void_p), ("n_coarse", C.c_int32), ("n_pah", C.c_int32),
                ("pah_cell_w", C.c_void_p)]


class _Run(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("first_id", C.c_uint64), ("n_packages", C.c_uint64),
                ("n_total", C.c_uint64), ("mode", C.c_int32), ("pad", C.c_int32),
                ("max_events", C.c_uint64), ("t_min", C.c_double),
                ("T_frozen", C.c_void_p), ("obs_dir", C.c_double * 3),
                ("plane_of_bin", C.c_void_p), ("n_planes", C.c_int32), ("nx", C.c_int32),
                ("ny", C.c_int32), ("pad2", C.c_int32), ("img_half", C.c_double)]


class _Tally(C.Structure):
    _fields_ = [("count", C.c_void_p), ("sed", C.c_void_p), ("pahabs", C.c_void_p),
                ("pathabs", C.c_void_p), ("image", C.c_void_p), ("emitted", C.c_uint64),
                ("escaped", C.c_uint64), ("capped", C.c_uint64),
                ("absorptions", C.c_uint64), ("scatters", C.c_uint64),
                ("crossings", C.c_uint64), ("errors", C.c_uint64)]


class _Trace(C.Structure):
    _fields_ = [("id", C.c_uint64), ("events", C.c_uint64), ("absorptions", C.c_uint64),
                ("scatters", C.c_uint64), ("crossings", C.c_uint64),
                ("escaped", C.c_int32), ("capped", C.c_int32), ("final_bin", C.c_int32),
                ("dir_bin", C.c_int32), ("last_leaf", C.c_int64),
                ("dir", C.c_double * 3)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, u32p, dp = C.c_double, C.POINTER(C.c_uint32), C.c_void_p
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = d
            for f in (L.orc_planck_bin, L.orc_dplanck_bin):
                f.argtypes = [d, d, d]
                f.restype = d
            L.orc_emission_per_mass.argtypes = [dp, dp, C.c_int, d]
            L.orc_emission_per_mass.restype = d
            L.orc_temperature.argtypes = [dp, dp, C.c_int, d]
            L.orc_temperature.restype = d
            L.orc_hg_mu.argtypes = [d, d]
            L.orc_hg_mu.restype = d
            L.orc_rotate.argtypes = [dp, d, d]
            L.orc_locate.argtypes = [C.POINTER(_Model), dp, dp, dp]
            L.orc_locate.restype = C.c_int
            L.orc_ray_cells.argtypes = [C.POINTER(_Model), dp, dp, C.c_int64, dp, dp]
            L.orc_ray_cells.restype = C.c_int64
            L.orc_package_energy.argtypes = [C.POINTER(_Model), C.c_uint64]
            L.orc_package_energy.restype = d
            L.orc_optical_depth.argtypes = [C.POINTER(_Model), dp, dp, C.c_int]
            L.orc_optical_depth.restype = d
            L.orc_transport.argtypes = [C.POINTER(_Model), C.POINTER(_Run), C.POINTER(_Tally)]
            L.orc_transport.restype = C.c_int
            L.orc_trace.argtypes = [C.POINTER(_Model), C.POINTER(_Run), dp, C.c_int64, dp]
            L.orc_trace.restype = C.c_int
            L.orc_trace_events.argtypes = [C.POINTER(_Model), C.POINTER(_Run), C.c_uint64,
                                           C.c_int64, dp, C.POINTER(C.c_int64)]
            L.orc_trace_events.restype = C.c_int
            L.orc_temperatures.argtypes = [C.POINTER(_Model), dp, d, dp]
            L.orc_temperatures.restype = C.c_int
            L.orc_reemit_bin.argtypes = [C.POINTER(_Model), C.c_int, C.c_int, C.c_uint64, d,
                                         d, d, d, d]
            L.orc_reemit_bin.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ------------------------------------------------------------------ scalar functions

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(x: int) -> float:
    return lib().orc_uniform(int(x) & 0xFFFFFFFF)


def planck_bin(nu0, nu1, T):
    return lib().orc_planck_bin(float(nu0), float(nu1), float(T))


def dplanck_bin(nu0, nu1, T):
    return lib().orc_dplanck_bin(float(nu0), float(nu1), float(T))


def emission_per_mass(kabs, nu_edges, T):
    ka = np.ascontiguousarray(kabs, dtype=np.float64)
    nu = np.ascontiguousarray(nu_edges, dtype=np.float64)
    return lib().orc_emission_per_mass(_ptr(ka), _ptr(nu), ka.shape[0], float(T))


def temperature(kabs, nu_edges, u):
    ka = np.ascontiguousarray(kabs, dtype=np.float64)
    nu = np.ascontiguousarray(nu_edges, dtype=np.float64)
    return lib().orc_temperature(_ptr(ka), _ptr(nu), ka.shape[0], float(u))


def hg_mu(g, xi):
    return lib().orc_hg_mu(float(g), float(xi))


def rotate(d, mu, phi):
    a = np.ascontiguousarray(d, dtype=np.float64).copy()
    lib().orc_rotate(_ptr(a), float(mu), float(phi))
    return a


# ------------------------------------------------------------------ models

N_COARSE = 64


class OracleModel:
    """ctypes view of a ``workloads.Model`` (arrays kept alive here). For PAH species
    the template re-emission spectra come from ``oracle.pah`` unless given;
    ``pah_cell_spectra`` [n_pah][N][B] gives each cell its own PAH re-emission
    spectrum (rows of zeros: the template)."""

    def __init__(self, model, pah_template=None, pah_cell_spectra=None):
        t = model.tree
        self.model = model
        self.base = np.ascontiguousarray(t.base, dtype=np.int32)
        self.child = np.ascontiguousarray(t.child if t.child.size else np.zeros(8, np.int32),
                                          dtype=np.int32)
        self.rho = np.ascontiguousarray(model.rho, dtype=np.float64)
        kabs, ksca, g = model.opacity_arrays()
        self.kabs = np.ascontiguousarray(kabs)
        self.ksca = np.ascontiguousarray(ksca)
        self.g = np.ascontiguousarray(g)
        self.nu = np.ascontiguousarray(model.nu_edges, dtype=np.float64)
        st = model.star
        self.pah_species = [i for i, sp in enumerate(model.species) if sp.is_pah]
        self.n_pah = len(self.pah_species)
        self.n_coarse = min(N_COARSE, model.n_bins)
        self.pah_index = np.full(model.n_species, -1, dtype=np.int32)
        for p, i in enumerate(self.pah_species):
            self.pah_index[i] = p
        if self.n_pah and pah_template is None:
            from . import pah as _pah
            pah_template = np.stack([_pah.template_spectrum(model.species[i], model.nu_edges,
                                                            st.T) for i in self.pah_species])
        self.pah_template = (np.ascontiguousarray(pah_template, dtype=np.float64)
                             if self.n_pah else np.zeros(1))
        self.pah_cell = None
        if pah_cell_spectra is not None:
            self.pah_cell = np.ascontiguousarray(pah_cell_spectra, dtype=np.float64).reshape(
                self.n_pah, t.n_leaves, model.n_bins)
        self.s = _Model(half_size=model.half_size, n_base=t.n_base, max_level=t.max_level,
                        base=_ptr(self.base), child=_ptr(self.child), n_blocks=t.n_blocks,
                        n_leaves=t.n_leaves, n_species=model.n_species,
                        n_bins=model.n_bins, rho=_ptr(self.rho), kabs=_ptr(self.kabs),
                        ksca=_ptr(self.ksca), g=_ptr(self.g), nu_edges=_ptr(self.nu),
                        star_T=st.T, star_L=st.L, star_pos=(C.c_double * 3)(*st.pos_cm),
                        source_kind=st.kind, n_sed_dirs=model.n_sed_dirs,
                        beam_dir=(C.c_double * 3)(*st.beam_dir),
                        pah_index=_ptr(self.pah_index) if self.n_pah else None,
                        pah_template=_ptr(self.pah_template), n_coarse=self.n_coarse,
                        n_pah=self.n_pah,
                        pah_cell_w=_ptr(self.pah_cell) if self.pah_cell is not None else None)

    @property
    def S(self):
        return self.model.n_species

    @property
    def N(self):
        return self.model.tree.n_leaves

    @property
    def B(self):
        return self.model.n_bins


def as_oracle(model) -> OracleModel:
    return model if isinstance(model, OracleModel) else OracleModel(model)


def locate(model, p, d):
    om = as_oracle(model)
    pp = np.ascontiguousarray(p, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(5, dtype=np.int64)
    rc = lib().orc_locate(C.byref(om.s), _ptr(pp), _ptr(dd), _ptr(out))
    return rc, out


def ray_cells(model, p, d, max_cells: int = 1 << 20):
    om = as_oracle(model)
    pp = np.ascontiguousarray(p, dtype=np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    leaves = np.zeros(max_cells, dtype=np.int64)
    lens = np.zeros(max_cells, dtype=np.float64)
    k = lib().orc_ray_cells(C.byref(om.s), _ptr(pp), _ptr(dd), max_cells, _ptr(leaves),
                            _ptr(lens))
    if k < 0:
        raise RuntimeError("ray walk failed")
    return leaves[:k].copy(), lens[:k].copy()


def package_energy(model, n_total: int) -> float:
    om = as_oracle(model)
    return lib().orc_package_energy(C.byref(om.s), int(n_total))


def optical_depth(model, p_cm, direction, bin: int) -> float:
    """Extinction optical depth from p (cm, model centre at 0) along `direction` to
    the model boundary at frequency bin `bin`."""
    om = as_oracle(model)
    pp = np.ascontiguousarray(p_cm, dtype=np.float64)
    dd = np.ascontiguousarray(direction, dtype=np.float64)
    return lib().orc_optical_depth(C.byref(om.s), _ptr(pp), _ptr(dd), int(bin))


@dataclass
class Peel:
    """Peel-off images toward a distant observer: `plane_of_bin[b]` is the image
    plane that bin b contributes to (-1: none); each plane is nx by ny pixels over a
    square of half width `half_width` cm centred on the model, seen along
    `obs_dir` (unit vector pointing to the observer)."""
    obs_dir: np.ndarray
    plane_of_bin: np.ndarray
    nx: int
    ny: int
    half_width: float

    @property
    def n_planes(self) -> int:
        return int(np.max(self.plane_of_bin)) + 1 if np.any(self.plane_of_bin >= 0) else 0


@dataclass
class Tally:
    count: np.ndarray     # uint64 [S][N]
    sed: np.ndarray       # uint64 [2][n_dir][B]
    pahabs: np.ndarray    # uint64 [n_pah][N][n_coarse]
    pathabs: np.ndarray   # float64 [S][N] path-length sums (absorption optical depth)
    image: Optional[np.ndarray] = None  # float64 [n_planes][ny][nx] erg/s/sr (peel-off)
    emitted: int = 0
    escaped: int = 0
    capped: int = 0
    absorptions: int = 0
    scatters: int = 0
    crossings: int = 0
    errors: int = 0


def new_tally(model, peel: Optional[Peel] = None) -> Tally:
    om = as_oracle(model)
    img = None
    if peel is not None:
        img = np.zeros((peel.n_planes, peel.ny, peel.nx), dtype=np.float64)
    return Tally(np.zeros((om.S, om.N), dtype=np.uint64),
                 np.zeros((2, om.model.n_sed_dirs, om.B), dtype=np.uint64),
                 np.zeros((max(om.n_pah, 1), om.N, om.n_coarse), dtype=np.uint64),
                 np.zeros((om.S, om.N), dtype=np.float64), img)


def _run(n_packages, seed, first_id, n_total, mode, max_events, t_min, T_frozen,
         peel: Optional[Peel] = None):
    tf = None
    if T_frozen is not None:
        tf = np.ascontiguousarray(T_frozen, dtype=np.float64)
    r = _Run(seed=int(seed), first_id=int(first_id), n_packages=int(n_packages),
             n_total=int(n_total), mode=int(mode), pad=0, max_events=int(max_events),
             t_min=float(t_min), T_frozen=_ptr(tf) if tf is not None else None)
    keep = [tf]
    if peel is not None:
        o = np.asarray(peel.obs_dir, dtype=np.float64)
        o = o / np.linalg.norm(o)
        pob = np.ascontiguousarray(peel.plane_of_bin, dtype=np.int32)
        keep.append(pob)
        r.obs_dir = (C.c_double * 3)(*o)
        r.plane_of_bin = _ptr(pob)
        r.n_planes, r.nx, r.ny = peel.n_planes, int(peel.nx), int(peel.ny)
        r.img_half = float(peel.half_width)
    return r, keep


def transport(model, n_packages: int, seed: int = 0, first_id: int = 0,
              n_total: Optional[int] = None, mode: int = MODE_BW,
              max_events: int = 10_000_000, t_min: float = T_MIN_DEFAULT,
              T_frozen: Optional[np.ndarray] = None, tally: Optional[Tally] = None,
              peel: Optional[Peel] = None) -> Tally:
    """Follow packages ``first_id .. first_id+n_packages-1``; counts accumulate into
    ``tally`` (a new one if None). With ``peel``, every emission, scattering and
    re-emission also sends its share toward the observer into ``tally.image``."""
    om = as_oracle(model)
    tl = tally if tally is not None else new_tally(om, peel)
    if peel is not None and (tl.image is None or tl.image.shape !=
                             (peel.n_planes, peel.ny, peel.nx)):
        raise ValueError("tally has no image of the peel-off shape")
    r, keep = _run(n_packages, seed, first_id, n_total or n_packages, mode, max_events,
                   t_min, T_frozen, peel)
    ct = _Tally(count=_ptr(tl.count), sed=_ptr(tl.sed), pahabs=_ptr(tl.pahabs),
                pathabs=_ptr(tl.pathabs),
                image=_ptr(tl.image) if (peel is not None) else None,
                emitted=tl.emitted,
                escaped=tl.escaped, capped=tl.capped, absorptions=tl.absorptions,
                scatters=tl.scatters, crossings=tl.crossings, errors=tl.errors)
    rc = lib().orc_transport(C.byref(om.s), C.byref(r), C.byref(ct))
    if rc != 0:
        raise RuntimeError(f"oracle transport failed ({rc})")
    for f in ("emitted", "escaped", "capped", "absorptions", "scatters", "crossings",
              "errors"):
        setattr(tl, f, int(getattr(ct, f)))
    return tl


TRACE_DTYPE = np.dtype([("id", np.uint64), ("events", np.uint64), ("absorptions", np.uint64),
                        ("scatters", np.uint64), ("crossings", np.uint64),
                        ("escaped", np.int32), ("capped", np.int32), ("final_bin", np.int32),
                        ("dir_bin", np.int32), ("last_leaf", np.int64),
                        ("dir", np.float64, (3,))])
assert TRACE_DTYPE.itemsize == C.sizeof(_Trace)


def trace(model, ids, T_frozen, seed: int = 0, n_total: int = 1,
          max_events: int = 10_000_000, t_min: float = T_MIN_DEFAULT) -> np.ndarray:
    """Histories of the listed packages in the frozen-temperature mode."""
    om = as_oracle(model)
    idv = np.ascontiguousarray(ids, dtype=np.uint64)
    out = np.zeros(idv.shape[0], dtype=TRACE_DTYPE)
    r, keep = _run(0, seed, 0, n_total, MODE_FROZEN, max_events, t_min, T_frozen)
    rc = lib().orc_trace(C.byref(om.s), C.byref(r), _ptr(idv), idv.shape[0], _ptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle trace failed ({rc})")
    return out


EVENT_DTYPE = np.dtype([("kind", np.int32), ("species", np.int32), ("leaf", np.int64),
                        ("bin", np.int32), ("pad", np.int32), ("pos", np.float64, (3,))])
EVENT_EMIT, EVENT_SCATTER, EVENT_ABSORB, EVENT_ESCAPE, EVENT_CAPPED = 0, 1, 2, 3, 4


def trace_events(model, package_id: int, T_frozen, seed: int = 0, n_total: int = 1,
                 max_events: int = 10_000_000, t_min: float = T_MIN_DEFAULT,
                 max_out: int = 1 << 16):
    """The events of one package in the frozen-temperature mode: its emission (bin,
    source position), every scattering and absorption (kind, species, cell, bin after
    the event, position in base-cube units), then its escape or cap. Returns (events,
    total number of events)."""
    om = as_oracle(model)
    out = np.zeros(max_out, dtype=EVENT_DTYPE)
    n = C.c_int64()
    r, keep = _run(0, seed, 0, n_total, MODE_FROZEN, max_events, t_min, T_frozen)
    rc = lib().orc_trace_events(C.byref(om.s), C.byref(r), int(package_id), int(max_out),
                                _ptr(out), C.byref(n))
    if rc != 0:
        raise RuntimeError(f"oracle event trace failed ({rc})")
    return out[:min(n.value, max_out)].copy(), int(n.value)


def temperatures(model, count: np.ndarray, eps: float) -> np.ndarray:
    om = as_oracle(model)
    cnt = np.ascontiguousarray(count, dtype=np.uint64).reshape(om.S, om.N)
    T = np.zeros((om.S, om.N), dtype=np.float64)
    rc = lib().orc_temperatures(C.byref(om.s), _ptr(cnt), float(eps), _ptr(T))
    if rc != 0:
        raise RuntimeError("oracle temperatures failed")
    return T


def reemit_bin(model, species: int, mode: int, n: int, eps_over_m: float, u_frozen: float,
               t_min: float, xi_u: float, xi_bin: float) -> int:
    om = as_oracle(model)
    return lib().orc_reemit_bin(C.byref(om.s), species, mode, n, eps_over_m, u_frozen,
                                t_min, xi_u, xi_bin)
