"""Python binding of librt_gb300 (include/rt.h) through ctypes.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. Importing this module loads the library and raises if it cannot be
found or built; there is no fallback. PyTorch, when used, only supplies device
buffers (``tensor.data_ptr()``) and streams (``stream.cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import _build

REEMIT_BW, REEMIT_NOCORR, REEMIT_FROZEN = 0, 1, 2
EST_PATHLENGTH = 1
PAH_EXACT, PAH_SURROGATE, PAH_AUTO = 0, 1, 2
KERNEL_POOL, KERNEL_PLAIN_F32, KERNEL_PLAIN_F64 = 0, 1, 2
WALK_AUTO, WALK_LINKED, WALK_PATH = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA runtime error",
          4: "kernel stopped at its time budget", 5: "call out of order",
          6: "package ids beyond the planned total", 7: "malformed grid met on the device",
          8: "request exceeds a fixed maximum"}

EVENT_DTYPE = np.dtype([("kind", np.int32), ("species", np.int32), ("leaf", np.int32),
                        ("bin", np.int32), ("pos", np.float32, (3,)), ("pad", np.int32)])
EVENT_EMIT, EVENT_SCATTER, EVENT_ABSORB, EVENT_ESCAPE, EVENT_CAPPED = 0, 1, 2, 3, 4

TRACE_FIELDS = ("events", "absorptions", "scatters", "crossings", "escaped", "capped",
                "final_bin", "dir_bin", "last_leaf")


class RTError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


class _Desc(C.Structure):
    _fields_ = [("half_size_cm", C.c_double), ("n_base", C.c_int32), ("max_level", C.c_int32),
                ("n_blocks", C.c_int64), ("n_leaves", C.c_int64), ("base", C.c_void_p),
                ("child", C.c_void_p), ("n_species", C.c_int32), ("n_bins", C.c_int32),
                ("rho", C.c_void_p), ("nu_edges", C.c_void_p), ("n_sed_dirs", C.c_int32),
                ("n_temp", C.c_int32), ("t_min", C.c_double), ("t_max", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("kernel", C.c_int32), ("max_events", C.c_uint64),
                ("blocks_per_sm", C.c_int32), ("threads", C.c_int32),
                ("refill_period", C.c_int32), ("interaction_batch", C.c_int32),
                ("budget_s", C.c_double), ("estimators", C.c_int32),
                ("count_scale", C.c_int32), ("walk", C.c_int32), ("reserved", C.c_int32)]


class _Counters(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("emitted", "escaped", "capped", "absorptions",
                                          "scatters", "crossings", "errors", "clamped",
                                          "levels", "peel_events", "peel_crossings",
                                          "peel_dropped")]


class _PtCase(C.Structure):
    _fields_ = [("modes", (C.c_double * 2) * 4), ("n_groups", C.c_int32),
                ("reserved", C.c_int32), ("h_nu_erg", C.c_double), ("rate", C.c_double),
                ("t_top", C.c_double)]


class _ImageDesc(C.Structure):
    _fields_ = [("obs_dir", C.c_double * 3), ("nx", C.c_int32), ("ny", C.c_int32),
                ("half_width_cm", C.c_double), ("tau_max", C.c_double),
                ("event_capacity", C.c_uint64)]


_lib = None

# exported symbols with their argument types; every name declared in include/rt.h
SIGNATURES = {
    "rt_grid_create": [C.POINTER(_Desc), C.POINTER(C.c_void_p)],
    "rt_grid_destroy": [C.c_void_p],
    "rt_set_dust": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                    C.c_int],
    "rt_emit_star": [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_int, C.c_void_p,
                     C.c_uint64],
    "rt_set_frozen_temperatures": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_transport": [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(_Opts),
                     C.c_void_p],
    "rt_reset": [C.c_void_p, C.c_void_p],
    "rt_cell_temperatures": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_sed": [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p],
    "rt_counts": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_cell_temperatures_pathlength": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_pathlength": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_set_counts": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_get_counters": [C.c_void_p, C.POINTER(_Counters)],
    "rt_set_images": [C.c_void_p, C.POINTER(_ImageDesc), C.c_void_p],
    "rt_images": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_image_profile": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                         C.c_void_p],
    "rt_trace": [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_uint64, C.c_void_p],
    "rt_trace_events": [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_uint64, C.c_int64,
                        C.c_void_p, C.c_void_p],
    "rt_philox": [C.c_void_p, C.c_int64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_void_p],
    "rt_status_string": [C.c_int],
    "rt_batch_create": [C.c_void_p, C.c_int, C.c_void_p, C.c_uint64, C.POINTER(_Opts),
                        C.c_uint64, C.POINTER(C.c_void_p)],
    "rt_batch_destroy": [C.c_void_p],
    "rt_batch_run": [C.c_void_p, C.c_int, C.c_int, C.c_void_p],
    "rt_batch_run_graph": [C.c_void_p, C.c_void_p],
    "rt_batch_temperatures": [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p],
    "rt_mlp_create": [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_void_p)],
    "rt_mlp_destroy": [C.c_void_p],
    "rt_mlp_n_params": [C.c_void_p, C.POINTER(C.c_int64)],
    "rt_mlp_get_params": [C.c_void_p, C.c_void_p],
    "rt_mlp_set_params": [C.c_void_p, C.c_void_p],
    "rt_mlp_forward": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p],
    "rt_mlp_loss_grad": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                         C.c_void_p],
    "rt_mlp_adam_step": [C.c_void_p, C.c_float, C.c_void_p],
    "rt_set_pah": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_int,
                   C.c_int, C.c_double],
    "rt_pah_absorbed": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "rt_pah_temperature_distribution": [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                        C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p],
    "rt_set_pah_spectra": [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_int,
                           C.c_void_p],
    "rt_pah_emission": [C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_void_p,
                        C.c_float, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "rt_pah_emission_active": [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_float, C.c_int64,
                               C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int64),
                               C.c_void_p, C.c_void_p],
    "rt_pah_training_pairs": [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p],
    "rt_mlp_dims": [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "rt_mlp_set_range": [C.c_void_p, C.c_float, C.c_float],
    "rt_mlp_get_range": [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)],
    "rt_cell_temperatures_noalloc": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_double,
                                     C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                     C.c_void_p],
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librt_gb300.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"librt_gb300.so not found at {path}; run __graft_entry__.build()")
    L = C.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_char_p if name == "rt_status_string" else C.c_int
    _lib = L
    return L


def _check(code: int, where: str):
    if code != 0:
        raise RTError(code, where)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# element types a buffer may have for each kind of array the library reads or writes
# (torch has no unsigned 64- or 32-bit type in every version: the signed one of the
# same width stands in)
_KINDS = {"f32": ("float32",), "f64": ("float64",), "u64": ("uint64", "int64"),
          "u32": ("uint32", "int32"), "i32": ("int32",)}


def _torch_device():
    """The current CUDA device as torch sees it, or None when torch is not in use."""
    import sys
    torch = sys.modules.get("torch")
    if torch is None or not torch.cuda.is_available():
        return None
    return torch.cuda.current_device()


def _buf(x, kind: str, n: int, what: str, exact: bool = False, device=None):
    """(pointer, mem kind) of a numpy array or a torch tensor that the library will read
    or write as n elements of `kind`: checked to be contiguous, of that element type,
    at least (exact: exactly) n elements long and, for a CUDA tensor, on `device` when
    that is known. ValueError before anything is handed to the library otherwise."""
    if hasattr(x, "data_ptr"):  # torch tensor
        dtype = str(x.dtype).replace("torch.", "")
        numel, contiguous = int(x.numel()), bool(x.is_contiguous())
        if x.is_cuda and device is not None and x.device.index != device:
            raise ValueError(f"{what} is on cuda:{x.device.index}, the grid on cuda:{device}")
        ptr, mem = x.data_ptr(), (MEM_DEVICE if x.is_cuda else MEM_HOST)
    elif isinstance(x, np.ndarray):
        dtype, numel, contiguous = x.dtype.name, int(x.size), bool(x.flags.c_contiguous)
        ptr, mem = x.ctypes.data, MEM_HOST
    else:
        raise TypeError(f"{what} must be a numpy array or a torch tensor")
    if dtype not in _KINDS[kind]:
        raise ValueError(f"{what} has dtype {dtype}, not {' or '.join(_KINDS[kind])}")
    if not contiguous:
        raise ValueError(f"{what} must be contiguous")
    if numel < n or (exact and numel != n):
        raise ValueError(f"{what} holds {numel} elements, {'exactly ' if exact else ''}"
                         f"{n} needed")
    return ptr, mem


def _dev_buf(x, kind: str, n: int, what: str, exact: bool = False, device=None):
    """Device pointer of a CUDA tensor checked as in _buf (for calls that take device
    buffers only)."""
    ptr, mem = _buf(x, kind, n, what, exact=exact, device=device)
    if mem != MEM_DEVICE:
        raise ValueError(f"{what} must be a CUDA tensor")
    return ptr


class Grid:
    """One model on the device (handle to ``rt_grid``)."""

    def __init__(self, model, n_temp: int = 0, t_min: float = 0.0, t_max: float = 0.0,
                 pah_levels: int = 400, pah_t_top: float = 2500.0):
        L = load()
        t = model.tree
        self.model = model
        self.S, self.N, self.B = model.n_species, t.n_leaves, model.n_bins
        self.n_dir = model.n_sed_dirs
        base = np.ascontiguousarray(t.base, dtype=np.int32)
        child = np.ascontiguousarray(t.child, dtype=np.int32)
        rho = np.ascontiguousarray(model.rho, dtype=np.float64)
        nu = np.ascontiguousarray(model.nu_edges, dtype=np.float64)
        d = _Desc(half_size_cm=model.half_size, n_base=t.n_base, max_level=t.max_level,
                  n_blocks=t.n_blocks, n_leaves=t.n_leaves, base=base.ctypes.data,
                  child=child.ctypes.data if child.size else None, n_species=self.S,
                  n_bins=self.B, rho=rho.ctypes.data, nu_edges=nu.ctypes.data,
                  n_sed_dirs=self.n_dir, n_temp=n_temp, t_min=t_min, t_max=t_max)
        h = C.c_void_p()
        _check(L.rt_grid_create(C.byref(d), C.byref(h)), "rt_grid_create")
        self._h = h
        kabs, ksca, g = model.opacity_arrays()
        for s, sp in enumerate(model.species):
            ka = np.ascontiguousarray(kabs[s])
            ks = np.ascontiguousarray(ksca[s])
            gg = np.ascontiguousarray(g[s])
            _check(L.rt_set_dust(h, s, ka.ctypes.data, ks.ctypes.data, gg.ctypes.data,
                                 self.B, int(sp.is_pah), int(sp.n_carbon)), "rt_set_dust")
            if sp.is_pah:
                modes = np.ascontiguousarray(np.array(sp.modes, dtype=np.float64).ravel())
                _check(L.rt_set_pah(h, s, int(sp.n_carbon), int(sp.n_hydrogen),
                                    float(sp.mol_mass), modes.ctypes.data, len(sp.modes),
                                    pah_levels, float(pah_t_top)), "rt_set_pah")
        self.n_pah = sum(1 for sp in model.species if sp.is_pah)
        self.n_coarse = min(64, self.B)
        self.device = _torch_device()  # the device the grid lives on, when torch knows it

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            load().rt_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- set-up
    def emit_star(self, n_total: int, star=None):
        st = star if star is not None else self.model.star
        pos = (C.c_double * 3)(*st.pos_cm)
        beam = (C.c_double * 3)(*st.beam_dir)
        _check(load().rt_emit_star(self._h, st.T, st.L, pos, int(st.kind), beam, int(n_total)),
               "rt_emit_star")
        self.n_total = int(n_total)

    def set_frozen_temperatures(self, T, stream=None):
        if not hasattr(T, "data_ptr"):
            T = np.ascontiguousarray(T, dtype=np.float32).reshape(self.S, self.N)
        p, mem = _buf(T, "f32", self.S * self.N, "T", exact=True, device=self.device)
        _check(load().rt_set_frozen_temperatures(self._h, p, mem, _stream(stream)),
               "rt_set_frozen_temperatures")

    # -- work
    def transport(self, n_packages: int, seed: int = 0, first_id: int = 0,
                  mode: int = REEMIT_BW, kernel: int = KERNEL_POOL, max_events: int = 0,
                  blocks_per_sm: int = 0, threads: int = 0, refill_period: int = 0,
                  interaction_batch: int = 0, budget_s: float = 0.0, estimators: int = 0,
                  count_scale: int = 0, walk: int = WALK_AUTO, stream=None):
        o = _Opts(mode=mode, kernel=kernel, max_events=max_events, blocks_per_sm=blocks_per_sm,
                  threads=threads, refill_period=refill_period,
                  interaction_batch=interaction_batch, budget_s=budget_s,
                  estimators=estimators, count_scale=count_scale, walk=walk, reserved=0)
        _check(load().rt_transport(self._h, int(n_packages), int(seed), int(first_id),
                                   C.byref(o), _stream(stream)), "rt_transport")

    def reset(self, stream=None):
        _check(load().rt_reset(self._h, _stream(stream)), "rt_reset")

    def temperatures(self, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros((self.S, self.N), dtype=np.float32)
        p, mem = _buf(out, "f32", self.S * self.N, "out", device=self.device)
        _check(load().rt_cell_temperatures(self._h, p, mem, _stream(stream)),
               "rt_cell_temperatures")
        return out

    def temperatures_pathlength(self, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros((self.S, self.N), dtype=np.float32)
        p, mem = _buf(out, "f32", self.S * self.N, "out", device=self.device)
        _check(load().rt_cell_temperatures_pathlength(self._h, p, mem, _stream(stream)),
               "rt_cell_temperatures_pathlength")
        return out

    def pathlength(self, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros((self.S, self.N), dtype=np.float32)
        p, mem = _buf(out, "f32", self.S * self.N, "out", device=self.device)
        _check(load().rt_pathlength(self._h, p, mem, _stream(stream)), "rt_pathlength")
        return out

    def sed(self, out=None, stream=None):
        if out is None:
            out = np.zeros((2, self.n_dir, self.B), dtype=np.uint64)
        p, mem = _buf(out, "u64", 2 * self.n_dir * self.B, "out", device=self.device)
        eps = C.c_double()
        _check(load().rt_sed(self._h, p, mem, C.byref(eps), _stream(stream)), "rt_sed")
        return out, eps.value

    def counts(self, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros((self.S, self.N), dtype=np.uint64)
        p, mem = _buf(out, "u64", self.S * self.N, "out", device=self.device)
        _check(load().rt_counts(self._h, p, mem, _stream(stream)), "rt_counts")
        return out

    def set_counts(self, counts, stream=None):
        if not hasattr(counts, "data_ptr"):
            counts = np.ascontiguousarray(counts, dtype=np.uint64).reshape(self.S, self.N)
        p, mem = _buf(counts, "u64", self.S * self.N, "counts", exact=True, device=self.device)
        _check(load().rt_set_counts(self._h, p, mem, _stream(stream)), "rt_set_counts")

    def pah_absorbed(self, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros((self.n_pah, self.N, self.n_coarse), dtype=np.uint32)
        p, mem = _buf(out, "u32", self.n_pah * self.N * self.n_coarse, "out",
                      device=self.device)
        _check(load().rt_pah_absorbed(self._h, p, mem, _stream(stream)), "rt_pah_absorbed")
        return out

    def pah_emission(self, first: int = 0, n: Optional[int] = None, mode: int = PAH_EXACT,
                     surrogate=None, tol: float = 0.0, out=None, pah: int = -1, stream=None,
                     count_fallback: bool = True):
        n = self.N - first if n is None else n
        if out is None:
            out = np.zeros((n, self.B), dtype=np.float32)
        p, mem = _buf(out, "f32", int(n) * self.B, "out", device=self.device)
        nf = C.c_uint64()
        _check(load().rt_pah_emission(self._h, int(first), int(n), int(pah), int(mode),
                                      surrogate._h if surrogate is not None else None,
                                      float(tol), p, mem,
                                      C.byref(nf) if count_fallback else None,
                                      _stream(stream)), "rt_pah_emission")
        return out, int(nf.value)

    def pah_emission_active(self, mode: int = PAH_EXACT, surrogate=None, tol: float = 0.0,
                            cells=None, out=None, pah: int = -1, stream=None):
        """Emission rows of the PAH-active cells only: returns (cells [n], rows [n][B],
        n_fallback). `cells` (int32) and `out` (float32 [max][B]) are preallocated
        outputs, both host (numpy) or both device (torch); by default host arrays
        large enough for every cell."""
        if out is None:
            cells = np.zeros(self.N, dtype=np.int32)
            out = np.zeros((self.N, self.B), dtype=np.float32)
        if len(out.shape) != 2 or int(out.shape[1]) != self.B:
            raise ValueError(f"out must be [rows][{self.B}]")
        rows = int(out.shape[0])
        pc, mc = _buf(cells, "i32", rows, "cells", device=self.device)
        p, mem = _buf(out, "f32", rows * self.B, "out", exact=True, device=self.device)
        if mc != mem:
            raise ValueError("cells and out must both be host or both be device memory")
        na = C.c_int64()
        nf = C.c_uint64()
        _check(load().rt_pah_emission_active(self._h, int(pah), int(mode),
                                             surrogate._h if surrogate is not None else None,
                                             float(tol), int(out.shape[0]), pc, p, mem,
                                             C.byref(na), C.byref(nf), _stream(stream)),
               "rt_pah_emission_active")
        n = int(na.value)
        return cells[:n], out[:n], int(nf.value)

    def set_pah_spectra(self, pah: int, J, first: int = 0, stream=None):
        """Per-cell re-emission spectra of PAH `pah` for cells first .. first+len(J)-1
        (rows [n][B]); None removes the spectra of every PAH."""
        if J is None:
            _check(load().rt_set_pah_spectra(self._h, 0, 0, 0, None, MEM_HOST,
                                             _stream(stream)), "rt_set_pah_spectra")
            return
        if not hasattr(J, "data_ptr"):
            J = np.ascontiguousarray(J, dtype=np.float32).reshape(-1, self.B)
        p, mem = _buf(J, "f32", int(J.shape[0]) * self.B, "J", exact=True, device=self.device)
        _check(load().rt_set_pah_spectra(self._h, int(pah), int(first), int(J.shape[0]), p, mem,
                                         _stream(stream)), "rt_set_pah_spectra")

    def pah_training_pairs(self, pah: int, X, Y, p_abs, first: int = 0, stream=None):
        """Training pairs of PAH `pah` for cells first .. first+n-1 into CUDA tensors X
        [n][n_coarse+2], Y [n][B] and p_abs [n] (float32)."""
        n = int(X.shape[0])
        px = _dev_buf(X, "f32", n * (self.n_coarse + 2), "X", exact=True, device=self.device)
        py = _dev_buf(Y, "f32", n * self.B, "Y", exact=True, device=self.device)
        pa = _dev_buf(p_abs, "f32", n, "p_abs", exact=True, device=self.device)
        _check(load().rt_pah_training_pairs(self._h, int(pah), int(first), n, px, py, pa,
                                            _stream(stream)), "rt_pah_training_pairs")

    image_shape = (0, 0, 0)

    def set_images(self, obs_dir, plane_of_bin, nx: int, ny: int, half_width_cm: float,
                   tau_max: float = 0.0, event_capacity: int = 0):
        """Peel-off images toward `obs_dir`; plane_of_bin[b] = image plane of bin b or -1.
        None for plane_of_bin removes the images."""
        if plane_of_bin is None:
            _check(load().rt_set_images(self._h, None, None), "rt_set_images")
            self.n_planes = 0
            self.image_shape = (0, 0, 0)
            return
        pob = np.ascontiguousarray(plane_of_bin, dtype=np.int32)
        d = _ImageDesc(obs_dir=(C.c_double * 3)(*[float(x) for x in obs_dir]), nx=int(nx),
                       ny=int(ny), half_width_cm=float(half_width_cm), tau_max=float(tau_max),
                       event_capacity=int(event_capacity))
        _check(load().rt_set_images(self._h, C.byref(d), pob.ctypes.data), "rt_set_images")
        self.n_planes = int(pob.max()) + 1
        self.image_shape = (self.n_planes, int(ny), int(nx))

    def images(self, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros(self.image_shape, dtype=np.float64)
        p, mem = _buf(out, "f64", int(np.prod(self.image_shape)), "out", device=self.device)
        _check(load().rt_images(self._h, p, mem, _stream(stream)), "rt_images")
        return out

    def image_profile(self, plane_a: int, plane_b: int = -1, half_rows: int = 0, out=None,
                      stream=None) -> np.ndarray:
        if out is None:
            out = np.zeros(max(self.image_shape[2], 1), dtype=np.float64)
        p, mem = _buf(out, "f64", self.image_shape[2], "out", device=self.device)
        _check(load().rt_image_profile(self._h, int(plane_a), int(plane_b), int(half_rows), p,
                                       mem, _stream(stream)), "rt_image_profile")
        return out

    def counters(self) -> dict:
        c = _Counters()
        code = load().rt_get_counters(self._h, C.byref(c))
        out = {n: int(getattr(c, n)) for n, _ in _Counters._fields_}
        _check(code, "rt_get_counters")
        return out

    def trace(self, ids, seed: int = 0, max_events: int = 0) -> np.ndarray:
        idv = np.ascontiguousarray(ids, dtype=np.uint64)
        out = np.zeros((idv.shape[0], 9), dtype=np.int64)
        _check(load().rt_trace(self._h, idv.ctypes.data, idv.shape[0], int(seed),
                               int(max_events), out.ctypes.data), "rt_trace")
        return out

    def trace_events(self, ids, seed: int = 0, max_events: int = 0, max_out: int = 4096):
        """Event-level replay (frozen mode): for each id a structured array of its
        events (kind, species, leaf, bin, pos), and the total number of events."""
        idv = np.ascontiguousarray(ids, dtype=np.uint64)
        out = np.zeros((idv.shape[0], max_out), dtype=EVENT_DTYPE)
        n = np.zeros(idv.shape[0], dtype=np.int64)
        _check(load().rt_trace_events(self._h, idv.ctypes.data, idv.shape[0], int(seed),
                                      int(max_events), int(max_out), out.ctypes.data,
                                      n.ctypes.data), "rt_trace_events")
        return [out[i, :min(int(n[i]), max_out)].copy() for i in range(idv.shape[0])], n


def pah_temperature_distribution(cases, nu_edges, sigma, n_levels: int = 400,
                                 t_sub: float = 2500.0):
    """P(T) of PAHs in monochromatic fields. `cases`: dicts with modes ((n, theta),
    ...), h_nu (erg), rate (photons/s per molecule) and optionally t_top (K); sigma
    [n_cases][n_bins] cross sections per molecule. Returns P, T [n][n_levels],
    p_above [n] and the emission per bin [n][n_bins]."""
    n = len(cases)
    arr = (_PtCase * n)()
    for i, c in enumerate(cases):
        modes = list(c["modes"])
        for k, (cnt, th) in enumerate(modes):
            arr[i].modes[k][0] = float(cnt)
            arr[i].modes[k][1] = float(th)
        arr[i].n_groups = len(modes)
        arr[i].h_nu_erg = float(c["h_nu"])
        arr[i].rate = float(c["rate"])
        arr[i].t_top = float(c.get("t_top", 0.0))
    nu = np.ascontiguousarray(nu_edges, dtype=np.float64)
    B = nu.shape[0] - 1
    sig = np.ascontiguousarray(sigma, dtype=np.float64).reshape(n, B)
    P = np.zeros((n, n_levels))
    T = np.zeros((n, n_levels))
    a = np.zeros(n)
    em = np.zeros((n, B))
    _check(load().rt_pah_temperature_distribution(arr, n, nu.ctypes.data, B, sig.ctypes.data,
                                                  int(n_levels), float(t_sub), P.ctypes.data,
                                                  T.ctypes.data, a.ctypes.data, em.ctypes.data,
                                                  None), "rt_pah_temperature_distribution")
    return P, T, a, em


def philox(ids, event: int, block: int, seed: int) -> np.ndarray:
    idv = np.ascontiguousarray(ids, dtype=np.uint64)
    out = np.zeros((idv.shape[0], 4), dtype=np.uint32)
    _check(load().rt_philox(idv.ctypes.data, idv.shape[0], event, block, int(seed),
                            out.ctypes.data), "rt_philox")
    return out


class Batch:
    """Handle to ``rt_batch``: many grids transported in one persistent launch."""

    def __init__(self, grids, n_packages, seed: int = 0, mode: int = REEMIT_BW,
                 max_events: int = 0, blocks_per_sm: int = 0, refill_period: int = 0,
                 interaction_batch: int = 0, budget_s: float = 0.0, chunk: int = 0,
                 threads: int = 0):
        L = load()
        self.grids = list(grids)
        arr = (C.c_void_p * len(self.grids))(*[g._h.value for g in self.grids])
        npk = np.ascontiguousarray(n_packages, dtype=np.uint64)
        o = _Opts(mode=mode, kernel=KERNEL_POOL, max_events=max_events,
                  blocks_per_sm=blocks_per_sm, threads=threads, refill_period=refill_period,
                  interaction_batch=interaction_batch, budget_s=budget_s, estimators=0,
                  count_scale=0, walk=0, reserved=0)
        h = C.c_void_p()
        _check(L.rt_batch_create(C.cast(arr, C.c_void_p), len(self.grids), npk.ctypes.data,
                                 int(seed), C.byref(o), int(chunk), C.byref(h)),
               "rt_batch_create")
        self._h = h

    def run(self, reset: bool = True, temperatures: bool = True, stream=None):
        _check(load().rt_batch_run(self._h, int(reset), int(temperatures), _stream(stream)),
               "rt_batch_run")

    def run_graph(self, stream=None):
        _check(load().rt_batch_run_graph(self._h, _stream(stream)), "rt_batch_run_graph")

    def temperatures(self, model: int, out=None, stream=None):
        g = self.grids[model]
        if out is None:
            out = np.zeros((g.S, g.N), dtype=np.float32)
        p, mem = _buf(out, "f32", g.S * g.N, "out", device=g.device)
        _check(load().rt_batch_temperatures(self._h, int(model), p, mem, _stream(stream)),
               "rt_batch_temperatures")
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().rt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """Handle to ``rt_mlp`` (the surrogate network)."""

    def __init__(self, n_in: int, n_hidden: int = 256, n_layers: int = 3, n_out: int = 200,
                 seed: int = 0):
        L = load()
        h = C.c_void_p()
        _check(L.rt_mlp_create(n_in, n_hidden, n_layers, n_out, int(seed), C.byref(h)),
               "rt_mlp_create")
        self._h = h
        self.n_in, self.n_hidden, self.n_layers, self.n_out = n_in, n_hidden, n_layers, n_out
        self.device = _torch_device()  # the device the network lives on, when torch knows it
        n = C.c_int64()
        _check(L.rt_mlp_n_params(h, C.byref(n)), "rt_mlp_n_params")
        self.n_params = int(n.value)

    def close(self):
        if getattr(self, "_h", None):
            load().rt_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().rt_mlp_get_params(self._h, out.ctypes.data), "rt_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError(f"{p.size} parameters, the network has {self.n_params}")
        _check(load().rt_mlp_set_params(self._h, p.ctypes.data), "rt_mlp_set_params")

    def forward(self, x, y, stream=None):
        """y [M][n_out] = network(x [M][n_in]); CUDA float32 tensors."""
        M = int(x.shape[0])
        px = _dev_buf(x, "f32", M * self.n_in, "x", exact=True, device=self.device)
        py = _dev_buf(y, "f32", M * self.n_out, "y", device=self.device)
        _check(load().rt_mlp_forward(self._h, px, py, M, _stream(stream)), "rt_mlp_forward")
        return y

    def loss_grad(self, x, t, want_loss: bool = True, want_grad: bool = False, stream=None):
        loss = C.c_float()
        g = np.zeros(self.n_params, dtype=np.float32) if want_grad else None
        M = int(x.shape[0])
        px = _dev_buf(x, "f32", M * self.n_in, "x", exact=True, device=self.device)
        pt = _dev_buf(t, "f32", M * self.n_out, "t", exact=True, device=self.device)
        _check(load().rt_mlp_loss_grad(self._h, px, pt, M,
                                       C.byref(loss) if want_loss else None,
                                       g.ctypes.data if want_grad else None, _stream(stream)),
               "rt_mlp_loss_grad")
        return (loss.value if want_loss else None), g

    def set_range(self, lo: float, hi: float):
        _check(load().rt_mlp_set_range(self._h, float(lo), float(hi)), "rt_mlp_set_range")

    def adam_step(self, lr: float, stream=None):
        _check(load().rt_mlp_adam_step(self._h, float(lr), _stream(stream)), "rt_mlp_adam_step")


def cell_temperatures_noalloc(count, rho, volume, kabs, nu_edges, eps: float, T_out,
                              n_clamped=None, t_min: float = 0.0, t_max: float = 0.0,
                              n_temp: int = 0, stream=None):
    """Temperatures from caller-owned device tensors (counts uint64/int64 [S][N], rho
    float64 [S][N], volume float64 [N], kabs float64 [S][B], nu_edges float64 [B+1],
    T_out float32 [S][N], n_clamped int64/uint64 [1] or None); the library allocates
    nothing for this call (its table lives in a fixed device array). Every tensor
    must be contiguous and on the current CUDA device; ValueError otherwise, before
    anything is launched."""
    import torch
    if count.dim() != 2 or kabs.dim() != 2:
        raise ValueError("count must be [S][N] and kabs [S][B]")
    S, N = int(count.shape[0]), int(count.shape[1])
    B = int(kabs.shape[1])
    u64 = getattr(torch, "uint64", None)
    spec = (("count", count, (torch.int64,) + ((u64,) if u64 is not None else ()), (S, N)),
            ("rho", rho, (torch.float64,), (S, N)),
            ("volume", volume, (torch.float64,), (N,)),
            ("kabs", kabs, (torch.float64,), (S, B)),
            ("nu_edges", nu_edges, (torch.float64,), (B + 1,)),
            ("T_out", T_out, (torch.float32,), (S, N)))
    if n_clamped is not None:
        spec += (("n_clamped", n_clamped,
                  (torch.int64,) + ((u64,) if u64 is not None else ()), (1,)),)
    cur = torch.cuda.current_device()
    for name, t, dtypes, shape in spec:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                             f"cuda:{cur}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} must have dtype {' or '.join(map(str, dtypes))}, "
                             f"not {t.dtype}")
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, not {tuple(t.shape)}")
    _check(load().rt_cell_temperatures_noalloc(
        count.data_ptr(), rho.data_ptr(), volume.data_ptr(), kabs.data_ptr(),
        nu_edges.data_ptr(), S, N, B, float(eps), float(t_min), float(t_max), int(n_temp),
        T_out.data_ptr(), n_clamped.data_ptr() if n_clamped is not None else None,
        _stream(stream)), "rt_cell_temperatures_noalloc")
    return T_out


def status_string(code: int) -> str:
    return load().rt_status_string(code).decode()
