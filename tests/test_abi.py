"""The C-ABI library loads and exports every entry point include/rt.h declares, and
its host-side validation rejects malformed input -- all without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1201_3588_gb300 import rt, workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = rt.load()
    names = _declared()
    assert "rt_transport" in names and "rt_grid_create" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(rt.SIGNATURES)


def test_status_strings():
    for code, text in rt.STATUS.items():
        assert rt.status_string(code) == text


def _desc(tree, rho, nu, S=1):
    base = np.ascontiguousarray(tree.base, dtype=np.int32)
    child = np.ascontiguousarray(tree.child, dtype=np.int32)
    keep = (base, child, rho, nu)
    d = rt._Desc(half_size_cm=w.AU, n_base=tree.n_base, max_level=tree.max_level,
                 n_blocks=tree.n_blocks, n_leaves=tree.n_leaves, base=base.ctypes.data,
                 child=child.ctypes.data if child.size else None, n_species=S,
                 n_bins=nu.shape[0] - 1, rho=rho.ctypes.data, nu_edges=nu.ctypes.data,
                 n_sed_dirs=1, n_temp=0, t_min=0.0, t_max=0.0)
    return d, keep


def _create(d):
    h = C.c_void_p()
    return rt.load().rt_grid_create(C.byref(d), C.byref(h))


@pytest.mark.gpu
def test_malformed_trees_are_rejected():
    """The tree is walked on the device: a malformed one is rejected before use."""
    t = w.build_tree(2, 1, lambda l, lo, hi: (lo == 0).all(axis=1))
    nu = w.frequency_edges(4)
    rho = np.ones(t.n_leaves)
    # a leaf id used twice
    bad = w.Tree(t.n_base, t.max_level, t.base.copy(), t.child.copy(), t.leaf_level, t.leaf_ijk)
    bad.child[3] = bad.child[2]
    d, keep = _desc(bad, rho, nu)
    assert _create(d) == 1
    # a leaf id out of range
    bad = w.Tree(t.n_base, t.max_level, t.base.copy(), t.child.copy(), t.leaf_level, t.leaf_ijk)
    bad.base[5] = t.n_leaves + 3
    d, keep = _desc(bad, rho, nu)
    assert _create(d) == 1
    # deeper than max_level
    bad = w.Tree(t.n_base, 0, t.base.copy(), t.child.copy(), t.leaf_level, t.leaf_ijk)
    d, keep = _desc(bad, rho, nu)
    assert _create(d) == 1
    # a block referenced twice (cycle-free but shared)
    bad = w.Tree(t.n_base, t.max_level, t.base.copy(), t.child.copy(), t.leaf_level, t.leaf_ijk)
    bad.base[1] = bad.base[0]
    d, keep = _desc(bad, rho, nu)
    assert _create(d) == 1


@pytest.mark.parametrize("what", [
    "nu_order", "species", "bins",
    pytest.param("rho_nan", marks=pytest.mark.gpu),   # densities are checked on the device
    pytest.param("rho_neg", marks=pytest.mark.gpu)])
def test_bad_descriptors_are_rejected(what):
    t = w.build_tree(2, 0)
    nu = w.frequency_edges(4)
    rho = np.ones(t.n_leaves)
    S = 1
    if what == "nu_order":
        nu = nu[::-1].copy()
    elif what == "rho_nan":
        rho[3] = np.nan
    elif what == "rho_neg":
        rho[2] = -1.0
    elif what == "species":
        S = 9
        rho = np.ones(9 * t.n_leaves)
    elif what == "bins":
        nu = np.logspace(8, 16, 1026)
    d, keep = _desc(t, rho, nu, S)
    assert _create(d) == 1


def test_null_arguments():
    L = rt.load()
    assert L.rt_grid_create(None, None) == 1
    assert L.rt_transport(None, 1, 0, 0, None, None) == 1
    assert L.rt_grid_destroy(None) == 0
    assert L.rt_philox(None, -1, 0, 0, 0, None) == 1
