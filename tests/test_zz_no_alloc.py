"""The allocation-free temperature entry point (rt_cell_temperatures_noalloc) gives
the same temperatures as rt_cell_temperatures, on two calls in a row with different
models, so that the second call cannot lean on what the first left in the shared
fixed-size device array.

Callers of that entry point are those that may not call cudaMalloc when they need
temperatures (memory handed out only by their own pool, or a fixed device-memory
budget); they pass every buffer themselves. This file is collected last so that a
failure here comes after every other test has run."""
import numpy as np
import pytest

from paper_1201_3588_gb300 import rt, workloads as w

pytestmark = pytest.mark.gpu


def _reference_and_inputs(model, n_packages, seed, t_max=0.0):
    with rt.Grid(model, t_max=t_max) as g:
        g.emit_star(n_packages)
        g.transport(n_packages, seed=seed)
        T_ref = g.temperatures()
        cnt = g.counts()
        _, eps = g.sed()
    clamped_ref = int(((T_ref == (t_max or 3000.0)) & (cnt > 0)).sum())
    d0 = 2 * model.half_size / model.tree.n_base
    vol = (d0 * np.ldexp(1.0, -model.tree.leaf_level.astype(np.int64))) ** 3
    kabs, _, _ = model.opacity_arrays()
    return T_ref, cnt, eps, vol, kabs, clamped_ref


def _noalloc(torch, model, cnt, eps, vol, kabs, t_max=0.0):
    dev = torch.device("cuda", 0)
    count = torch.from_numpy(cnt.view(np.int64)).to(dev)
    rho = torch.from_numpy(np.ascontiguousarray(model.rho)).to(dev)
    volume = torch.from_numpy(np.ascontiguousarray(vol)).to(dev)
    ka = torch.from_numpy(np.ascontiguousarray(kabs)).to(dev)
    nu = torch.from_numpy(np.ascontiguousarray(model.nu_edges)).to(dev)
    T = torch.full(tuple(cnt.shape), -1.0, dtype=torch.float32, device=dev)
    ncl = torch.full((1,), -7, dtype=torch.int64, device=dev)
    rt.cell_temperatures_noalloc(count, rho, volume, ka, nu, eps, T, ncl, t_max=t_max)
    torch.cuda.synchronize()
    return T.cpu().numpy(), int(ncl.item())


def test_noalloc_matches_cell_temperatures_twice():
    torch = pytest.importorskip("torch")
    sphere = w.sphere_model()
    nu = w.frequency_edges(100)
    sp = [w.powerlaw_species("sil", nu, 1.0e4, 0.5, 1.5),
          w.powerlaw_species("carb", nu, 2.0e4, 0.3, 1.0)]
    disk = w.disk_model(n_base=32, max_level=2, n_bins=100, tau_v_mid=50.0, species=sp)
    for model, n, seed in ((sphere, 10 ** 6, 1), (disk, 2 * 10 ** 6, 2)):
        T_ref, cnt, eps, vol, kabs, clamped_ref = _reference_and_inputs(model, n, seed)
        T, ncl = _noalloc(torch, model, cnt, eps, vol, kabs)
        pos = cnt > 0
        assert pos.sum() > 1000
        assert (T[~pos] == 0).all()
        np.testing.assert_allclose(T[pos], T_ref[pos], rtol=1e-5)
        assert ncl == clamped_ref


def test_noalloc_rejects_requests_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    S, N, B = 9, 4, 8
    cnt = torch.zeros((S, N), dtype=torch.int64, device=dev)
    rho = torch.ones((S, N), dtype=torch.float64, device=dev)
    vol = torch.ones(N, dtype=torch.float64, device=dev)
    ka = torch.ones((S, B), dtype=torch.float64, device=dev)
    nu = torch.linspace(1e12, 1e15, B + 1, dtype=torch.float64, device=dev)
    T = torch.zeros((S, N), dtype=torch.float32, device=dev)
    with pytest.raises(rt.RTError) as e:
        rt.cell_temperatures_noalloc(cnt, rho, vol, ka, nu, 1.0, T)
    assert e.value.code == 8
    with pytest.raises(rt.RTError) as e:
        rt.cell_temperatures_noalloc(cnt[:2], rho[:2], vol, ka[:2], nu, 1.0, T[:2],
                                     n_temp=4096)
    assert e.value.code == 8


def test_noalloc_clamps_and_restarts_its_counter():
    """With a low table top (30 K) many cells lie beyond it: both entry points set
    them to t_max and count them alike, and a second identical call reports the
    same count (the counter in the shared array starts from zero every call)."""
    torch = pytest.importorskip("torch")
    model = w.sphere_model()
    T_ref, cnt, eps, vol, kabs, clamped_ref = _reference_and_inputs(model, 10 ** 6, 3,
                                                                    t_max=30.0)
    assert clamped_ref > 100
    for _ in range(2):
        T, ncl = _noalloc(torch, model, cnt, eps, vol, kabs, t_max=30.0)
        pos = cnt > 0
        np.testing.assert_allclose(T[pos], T_ref[pos], rtol=1e-5)
        assert ncl == clamped_ref


def test_noalloc_binding_rejects_mismatched_tensors():
    """Wrong dtypes, shapes or devices are refused before anything is launched."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    S, N, B = 2, 16, 8
    ok = dict(count=torch.zeros((S, N), dtype=torch.int64, device=dev),
              rho=torch.ones((S, N), dtype=torch.float64, device=dev),
              volume=torch.ones(N, dtype=torch.float64, device=dev),
              kabs=torch.ones((S, B), dtype=torch.float64, device=dev),
              nu_edges=torch.linspace(1e12, 1e15, B + 1, dtype=torch.float64, device=dev),
              T_out=torch.zeros((S, N), dtype=torch.float32, device=dev))
    rt.cell_temperatures_noalloc(eps=1.0, **ok)
    torch.cuda.synchronize()
    bad = [("rho", ok["rho"].float()), ("count", ok["count"].int()),
           ("T_out", torch.zeros((S, N - 1), dtype=torch.float32, device=dev)),
           ("volume", torch.ones(N + 1, dtype=torch.float64, device=dev)),
           ("nu_edges", ok["nu_edges"][:B]),
           ("rho", ok["rho"].cpu()),
           ("rho", torch.ones((N, S), dtype=torch.float64, device=dev).t())]
    for name, t in bad:
        args = dict(ok)
        args[name] = t
        with pytest.raises(ValueError):
            rt.cell_temperatures_noalloc(eps=1.0, **args)
