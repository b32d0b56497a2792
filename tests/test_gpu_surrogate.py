"""The learned part: the PAH emission surrogate trained on the GPU by the library's
own kernels on exact transient-heating solutions of one disk, then evaluated on another
(held-out) disk against the exact solution: accuracy, energy balance, the fallback
of flagged cells to the exact solution, and the time it saves."""
import numpy as np
import pytest

from paper_1201_3588_gb300 import rt, surrogate, workloads as w

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _timed(fn):
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    out = fn()
    b.record(s)
    torch.cuda.synchronize()
    return out, a.elapsed_time(b) / 1e3


def test_surrogate_learns_and_gains():
    N = 2 * 10 ** 7
    train_models = [w.disk_pah_model(n_base=64, max_level=1, n_bins=200, tau_v_mid=100.0,
                                     perturbed=True),
                    w.disk_pah_model(n_base=64, max_level=1, n_bins=200, tau_v_mid=1000.0,
                                     perturbed=False)]
    held_model = w.disk_pah_model(n_base=64, max_level=1, n_bins=200, tau_v_mid=300.0,
                                  perturbed=False)
    grids = [rt.Grid(m) for m in train_models]
    for i, g in enumerate(grids):
        g.emit_star(N)
        g.transport(N, seed=1 + i)
    (net, hist, n_pairs), t_train = _timed(lambda: surrogate.build(grids))
    for g in grids:
        g.close()
    print("training pairs", n_pairs, "epochs", len(hist), "first/last loss", hist[0], hist[-1],
          f"training time {t_train:.1f} s")
    assert n_pairs > 50_000 and hist[-1] < 0.2 * hist[0]

    with rt.Grid(held_model) as h:
        h.emit_star(N)
        h.transport(N, seed=2)
        dev = torch.device("cuda", 0)
        J_ex = torch.zeros((h.N, h.B), device=dev)
        J_sur = torch.zeros((h.N, h.B), device=dev)
        J_auto = torch.zeros((h.N, h.B), device=dev)
        _, t_ex = _timed(lambda: h.pah_emission(mode=rt.PAH_EXACT, out=J_ex, count_fallback=False))
        _, t_sur = _timed(lambda: h.pah_emission(mode=rt.PAH_SURROGATE, surrogate=net, out=J_sur,
                                                 count_fallback=False))
        (_, nf), t_auto = _timed(lambda: h.pah_emission(mode=rt.PAH_AUTO, surrogate=net,
                                                        tol=0.05, out=J_auto))
        tal = h.pah_absorbed()
        _, eps = h.sed()
    J_ex, J_sur, J_auto = (x.cpu().numpy().astype(np.float64) for x in (J_ex, J_sur, J_auto))
    has = tal.sum(axis=(0, 2)) > 0
    n_cells = int(has.sum())
    absorbed = (tal.astype(np.float64) * eps).sum(axis=(0, 2))
    # energy: the exact solution and the rescaled surrogate both emit what was absorbed
    np.testing.assert_allclose(J_ex[has].sum(axis=1), absorbed[has], rtol=2e-4)
    np.testing.assert_allclose(J_sur[has].sum(axis=1), absorbed[has], rtol=2e-4)
    err = np.abs(J_sur[has] - J_ex[has]).sum(axis=1) / J_ex[has].sum(axis=1)
    err_auto = np.abs(J_auto[has] - J_ex[has]).sum(axis=1) / J_ex[has].sum(axis=1)
    print(f"held-out cells {n_cells}: surrogate L1 error median {np.median(err):.4f} "
          f"p90 {np.quantile(err, 0.9):.4f}; auto median {np.median(err_auto):.4f} "
          f"p90 {np.quantile(err_auto, 0.9):.4f}; fallback {nf} ({nf / n_cells:.3f}); "
          f"time exact {t_ex * 1e3:.1f} ms, surrogate {t_sur * 1e3:.1f} ms, "
          f"auto {t_auto * 1e3:.1f} ms")
    # evaluated against the exact computation on held-out cells
    assert np.median(err) < 0.05 and np.quantile(err, 0.9) < 0.10
    assert np.quantile(err_auto, 0.9) <= np.quantile(err, 0.9) + 1e-6
    assert nf < 0.05 * n_cells
    # what it gains: surrogate plus fallback in well under the exact-only time
    assert t_sur < 0.5 * t_ex and t_auto < 0.5 * t_ex
