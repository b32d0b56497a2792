"""The binding's buffer checks (no GPU): every array the library will read or write
is checked for its element type, contiguity and length before the call, so that a
wrong buffer raises ValueError instead of being overrun or misread."""
import numpy as np
import pytest

from paper_1201_3588_gb300 import rt


def test_matching_buffers_pass():
    a = np.zeros((3, 5), dtype=np.float32)
    p, mem = rt._buf(a, "f32", 15, "a", exact=True)
    assert p == a.ctypes.data and mem == rt.MEM_HOST
    assert rt._buf(np.zeros(20, np.float32), "f32", 15, "a")[1] == rt.MEM_HOST  # longer output
    for dt in (np.uint64, np.int64):
        rt._buf(np.zeros(4, dt), "u64", 4, "c", exact=True)
    for dt in (np.uint32, np.int32):
        rt._buf(np.zeros(4, dt), "u32", 4, "t")


@pytest.mark.parametrize("arr,kind,n,exact", [
    (np.zeros(15, np.float64), "f32", 15, False),        # FP64 where FP32 is written
    (np.zeros(15, np.float32), "f64", 15, False),
    (np.zeros(15, np.int32), "u64", 15, False),         # 4-byte counts where 8 are written
    (np.zeros(14, np.float32), "f32", 15, False),       # too short: would be overrun
    (np.zeros(16, np.float32), "f32", 15, True),        # an input of the wrong length
    (np.zeros((5, 6), np.float32)[:, :3], "f32", 15, False),  # not contiguous
])
def test_wrong_buffers_raise(arr, kind, n, exact):
    with pytest.raises(ValueError):
        rt._buf(arr, kind, n, "x", exact=exact)


def test_other_objects_raise():
    with pytest.raises(TypeError):
        rt._buf([0.0] * 15, "f32", 15, "x")


def test_torch_host_tensors():
    torch = pytest.importorskip("torch")
    t = torch.zeros((2, 8), dtype=torch.int64)
    p, mem = rt._buf(t, "u64", 16, "counts", exact=True)
    assert p == t.data_ptr() and mem == rt.MEM_HOST
    with pytest.raises(ValueError):
        rt._buf(torch.zeros(16, dtype=torch.float64), "f32", 16, "T")
    with pytest.raises(ValueError):
        rt._buf(torch.zeros((8, 4))[:, :2], "f32", 16, "T")


class _NoLibrary:
    """Stands in for the library: any call reaching it fails the test."""

    def __getattr__(self, name):
        raise AssertionError(f"{name} was called with a buffer the binding should reject")


@pytest.fixture
def fake_grid(monkeypatch):
    """A Grid of 2 species, 10 cells, 4 bins, one PAH and one escape direction, with no
    library behind it: only the checks before each call can run."""
    g = object.__new__(rt.Grid)
    g.S, g.N, g.B, g.n_dir, g.n_pah, g.n_coarse, g.device = 2, 10, 4, 1, 1, 4, None
    g.image_shape = (2, 3, 5)
    g._h = None
    monkeypatch.setattr(rt, "load", lambda *a, **k: _NoLibrary())
    return g


@pytest.mark.parametrize("call", [
    lambda g: g.temperatures(out=np.zeros((2, 10), np.float64)),
    lambda g: g.temperatures(out=np.zeros((2, 9), np.float32)),
    lambda g: g.temperatures_pathlength(out=np.zeros(19, np.float32)),
    lambda g: g.pathlength(out=np.zeros((10, 2), np.float32).T),
    lambda g: g.sed(out=np.zeros((2, 1, 3), np.uint64)),
    lambda g: g.counts(out=np.zeros((2, 10), np.uint32)),
    lambda g: g.pah_absorbed(out=np.zeros((1, 10, 3), np.uint32)),
    lambda g: g.pah_emission(first=2, n=5, out=np.zeros((4, 4), np.float32)),
    lambda g: g.pah_emission_active(cells=np.zeros(6, np.int32), out=np.zeros((6, 3), np.float32)),
    lambda g: g.pah_emission_active(cells=np.zeros(5, np.int32), out=np.zeros((6, 4), np.float32)),
    lambda g: g.pah_emission_active(cells=np.zeros(6, np.int64), out=np.zeros((6, 4), np.float32)),
    lambda g: g.images(out=np.zeros((2, 3, 4), np.float64)),
    lambda g: g.image_profile(0, out=np.zeros(4, np.float64)),
])
def test_grid_methods_reject_wrong_outputs(fake_grid, call):
    with pytest.raises(ValueError):
        call(fake_grid)


def test_grid_inputs_must_have_the_exact_length(fake_grid):
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        fake_grid.set_counts(torch.zeros(21, dtype=torch.int64))
    with pytest.raises(ValueError):
        fake_grid.set_frozen_temperatures(torch.zeros(19, dtype=torch.float32))
    with pytest.raises(ValueError):
        fake_grid.set_pah_spectra(0, torch.zeros((3, 5), dtype=torch.float32))


def test_device_only_calls_reject_host_and_misshapen_buffers(fake_grid, monkeypatch):
    torch = pytest.importorskip("torch")
    net = object.__new__(rt.MLP)
    net.n_in, net.n_out, net.n_params, net.device, net._h = 6, 4, 10, None, None
    x, y = torch.zeros((3, 6)), torch.zeros((3, 4))
    with pytest.raises(ValueError):           # host tensors where device buffers are read
        net.forward(x, y)
    with pytest.raises(ValueError):
        net.loss_grad(np.zeros((3, 6), np.float32), y)
    with pytest.raises(ValueError):
        fake_grid.pah_training_pairs(0, torch.zeros((5, 6)), torch.zeros((5, 4)),
                                     torch.zeros(5))
    with pytest.raises(ValueError):
        net.set_params(np.zeros(9, np.float32))
