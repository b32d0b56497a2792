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
