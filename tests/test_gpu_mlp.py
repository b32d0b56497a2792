"""The surrogate network's tensor-core kernels against the FP64 oracle: forward
outputs within BF16 error, loss and gradients on the same weights and batch
(cosine > 0.999, relative L2 < 2e-2), and Adam training that lowers the loss."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1201_3588_gb300 import rt

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def net():
    return rt.MLP(66, 256, 3, 200, seed=3)


def test_forward_matches_oracle(net):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1000, 66)).astype(np.float32)
    y = torch.zeros((1000, 200), device="cuda")
    net.forward(_dev(x), y)
    torch.cuda.synchronize()
    p = net.get_params().astype(np.float64)
    shapes = omlp.layer_shapes(66, 256, 3, 200)
    ref, _ = omlp.forward(p, shapes, x.astype(np.float64))
    got = y.cpu().numpy()
    scale = np.sqrt((ref ** 2).mean())
    assert np.abs(got - ref).max() < 0.05 * scale
    assert np.sqrt(((got - ref) ** 2).mean()) < 0.01 * scale


@pytest.mark.parametrize("M", [64, 1000, 4099])
def test_gradients_match_oracle(net, M):
    rng = np.random.default_rng(M)
    x = rng.normal(size=(M, 66)).astype(np.float32)
    t = rng.normal(size=(M, 200)).astype(np.float32)
    loss, g = net.loss_grad(_dev(x), _dev(t), want_loss=True, want_grad=True)
    p = net.get_params().astype(np.float64)
    shapes = omlp.layer_shapes(66, 256, 3, 200)
    ref_loss, ref = omlp.loss_and_grad(p, shapes, x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=2e-2)
    cos = float(g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref)))
    rel = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
    assert cos > 0.999 and rel < 2e-2, (cos, rel)


def test_adam_training_reduces_loss():
    rng = np.random.default_rng(1)
    net = rt.MLP(16, 64, 2, 8, seed=5)
    A = rng.normal(size=(16, 8))
    x = rng.normal(size=(4096, 16)).astype(np.float32)
    t = np.sin(x @ A / 4.0).astype(np.float32)
    xd, td = _dev(x), _dev(t)
    first, _ = net.loss_grad(xd, td)
    for _ in range(300):
        net.loss_grad(xd, td, want_loss=False)
        net.adam_step(2e-3)
    last, _ = net.loss_grad(xd, td)
    assert last < 0.1 * first, (first, last)
    net.close()
