"""The fused tensor-core forward pass (tcgen05.mma into tensor memory) of the
surrogate network: against the FP64 oracle within BF16 error, against the
layer-by-layer forward of the training path (tcgen05 GEMMs per layer on the same BF16
weights, so nearly identical), for ragged row counts, after the weights change, with an output layer
wider than one MMA (run in chunks of 256 columns), and with a hidden layer too wide
for it (the layer-by-layer path takes over)."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1201_3588_gb300 import rt

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _check_against_oracle(net, shapes, x, y):
    p = net.get_params().astype(np.float64)   # also reports a tensor-core wait timeout
    ref, _ = omlp.forward(p, shapes, x.astype(np.float64))
    got = y.cpu().numpy()
    scale = np.sqrt((ref ** 2).mean())
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() < 0.05 * scale
    assert np.sqrt(((got - ref) ** 2).mean()) < 0.01 * scale
    return got


@pytest.mark.parametrize("M", [1, 127, 128, 1000, 70_001])
def test_fused_forward_matches_oracle_and_layer_path(M):
    net = rt.MLP(66, 256, 3, 200, seed=7)
    shapes = omlp.layer_shapes(66, 256, 3, 200)
    rng = np.random.default_rng(M)
    x = rng.normal(size=(M, 66)).astype(np.float32)
    y = torch.full((M, 200), float("nan"), device="cuda")
    net.forward(_dev(x), y)
    torch.cuda.synchronize()
    got = _check_against_oracle(net, shapes, x, y)
    # the training path's layer-by-layer forward on the same weights: the loss of the
    # fused outputs as targets is their mean squared difference
    loss, _ = net.loss_grad(_dev(x), y.contiguous(), want_loss=True)
    assert loss < 1e-6 * float((got ** 2).mean()), loss


def test_fused_forward_follows_weight_updates():
    net = rt.MLP(16, 64, 2, 8, seed=5)
    shapes = omlp.layer_shapes(16, 64, 2, 8)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(512, 16)).astype(np.float32)
    t = rng.normal(size=(512, 8)).astype(np.float32)
    xd, td = _dev(x), _dev(t)
    y0 = torch.zeros((512, 8), device="cuda")
    net.forward(xd, y0)
    for _ in range(5):
        net.loss_grad(xd, td, want_loss=False)
        net.adam_step(1e-2)
    y1 = torch.zeros((512, 8), device="cuda")
    net.forward(xd, y1)
    torch.cuda.synchronize()
    assert not torch.equal(y0, y1)
    _check_against_oracle(net, shapes, x, y1)


@pytest.mark.parametrize("n_out,M", [(400, 1000), (400, 70_001), (258, 333), (514, 129)])
def test_wide_output_layer_in_chunks(n_out, M):
    # 400 bins (the large disk), and widths that leave a ragged last chunk (16 and 2
    # columns past a multiple of 256; 258 and 514 are not multiples of 4)
    net = rt.MLP(66, 256, 3, n_out, seed=11)
    shapes = omlp.layer_shapes(66, 256, 3, n_out)
    rng = np.random.default_rng(n_out + M)
    x = rng.normal(size=(M, 66)).astype(np.float32)
    y = torch.full((M, n_out), float("nan"), device="cuda")
    net.forward(_dev(x), y)
    torch.cuda.synchronize()
    got = _check_against_oracle(net, shapes, x, y)
    loss, _ = net.loss_grad(_dev(x), y.contiguous(), want_loss=True)
    assert loss < 1e-6 * float((got ** 2).mean()), loss


def test_too_wide_layers_use_the_layer_path():
    net = rt.MLP(40, 300, 2, 24, seed=9)   # 304 > 256: not one tensor-core MMA
    shapes = omlp.layer_shapes(40, 300, 2, 24)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(333, 40)).astype(np.float32)
    y = torch.zeros((333, 24), device="cuda")
    net.forward(_dev(x), y)
    torch.cuda.synchronize()
    _check_against_oracle(net, shapes, x, y)
