"""Pin of the oracle's MLP gradients: central finite differences in FP64."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    shapes = mlp.layer_shapes(5, 7, 2, 3)
    n = sum(r * c + r for r, c in shapes)
    p = rng.normal(scale=0.5, size=n)
    x = rng.normal(size=(4, 5))
    t = rng.normal(size=(4, 3))
    loss, g = mlp.loss_and_grad(p, shapes, x, t)
    h = 1e-6
    fd = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (mlp.loss_and_grad(p + e, shapes, x, t)[0] -
                 mlp.loss_and_grad(p - e, shapes, x, t)[0]) / (2 * h)
    assert np.abs(fd - g).max() < 1e-7 * max(1.0, np.abs(g).max())
    # loss is the mean squared error of the forward pass
    y, _ = mlp.forward(p, shapes, x)
    assert loss == np.mean((y - t) ** 2)


def test_silu_and_its_derivative():
    z = np.array([-30.0, -1.0, 0.0, 1.0, 30.0])
    assert np.allclose(mlp.silu(z), z / (1 + np.exp(-z)))
    assert mlp.silu(np.array([0.0]))[0] == 0.0 and mlp.dsilu(np.array([0.0]))[0] == 0.5
    h = 1e-6
    assert np.allclose((mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), mlp.dsilu(z), atol=1e-8)
