"""Training of the PAH emission surrogate on the GPU through the library's own
kernels: training pairs from the exact transient-heating solution
(rt_pah_training_pairs), minibatch loss/gradient and Adam steps (rt_mlp_loss_grad,
rt_mlp_adam_step). PyTorch only holds the device buffers and shuffles row indices."""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from . import rt

N_HIDDEN = 256
N_LAYERS = 3


def training_pairs(grid: "rt.Grid", device="cuda", chunk: int = 1 << 18):
    """(X, Y) torch tensors of every (cell, PAH) with PAH absorptions in the grid."""
    import torch
    F = grid.n_coarse + 2
    xs, ys = [], []
    for p in range(grid.n_pah):
        for c0 in range(0, grid.N, chunk):
            n = min(chunk, grid.N - c0)
            X = torch.empty((n, F), dtype=torch.float32, device=device)
            Y = torch.empty((n, grid.B), dtype=torch.float32, device=device)
            pa = torch.empty(n, dtype=torch.float32, device=device)
            grid.pah_training_pairs(p, X, Y, pa, first=c0)
            keep = pa > 0
            xs.append(X[keep])
            ys.append(Y[keep])
    return torch.cat(xs), torch.cat(ys)


def train(net: "rt.MLP", X, Y, epochs: int = 40, batch: int = 1024, lr: float = 2e-3,
          seed: int = 0, lr_final: float = 2e-5) -> List[float]:
    """Adam on shuffled minibatches; learning rate decays geometrically to lr_final.
    Returns the loss of each epoch's last minibatch."""
    import torch
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    n = X.shape[0]
    steps = epochs * max(1, n // batch)
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    hist, k = [], 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g, device=X.device)
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = X[idx].contiguous()
            yb = Y[idx].contiguous()
            last = b0 + 2 * batch > n
            loss, _ = net.loss_grad(xb, yb, want_loss=last)
            net.adam_step(lr * decay ** k)
            k += 1
            if last:
                hist.append(loss)
    return hist


def build(grids: Sequence["rt.Grid"], epochs: int = 40, seed: int = 0, batch: int = 1024,
          lr: float = 2e-3, margin: float = 0.25):
    """A surrogate trained on the PAH cells of the given grids (after transport). The
    admissible range of the absorbed-power feature is the training range widened by
    `margin`."""
    import torch
    pairs = [training_pairs(g) for g in grids]
    X = torch.cat([p[0] for p in pairs])
    Y = torch.cat([p[1] for p in pairs])
    g0 = grids[0]
    net = rt.MLP(g0.n_coarse + 2, N_HIDDEN, N_LAYERS, g0.B, seed=seed)
    hist = train(net, X, Y, epochs=epochs, batch=batch, lr=lr, seed=seed)
    xp = X[:, -2]
    net.set_range(float(xp.min()) - margin, float(xp.max()) + margin)
    return net, hist, int(X.shape[0])
