"""Pins of the oracle MLP: central finite differences of the loss, and the
Adam step against its first-step closed form."""

import numpy as np

from oracle import mlp
from workloads.rng import normal


def _net(seed, dims):
    Ws, bs = [], []
    for l in range(len(dims) - 1):
        Ws.append(normal(seed + 2 * l, dims[l + 1] * dims[l]).reshape(dims[l + 1], dims[l]) * 0.5)
        bs.append(normal(seed + 2 * l + 1, dims[l + 1]) * 0.1)
    return Ws, bs


def test_mlp_gradient_matches_finite_differences():
    dims = [4, 7, 6, 3]
    Ws, bs = _net(10, dims)
    x = normal(50, 5 * 4).reshape(5, 4)
    t = normal(51, 5 * 3).reshape(5, 3)

    def loss(Ws_, bs_):
        return mlp.mse(mlp.forward(Ws_, bs_, x)[-1], t)[0]

    acts = mlp.forward(Ws, bs, x)
    _, dy = mlp.mse(acts[-1], t)
    gW, gb = mlp.backward(Ws, bs, x, acts, dy)
    h = 1e-6
    for l in range(3):
        for (i, j) in [(0, 0), (1, 2), (2, 1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (loss(Wp, bs) - loss(Wm, bs)) / (2 * h)
            assert abs(fd - gW[l][i, j]) <= 1e-7 * max(1.0, abs(fd))
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][1] += h
        bm[l][1] -= h
        fd = (loss(Ws, bp) - loss(Ws, bm)) / (2 * h)
        assert abs(fd - gb[l][1]) <= 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_is_signed_lr():
    """With zero moments, the bias-corrected first step is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, -0.01 * np.sign(g), atol=1e-15)
