"""FP64 oracle of the warm-start network (test infrastructure only).

A dense MLP with ReLU hidden layers and a linear output layer; weights W_l
(out x in) and biases b_l per layer, as plain numpy float64.  Forward,
backward of the mean-squared-error loss, and one Adam step (Kingma and Ba,
with bias correction), each written out directly."""

import numpy as np


def forward(Ws, bs, x):
    """Outputs of every layer (hidden ones after the ReLU)."""
    acts = []
    h = np.asarray(x, dtype=np.float64)
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if l + 1 < len(Ws) else z
        acts.append(h)
    return acts


def mse(y, t):
    r = y - t
    return float(np.mean(r * r)), 2.0 * r / r.size


def backward(Ws, bs, x, acts, dy):
    """Gradients of a loss with dLoss/doutput = dy, by the chain rule layer
    by layer: gW_l = dZ_l^T h_{l-1}, gb_l = sum over the batch of dZ_l,
    dZ_{l-1} = (dZ_l W_l) * [h_{l-1} > 0]."""
    gWs, gbs = [None] * len(Ws), [None] * len(Ws)
    dz = np.asarray(dy, dtype=np.float64)
    for l in range(len(Ws) - 1, -1, -1):
        hin = np.asarray(x, dtype=np.float64) if l == 0 else acts[l - 1]
        gWs[l] = dz.T @ hin
        gbs[l] = dz.sum(axis=0)
        if l > 0:
            dz = (dz @ Ws[l]) * (acts[l - 1] > 0)
    return gWs, gbs


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
