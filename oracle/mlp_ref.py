"""Reference of the dispatch cost model's MLP in float64 -- TEST INFRASTRUCTURE ONLY.

Same network, loss and parameter layout as the library's CUDA kernels: features
(5) -> 32 ReLU -> 32 ReLU -> 12 linear outputs; loss = sum of mask * (y - t)^2
over the sum of the mask; parameters W1 [32x5], b1, W2 [32x32], b2, W3 [12x32],
b3 in one flat array.  The gradient is derived by hand (reverse-mode chain
rule) and is itself checked against central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 5, 32, 12
SHAPES = [(H, IN), (H,), (H, H), (H,), (OUT, H), (OUT,)]


def n_params() -> int:
    return int(sum(np.prod(s) for s in SHAPES))


def unpack(p: np.ndarray):
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(p[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def forward(p, x):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    y = h2 @ W3.T + b3
    return y, (x, h1, h2)


def loss_and_grad(p, x, t, mask):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    y, (x, h1, h2) = forward(p, x)
    t = np.asarray(t, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)
    cnt = m.sum()
    loss = float((m * (y - t) ** 2).sum() / cnt)
    d3 = 2.0 * m * (y - t) / cnt               # dL/dy
    gW3 = d3.T @ h2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * (h2 > 0)                  # through ReLU of layer 2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (h1 > 0)
    gW1 = d1.T @ x
    gb1 = d1.sum(axis=0)
    g = np.concatenate([a.reshape(-1) for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g


def loss_only(p, x, t, mask) -> float:
    y, _ = forward(p, x)
    m = np.asarray(mask, dtype=np.float64)
    return float((m * (y - np.asarray(t, dtype=np.float64)) ** 2).sum() / m.sum())
