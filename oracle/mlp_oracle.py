"""FP64 CPU oracle of the warm-start network (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU baseline use this module; the library
never calls it. It is the plain definition of the network the library trains, written layer by
layer with numpy products (no fusion, no blocking):

    y_0 = x;  z_l = y_{l-1} W_l^T + b_l;  y_l = tanh(z_l) for hidden layers, y_L = z_L,
    L(θ) = mean over batch and outputs of (y_L - t)^2,

its gradient by the chain rule, one Adam step (Kingma and Ba, "Adam: a method for stochastic
optimization", ICLR 2015: first and second moment estimates with bias correction), and the
round-to-nearest-even conversion of float32 to bfloat16 that the library applies to its weights.
Parameters are one flat array: for each layer W_l row-major [out][in], then b_l [out].
Pinned in tests by central finite differences of the loss, closed forms of special cases, and
the bfloat16 format's definition.
"""
from __future__ import annotations

import numpy as np


def layout(sizes):
    """[(w_offset, b_offset, in, out)] per layer and the total parameter count."""
    out, off = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        out.append((off, off + i * o, i, o))
        off += i * o + o
    return out, off


def unpack(params, sizes):
    lay, n = layout(sizes)
    p = np.asarray(params, np.float64)
    assert p.size == n
    return [(p[w:w + i * o].reshape(o, i), p[b:b + o]) for (w, b, i, o) in lay]


def forward(params, sizes, x):
    """Activations [y_0 = x, y_1, ..., y_L] in FP64."""
    ys = [np.asarray(x, np.float64)]
    layers = unpack(params, sizes)
    for k, (W, b) in enumerate(layers):
        z = ys[-1] @ W.T + b
        ys.append(np.tanh(z) if k + 1 < len(layers) else z)
    return ys


def loss_grad(params, sizes, x, t):
    """Mean squared error and its gradient with respect to every parameter (flat layout)."""
    layers = unpack(params, sizes)
    ys = forward(params, sizes, x)
    t = np.asarray(t, np.float64)
    n = t.size
    loss = float(np.sum((ys[-1] - t) ** 2) / n)
    lay, npar = layout(sizes)
    g = np.zeros(npar)
    G = 2.0 * (ys[-1] - t) / n                      # dL/dz_L (linear output)
    for k in range(len(layers) - 1, -1, -1):
        W, _ = layers[k]
        w, b, i, o = lay[k]
        g[w:w + i * o] = (G.T @ ys[k]).ravel()      # dL/dW_k
        g[b:b + o] = G.sum(axis=0)                  # dL/db_k
        if k > 0:
            G = (G @ W) * (1.0 - ys[k] ** 2)        # through tanh of layer k-1
    return loss, g


def adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; step is the 1-based index of this update. Returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grads
    v = beta2 * v + (1.0 - beta2) * grads ** 2
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """float32 -> nearest bfloat16 (ties to even), returned as float32 (finite inputs)."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def weights_bf16(params, sizes):
    """The parameters with every weight rounded to bfloat16 and the biases kept (float32)."""
    p = np.asarray(params, np.float32).copy()
    for (w, b, i, o) in layout(sizes)[0]:
        p[w:w + i * o] = bf16_round(p[w:w + i * o])
    return p
