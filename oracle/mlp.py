"""FP64 reference of the warm-start network (oracle; test infrastructure only).

The paper has no learned component; this module is the plain definition of
the network the library trains, used to check the library's gradients:

    a_0 = x;  a_{l+1} = tanh(W_l a_l + b_l) for hidden layers,
    y = W_L a_L + b_L;  loss = mean over batch and outputs of (y - t)^2.

Flat parameter layout (shared with the C ABI): for each layer l, W_l
(d_{l+1} x d_l, row-major) then b_l (d_{l+1}).  Gradients by the chain rule,
written out layer by layer.

Adam (Kingma & Ba, "Adam: a method for stochastic optimization", 2015,
Algorithm 1) is written out as that paper defines it, with bias-corrected
moments.

Pins: tests/test_oracle_mlp.py (central finite differences of the loss, a
one-layer closed form, the first Adam step's closed form lr * sign(g)).
The quality of the learned guess itself: parity unpinned (the paper has no
counterpart; the guess is measured against the zero initial guess).
"""
from __future__ import annotations

import numpy as np


def layer_dims(in_dim, width, hidden, out_dim):
    return [in_dim] + [width] * hidden + [out_dim]


def unpack(p, dims):
    """Views (W_l, b_l) of the flat parameter vector."""
    out, off = [], 0
    for l in range(len(dims) - 1):
        nw = dims[l + 1] * dims[l]
        W = p[off:off + nw].reshape(dims[l + 1], dims[l])
        off += nw
        b = p[off:off + dims[l + 1]]
        off += dims[l + 1]
        out.append((W, b))
    assert off == p.size
    return out


def forward(p, dims, X):
    acts = [np.asarray(X, dtype=np.float64)]
    layers = unpack(np.asarray(p, dtype=np.float64), dims)
    for l, (W, b) in enumerate(layers):
        z = acts[-1] @ W.T + b
        acts.append(np.tanh(z) if l < len(layers) - 1 else z)
    return acts


def loss_and_grad(p, dims, X, T):
    p = np.asarray(p, dtype=np.float64)
    layers = unpack(p, dims)
    acts = forward(p, dims, X)
    Y = acts[-1]
    T = np.asarray(T, dtype=np.float64)
    cnt = Y.size
    loss = np.sum((Y - T) ** 2) / cnt
    grads = []
    dz = 2.0 * (Y - T) / cnt
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gW = dz.T @ acts[l]
        gb = dz.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            da = dz @ W
            dz = da * (1.0 - acts[l] ** 2)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(p, g, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); `step` counts from 1.
    Returns the new (p, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    mhat = m1 / (1.0 - beta1 ** step)
    vhat = m2 / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m1, m2
