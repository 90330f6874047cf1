"""Cost-model oracle: the FP64 forward pass, loss and analytic gradient of the
small fully connected network the library trains (TEST INFRASTRUCTURE ONLY).

Parameter layout (flat vector): for every layer, the weights W[out][in]
row-major, then the biases b[out].  Hidden layers use ReLU, the last layer is
linear with one output.  Loss: 0.5 * mean_n (y_n - t_n)^2.

Pinned by central differences in tests/test_oracle_pins.py (the analytic
gradient against numerical differentiation of the loss).
"""
import numpy as np


def layer_sizes(nin, hidden, nlayers):
    return [nin] + [hidden] * nlayers + [1]


def unpack(params, sizes):
    params = np.asarray(params, dtype=np.float64)
    Ws, bs, off = [], [], 0
    for i in range(len(sizes) - 1):
        ni, no = sizes[i], sizes[i + 1]
        Ws.append(params[off:off + no * ni].reshape(no, ni))
        off += no * ni
        bs.append(params[off:off + no])
        off += no
    assert off == params.size
    return Ws, bs


def forward(params, sizes, X):
    """Network output for every row of X (FP64)."""
    Ws, bs = unpack(params, sizes)
    a = np.asarray(X, dtype=np.float64)
    for i, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W.T + b
        a = np.maximum(z, 0.0) if i < len(Ws) - 1 else z
    return a[:, 0]


def loss(params, sizes, X, T):
    e = forward(params, sizes, X) - np.asarray(T, dtype=np.float64)
    return 0.5 * np.mean(e * e)


def loss_and_grad(params, sizes, X, T):
    """Loss and its gradient with respect to the flat parameter vector, by the
    chain rule written out layer by layer (FP64)."""
    Ws, bs = unpack(params, sizes)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    acts, pres = [X], []
    a = X
    for i, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W.T + b
        pres.append(z)
        a = np.maximum(z, 0.0) if i < len(Ws) - 1 else z
        acts.append(a)
    e = acts[-1][:, 0] - T
    L = 0.5 * np.mean(e * e)
    d = (e / n)[:, None]                 # dL/dz of the output layer
    grads_W, grads_b = [None] * len(Ws), [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        grads_W[i] = d.T @ acts[i]
        grads_b[i] = d.sum(axis=0)
        if i > 0:
            d = (d @ Ws[i]) * (pres[i - 1] > 0)
    g = []
    for gw, gb in zip(grads_W, grads_b):
        g.append(gw.reshape(-1))
        g.append(gb)
    return L, np.concatenate(g)


def adam_step(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba) in FP64; returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
