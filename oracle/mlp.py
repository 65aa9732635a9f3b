"""Float64 reference of the capacity MLP (test infrastructure only).

Plain numpy: forward pass of ReLU layers, the pinball (quantile) loss and its
gradient by backpropagation written out layer by layer, and one Adam step
(Kingma & Ba, 2015). The GPU training kernels are checked against these; the
functions here are pinned by central finite differences and closed forms in
tests/test_oracle_mlp.py. Parameters use the library's flat layout: for each
linear map, W[din][dout] then b[dout].
"""
from __future__ import annotations

import numpy as np


def unflatten(flat, dims):
    """dims = [n_in, h, ..., n_out] -> list of (W, b) views (float64 copies)."""
    out, off = [], 0
    flat = np.asarray(flat, dtype=np.float64)
    for din, dout in zip(dims[:-1], dims[1:]):
        W = flat[off:off + din * dout].reshape(din, dout)
        off += din * dout
        b = flat[off:off + dout]
        off += dout
        out.append((W.copy(), b.copy()))
    assert off == flat.size
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def forward(layers, x):
    """Activations [x, h1, ..., y]; ReLU on every layer but the last."""
    acts = [np.asarray(x, dtype=np.float64)]
    for i, (W, b) in enumerate(layers):
        z = acts[-1] @ W + b
        acts.append(np.maximum(z, 0.0) if i < len(layers) - 1 else z)
    return acts


def pinball(yhat, y, tau):
    """Mean over all entries of max(tau e, (tau - 1) e), e = y - yhat; and d/dyhat."""
    e = np.asarray(y, np.float64) - yhat
    loss = np.where(e > 0, tau * e, (tau - 1.0) * e).mean()
    d = np.where(e > 0, -tau, 1.0 - tau) / e.size
    return loss, d


def loss_and_grads(layers, x, y, tau):
    acts = forward(layers, x)
    loss, d = pinball(acts[-1], y, tau)
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        gW = acts[i].T @ d
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        if i > 0:
            d = (d @ W.T) * (acts[i] > 0)
    grads.reverse()
    return loss, grads


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


NOMINAL = None  # the nominal parameter values are passed in by the caller


def features(table, nominal):
    """table[B][12] = side, n0 sheep, n0 wolves, 8 params, horizon."""
    t = np.asarray(table, dtype=np.int64)
    u = lambda a: np.asarray(a, np.int64) & 0xFFFFFFFF  # noqa: E731
    x = np.zeros((t.shape[0], 12), np.float64)
    x[:, 0] = np.log1p(t[:, 0])
    x[:, 1] = np.log1p(t[:, 1])
    x[:, 2] = np.log1p(t[:, 2])
    x[:, 3:11] = u(t[:, 3:11]) / u(np.asarray(nominal))[None, :]
    x[:, 11] = t[:, 11] / 500.0
    return x


def capacity(yhat, margin, round_to, cap_max, n0):
    """min(cap_max, roundup(ceil(exp(yhat) (1 + margin)), round_to)), >= n0 and >= round_to."""
    want = np.ceil(np.exp(np.asarray(yhat, np.float64)) * (1.0 + margin))
    c = np.maximum(np.minimum(want, 2**31 - 1).astype(np.int64), np.asarray(n0, np.int64))
    c = (c + round_to - 1) // round_to * round_to
    c = np.maximum(c, round_to)
    return np.minimum(c, np.asarray(cap_max, np.int64))
