"""FP64 NumPy reference of the surrogate network -- TEST INFRASTRUCTURE.

Plain forward and backward of the MLP n_in -> [hidden, SiLU] x n_layers -> 2
with the library's parameter layout (per linear layer: W [in][out] row-major,
then b [out]) and loss

    L = mean_b ((y - mu)/tau)^2 + lam (r^2 exp(-2 s)/2 + s),  r = y - mu,

where r is held constant in the second term and s is clamped to [-16, 4]
(the gradient of a clamped s is zero outside).  Gradients by the chain rule,
written out layer by layer; pinned by finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(n_in, hidden, n_layers, n_out=2):
    dims = [n_in] + [hidden] * n_layers + [n_out]
    return [(dims[i], dims[i + 1]) for i in range(n_layers + 1)]


def unpack(params, n_in, hidden, n_layers):
    out, o = [], 0
    for a, b in layer_shapes(n_in, hidden, n_layers):
        W = params[o:o + a * b].reshape(a, b)
        o += a * b
        bb = params[o:o + b]
        o += b
        out.append((W, bb))
    assert o == params.size
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, n_in, hidden, n_layers):
    layers = unpack(np.asarray(params, np.float64), n_in, hidden, n_layers)
    h = np.asarray(x, np.float64)
    zs, hs = [], [h]
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        if li < n_layers:
            zs.append(z)
            h = silu(z)
            hs.append(h)
        else:
            h = z
    return h, zs, hs


def loss_and_grad(params, x, y, tau, lam, n_in, hidden, n_layers):
    params = np.asarray(params, np.float64)
    y = np.asarray(y, np.float64)
    out, zs, hs = forward(params, x, n_in, hidden, n_layers)
    B = out.shape[0]
    mu, s_raw = out[:, 0], out[:, 1]
    s = np.clip(s_raw, -16.0, 4.0)
    r = y - mu
    e2 = np.exp(-2.0 * s)
    loss = np.mean(r * r / tau ** 2 + lam * (0.5 * r * r * e2 + s))
    dout = np.zeros_like(out)
    dout[:, 0] = -2.0 * r / tau ** 2 / B
    ds = lam * (1.0 - r * r * e2) / B
    dout[:, 1] = np.where((s_raw >= -16.0) & (s_raw <= 4.0), ds, 0.0)
    layers = unpack(params, n_in, hidden, n_layers)
    grads = []
    dz = dout
    for li in range(n_layers, -1, -1):
        W, _ = layers[li]
        hin = hs[li]
        grads.append((hin.T @ dz, dz.sum(axis=0)))
        if li > 0:
            dz = (dz @ W.T) * dsilu(zs[li - 1])
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in reversed(grads)])
    return loss, g


def bf16_round(a):
    """Round FP32 values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, np.float32).copy()
    u = f.view(np.uint32)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)
