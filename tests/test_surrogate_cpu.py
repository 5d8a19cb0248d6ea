"""The FP64 reference MLP (oracle/mlp.py): gradients pinned by central finite
differences, and the bf16 rounding helper against torch."""
import numpy as np
import pytest

from oracle import mlp as omlp


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, hidden, n_layers = 8, 16, 3
    n = sum(a * b + b for a, b in omlp.layer_shapes(n_in, hidden, n_layers))
    params = rng.normal(size=n) * 0.3
    x = rng.normal(size=(12, n_in))
    y = rng.normal(size=12) * 0.2
    tau, lam = 0.5, 0.3
    _, g = omlp.loss_and_grad(params, x, y, tau, lam, n_in, hidden, n_layers)
    # the NLL term holds r fixed: compare against the finite difference of that
    # surrogate objective, with r frozen at the base point
    base_out, _, _ = omlp.forward(params, x, n_in, hidden, n_layers)
    r0 = y - base_out[:, 0]

    def objective(p):
        out, _, _ = omlp.forward(p, x, n_in, hidden, n_layers)
        mu, s = out[:, 0], np.clip(out[:, 1], -16, 4)
        r = y - mu
        return np.mean(r * r / tau ** 2 + lam * (0.5 * r0 * r0 * np.exp(-2 * s) + s))
    for idx in rng.choice(n, 25, replace=False):
        h = 1e-6
        e = np.zeros(n)
        e[idx] = h
        fd = (objective(params + e) - objective(params - e)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-7 + 1e-6 * abs(fd)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(1).normal(size=1000).astype(np.float32) * 100
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(omlp.bf16_round(x), ref)
