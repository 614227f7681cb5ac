"""Pins of the learned-proposal oracle (oracle/learned.py): bfloat16 rounding against
torch's conversion, the gradients against central finite differences in float64, and
AdamW against its closed form for one scalar."""
from __future__ import annotations

import numpy as np
import torch

from oracle import learned as ln


def random_params(rng, scale=0.2):
    return {name: (rng.standard_normal(shape) * scale).astype(np.float64) for name, shape in ln.PARAM_SHAPES}


def test_bf16_matches_torch():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 10.0 ** rng.integers(-8, 8, 10000),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -1 - 2 ** -8, 0.0, -0.0], np.float32)])
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ln.bf16(a), want)


def test_param_count():
    assert ln.param_count() == 64 * 16 * 7 + 64 + 2 * (64 * 64 * 7 + 64) + 64 * 64 + 64 + 65 + 65


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    net = ln.Net(bf16_mode=False)
    p = random_params(rng)
    n, B = 11, 3
    xs = [rng.standard_normal((ln.CIN, n)) * (np.arange(ln.CIN) < 3)[:, None] for _ in range(B)]
    targets = rng.integers(0, n, B)
    ys = rng.standard_normal(B)
    wfs = np.array([1.0, 0.5, 0.0])
    loss, g = net.batch_loss_and_grads(p, xs, targets, ys, wfs)
    flat = ln.flatten(p)
    gflat = ln.flatten(g)
    h = 1e-6
    idx = np.concatenate([np.arange(0, flat.size, 97), np.arange(flat.size - 200, flat.size)])
    num = np.empty(idx.size)
    for j, k in enumerate(idx):
        f = flat.copy()
        f[k] += h
        lp, _ = net.batch_loss_and_grads(ln.unflatten(f), xs, targets, ys, wfs)
        f[k] -= 2 * h
        lm, _ = net.batch_loss_and_grads(ln.unflatten(f), xs, targets, ys, wfs)
        num[j] = (lp - lm) / (2 * h)
    err = np.abs(num - gflat[idx])
    assert err.max() < 1e-6 * max(1.0, np.abs(num).max()), err.max()


def test_adamw_scalar_closed_form():
    p = {name: np.ones(shape, np.float32) for name, shape in ln.PARAM_SHAPES}
    g = {name: np.full(shape, 0.5, np.float32) for name, shape in ln.PARAM_SHAPES}
    m = {name: np.zeros(shape, np.float32) for name, shape in ln.PARAM_SHAPES}
    v = {name: np.zeros(shape, np.float32) for name, shape in ln.PARAM_SHAPES}
    out = ln.adamw(p, g, m, v, 1, lr=1e-3, wd=0.01)
    # first step: m_hat = g, v_hat = g^2, update = lr (sign(g) + wd p) for weights
    assert np.allclose(out["W2"], 1 - 1e-3 * (0.5 / (0.5 + 1e-8) + 0.01), rtol=0, atol=1e-7)
    assert np.allclose(out["b2"], 1 - 1e-3 * (0.5 / (0.5 + 1e-8)), rtol=0, atol=1e-7)


def test_bf16_forward_close_to_float64():
    rng = np.random.default_rng(2)
    p = random_params(rng, scale=0.1)
    x = rng.standard_normal((ln.CIN, 64)) * (np.arange(ln.CIN) < 3)[:, None]
    a = ln.Net(True).forward({k: v.astype(np.float32) for k, v in p.items()}, x.astype(np.float32))
    b = ln.Net(False).forward(p, x)
    rel = np.linalg.norm(a["score"] - b["score"]) / np.linalg.norm(b["score"])
    assert rel < 3e-2
