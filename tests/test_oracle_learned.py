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


# ---------------------------------------------------------------------------------
# Independent statement of the network in float64 torch (library convolutions,
# linear maps, mean pooling, softmax cross-entropy and autograd), compared element by
# element with the oracle's hand-written numpy forward, loss and backward.

def torch_net(p: dict, x: np.ndarray):
    """Scores [n], restart score and the parameter tensors (requires_grad) for one
    state x [CIN, n], stated with torch.nn.functional in float64."""
    F = torch.nn.functional
    t = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in p.items()}
    a = torch.tensor(np.asarray(x, np.float64))[None]  # [1, CIN, n]
    for l in (1, 2, 3):
        a = F.relu(F.conv1d(a, t["W%d" % l], t["b%d" % l], padding=3))
    a3 = a[0].T  # [n, 64]
    h = F.relu(F.linear(a3, t["W4"], t["b4"]))
    score = F.linear(h, t["w5"][None], t["b5"])[:, 0]
    restart = F.linear(a3.mean(dim=0)[None], t["w6"][None], t["b6"])[0, 0]
    return score, restart, t


def state_inputs(rng, n):
    return rng.standard_normal((ln.CIN, n)) * (np.arange(ln.CIN) < 3)[:, None]


def test_forward_matches_torch_statement():
    rng = np.random.default_rng(11)
    net = ln.Net(bf16_mode=False)
    for n in (1, 2, 7, 31, 101):
        p = random_params(rng)
        x = state_inputs(rng, n)
        fw = net.forward(p, x)
        score, restart, _ = torch_net(p, x)
        want_s = score.detach().numpy()
        assert fw["score"].shape == (n,)
        assert np.allclose(fw["score"], want_s, rtol=1e-12, atol=1e-12 * np.abs(want_s).max()), n
        assert abs(fw["restart"] - restart.item()) <= 1e-12 * max(1.0, abs(restart.item())), n


def test_loss_and_gradients_match_torch_autograd():
    rng = np.random.default_rng(12)
    net = ln.Net(bf16_mode=False)
    n, B = 23, 4
    p = random_params(rng)
    xs = [state_inputs(rng, n) for _ in range(B)]
    targets = rng.integers(0, n, B)
    ys = rng.standard_normal(B)
    wfs = np.array([1.0, 0.0, 0.25, 2.0])
    loss, g = net.batch_loss_and_grads(p, xs, targets, ys, wfs)

    t = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in p.items()}
    total = 0.0
    for b in range(B):
        score, restart, tb = torch_net({k: v for k, v in p.items()}, xs[b])
        ce = torch.nn.functional.cross_entropy(score[None], torch.tensor([int(targets[b])]))
        lb = (wfs[b] * ce + 0.5 * (restart - ys[b]) ** 2) / B
        lb.backward()
        total += lb.item()
        for k in t:
            t[k].grad = tb[k].grad if t[k].grad is None else t[k].grad + tb[k].grad
    assert abs(loss - total) <= 1e-12 * abs(total)
    for name, _ in ln.PARAM_SHAPES:
        want = t[name].grad.numpy()
        got = np.asarray(g[name], np.float64)
        assert got.shape == want.shape, name
        # b5's gradient sums softmax gradients and is zero up to rounding: absolute floor
        tol = 1e-10 * max(np.abs(want).max(), 1e-5)
        assert np.all(np.abs(got - want) <= tol), (name, np.abs(got - want).max(), tol)


def test_loss_grads_of_one_sample_match_torch():
    """The score and restart gradients of one sample (softmax cross-entropy and the
    squared restart error) against torch's."""
    rng = np.random.default_rng(13)
    net = ln.Net(bf16_mode=False)
    n = 17
    p = random_params(rng)
    x = state_inputs(rng, n)
    fw = net.forward(p, x)
    loss, ds, dr = net.loss_grads(fw, 5, 0.3, 0.7, 0.5)
    s = torch.tensor(fw["score"], requires_grad=True)
    r = torch.tensor(float(fw["restart"]), dtype=torch.float64, requires_grad=True)
    lt = 0.7 * torch.nn.functional.cross_entropy(s[None], torch.tensor([5])) + 0.5 * (r - 0.3) ** 2
    (0.5 * lt).backward()
    assert abs(loss - lt.item()) <= 1e-12 * abs(lt.item())
    assert np.allclose(ds, s.grad.numpy(), rtol=1e-12, atol=1e-15)
    assert abs(float(dr) - r.grad.item()) <= 1e-12


def test_features_follow_their_definitions():
    """x[0] = s_i, x[1] = C_{2(i+1)}/sqrt(L) (Eq. 1, zero past the last lag), x[2] =
    dISL_i/(8L) with dISL from flipping s_i and its mirror and recomputing Eq. 2."""
    import oracle

    rng = np.random.default_rng(14)
    for L in (5, 41, 101):
        n = (L + 1) // 2
        xfree = np.where(rng.random(n) < 0.5, -1, 1).astype(np.int8)
        s = oracle.skew_expand(xfree, L)
        corr = np.correlate(s.astype(np.int64), s.astype(np.int64), mode="full")[L - 1:]  # C_0..C_{L-1}
        isl0 = int((corr[1:] ** 2).sum())
        dl = []
        for i in range(n):
            f = s.astype(np.int64).copy()
            f[i] = -f[i]
            if L - 1 - i != i:
                f[L - 1 - i] = -f[L - 1 - i]
            cf = np.correlate(f, f, mode="full")[L:]
            dl.append(int((cf ** 2).sum()) - isl0)
        C_even = np.array([corr[2 * m] for m in range(1, n)])
        x = ln.features(s, C_even, np.array(dl))
        assert x.shape == (ln.CIN, n)
        assert np.array_equal(x[0], s[:n].astype(np.float32))
        c = np.zeros(n)
        c[:n - 1] = [corr[2 * (i + 1)] for i in range(n - 1)]
        assert np.array_equal(x[1], (c / np.sqrt(np.float32(L))).astype(np.float32))
        assert np.array_equal(x[2], (np.array(dl, np.float32) / np.float32(8 * L)))
        assert not x[3:].any()
