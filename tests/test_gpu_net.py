"""GPU parity of the learned-proposal network kernels against oracle/learned.py, which
rounds to bfloat16 at the same points, element by element.

The per-element bound is stated in tests/nettol.py.  AdamW agrees to float32 rounding."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import paper_2011_00068_gb300 as labs
from oracle import learned as ln
from tests.nettol import assert_close

pytestmark = pytest.mark.gpu


def lib():
    return labs.library()


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def net_ws(n, B):
    pc, wb = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib().labs_net_sizes(n, B, ctypes.byref(pc), ctypes.byref(wb)) == 0
    assert pc.value == ln.param_count()
    return torch.empty(wb.value, dtype=torch.uint8, device="cuda"), wb.value


def random_case(n, B, seed, scale=0.15):
    rng = np.random.default_rng(seed)
    params = {name: (rng.standard_normal(shape) * scale).astype(np.float32) for name, shape in ln.PARAM_SHAPES}
    x = rng.standard_normal((B, 3, n)).astype(np.float32)
    return params, x


def oracle_x(x):
    B, _, n = x.shape
    out = np.zeros((B, ln.CIN, n), np.float32)
    out[:, :3] = x
    return out


def gpu_forward(flat, x):
    B, _, n = x.shape
    ws, wb = net_ws(n, B)
    p = torch.from_numpy(flat).cuda()
    xd = torch.from_numpy(x).cuda()
    sc = torch.empty((B, n), device="cuda")
    rs = torch.empty(B, device="cuda")
    s = torch.cuda.current_stream()
    assert lib().labs_net_forward(ptr(p), ptr(xd), B, n, ptr(sc), ptr(rs), ptr(ws), wb,
                                  ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    return sc.cpu().numpy(), rs.cpu().numpy()


@pytest.mark.parametrize("n,B", [(13, 3), (101, 5), (128, 4), (152, 3), (251, 2)])
def test_forward_matches_oracle(n, B):
    params, x = random_case(n, B, seed=n)
    sc, rs = gpu_forward(ln.flatten(params), x)
    net = ln.Net(True)
    xo = oracle_x(x)
    worst = 0.0
    for b in range(B):
        fw = net.forward(params, xo[b])
        worst = max(worst, assert_close(sc[b], fw["score"], "score of sample %d" % b))
        # the restart score is one dot product: its scale is the sum of its terms' sizes
        terms = float(np.abs(fw["W"]["w6"] * fw["pooled"]).sum() + abs(params["b6"][0]))
        worst = max(worst, assert_close(rs[b], fw["restart"], "restart score of sample %d" % b, scale=terms))
    print("n=%d: worst error / bound %.3f" % (n, worst))


@pytest.mark.parametrize("n,B", [(13, 4), (101, 6), (128, 5)])
def test_gradients_match_oracle(n, B):
    params, x = random_case(n, B, seed=100 + n)
    rng = np.random.default_rng(n)
    target = rng.integers(0, n, B).astype(np.int32)
    y = rng.standard_normal(B).astype(np.float32)
    wf = (rng.random(B) < 0.7).astype(np.float32)
    ws, wb = net_ws(n, B)
    flat = ln.flatten(params)
    p = torch.from_numpy(flat).cuda()
    g = torch.empty_like(p)
    loss = torch.zeros(1, device="cuda")
    s = torch.cuda.current_stream()
    # keep every device input referenced until the asynchronous call has finished
    xd, td, yd, wd = (torch.from_numpy(a).cuda() for a in (x, target, y, wf))
    rc = lib().labs_net_gradients(ptr(p), ptr(xd), ptr(td), ptr(yd), ptr(wd), B, n, ptr(g), ptr(loss), ptr(ws), wb,
                                  ctypes.c_void_p(s.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    gpu = ln.unflatten(g.cpu().numpy())
    net = ln.Net(True)
    oloss, og = net.batch_loss_and_grads(params, list(oracle_x(x)), target, y, wf)
    assert_close(loss.item(), oloss, "loss", scale=0.0)
    worst = 0.0
    for name, _ in ln.PARAM_SHAPES:
        # b5's exact gradient is zero (each sample's softmax gradient sums to zero): both
        # sides hold float32 residue of n terms of size <= 1/B, below n * 2^-23
        scale = 1e-3 if name == "b5" else None
        worst = max(worst, assert_close(gpu[name], og[name], "gradient of " + name, scale=scale))
    print("n=%d: worst gradient error / bound %.3f" % (n, worst))


def test_adamw_matches_oracle():
    rng = np.random.default_rng(5)
    N = ln.param_count()
    p = rng.standard_normal(N).astype(np.float32)
    g = rng.standard_normal(N).astype(np.float32)
    m = (rng.standard_normal(N) * 0.1).astype(np.float32)
    v = (rng.random(N) * 0.1).astype(np.float32)
    t = 7
    P, G, M, V = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    s = torch.cuda.current_stream()
    assert lib().labs_net_adamw(ptr(P), ptr(G), ptr(M), ptr(V), t, ctypes.c_float(1e-3), ctypes.c_float(0.01),
                                ctypes.c_void_p(s.cuda_stream)) == 0
    om = ln.unflatten(m.copy())
    ov = ln.unflatten(v.copy())
    out = ln.flatten(ln.adamw(ln.unflatten(p.copy()), ln.unflatten(g.copy()), om, ov, t, lr=1e-3, wd=0.01))
    assert np.allclose(P.cpu().numpy(), out, rtol=1e-5, atol=1e-6)
    assert np.allclose(M.cpu().numpy(), ln.flatten(om), rtol=1e-6, atol=1e-7)


def test_init_is_bounded_and_seeded():
    N = ln.param_count()
    a = torch.empty(N, device="cuda")
    b = torch.empty(N, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib().labs_net_init(ptr(a), 11, s) == 0 and lib().labs_net_init(ptr(b), 11, s) == 0
    pa = ln.unflatten(a.cpu().numpy())
    assert torch.equal(a, b)
    assert np.abs(pa["W2"]).max() <= np.sqrt(6 / 448) + 1e-6 and np.abs(pa["W2"]).std() > 0.01
    assert np.all(pa["b2"] == 0)


def test_forward_large_batch_sampled():
    """B = 2048 states of n = 101 (1888 tiles of 128 rows: several tiles per CTA, so the
    operand and accumulator barriers run through many phases): sampled states against
    the oracle, element by element."""
    n, B = 101, 2048
    params, x = random_case(n, B, seed=7)
    sc, rs = gpu_forward(ln.flatten(params), x)
    net = ln.Net(True)
    xo = oracle_x(x)
    rng = np.random.default_rng(8)
    for b in sorted(set(rng.choice(B, 24, replace=False).tolist()) | {0, B - 1}):
        fw = net.forward(params, xo[b])
        assert_close(sc[b], fw["score"], "score of sample %d" % b)
        terms = float(np.abs(fw["W"]["w6"] * fw["pooled"]).sum() + abs(params["b6"][0]))
        assert_close(rs[b], fw["restart"], "restart score of sample %d" % b, scale=terms)


def test_gradients_large_batch():
    """B = 1024 states of n = 101: each weight-gradient CTA reduces several blocks of 64
    rows and the per-CTA partials are summed; every gradient entry against the oracle."""
    n, B = 101, 1024
    params, x = random_case(n, B, seed=9)
    rng = np.random.default_rng(10)
    target = rng.integers(0, n, B).astype(np.int32)
    y = rng.standard_normal(B).astype(np.float32)
    wf = (rng.random(B) < 0.7).astype(np.float32)
    ws, wb = net_ws(n, B)
    p = torch.from_numpy(ln.flatten(params)).cuda()
    g = torch.empty_like(p)
    loss = torch.zeros(1, device="cuda")
    s = torch.cuda.current_stream()
    xd, td, yd, wd = (torch.from_numpy(a).cuda() for a in (x, target, y, wf))
    assert lib().labs_net_gradients(ptr(p), ptr(xd), ptr(td), ptr(yd), ptr(wd), B, n, ptr(g), ptr(loss), ptr(ws), wb,
                                    ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    gpu = ln.unflatten(g.cpu().numpy())
    oloss, og = ln.Net(True).batch_loss_and_grads(params, list(oracle_x(x)), target, y, wf)
    assert_close(loss.item(), oloss, "loss", scale=0.0)
    worst = 0.0
    for name, _ in ln.PARAM_SHAPES:
        scale = 1e-3 if name == "b5" else None
        worst = max(worst, assert_close(gpu[name], og[name], "gradient of " + name, scale=scale))
    print("B=%d: worst gradient error / bound %.3f" % (B, worst))
