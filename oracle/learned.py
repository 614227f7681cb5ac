"""CPU oracle of the learned proposal network (the project's addition; the paper has no
learned component).  TEST INFRASTRUCTURE ONLY.

Network, per walker state of n free variables (positions i = 0..n-1):
    x       : 3 features per position (s_i, C_{2(i+1)}/sqrt(L), dISL_i/(8L)), zero-padded to 16 channels
    a1..a3  : a_l = relu(conv_l(a_{l-1}) + b_l), Conv1d with 64 output channels, 7 taps,
              zero padding 3 (positions outside 0..n-1 are zero)
    h       : relu(a3 W4^T + b4), 64 -> 64 per position
    score_i : h_i . w5 + b5                              (flip score)
    restart : mean_i(a3_i) . w6 + b6                     (restart score)
Loss per sample b (weights wf_b >= 0, targets t_b, y_b):
    wf_b * CE(softmax(score_b), t_b) + 0.5 (restart_b - y_b)^2, averaged over the batch.
Optimiser: AdamW (decoupled weight decay on weights, not biases).

Rounding: with bf16=True the values the GPU stores in bfloat16 are rounded to nearest-
even bfloat16 here too -- the inputs x, every weight used in a product, a1..a3, h, and
the back-propagated gradients entering each product -- and the rest is float32; with
bf16=False everything is float64 (used by the finite-difference pins).
"""
from __future__ import annotations

import numpy as np

C = 64      # channels
K = 7       # taps
CIN = 16    # padded input channels (3 used)
NFEAT = 3

PARAM_SHAPES = [
    ("W1", (C, CIN, K)), ("b1", (C,)),
    ("W2", (C, C, K)), ("b2", (C,)),
    ("W3", (C, C, K)), ("b3", (C,)),
    ("W4", (C, C)), ("b4", (C,)),
    ("w5", (C,)), ("b5", (1,)),
    ("w6", (C,)), ("b6", (1,)),
]


def param_count() -> int:
    return int(sum(np.prod(s) for _, s in PARAM_SHAPES))


def unflatten(flat: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shape in PARAM_SHAPES:
        size = int(np.prod(shape))
        out[name] = flat[off:off + size].reshape(shape)
        off += size
    return out


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[name]).reshape(-1) for name, _ in PARAM_SHAPES])


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    nan = np.isnan(a)
    out = rounded.astype(np.uint32).view(np.float32).copy()
    out[nan] = np.nan
    return out


class Net:
    def __init__(self, bf16_mode: bool = True):
        self.bf16_mode = bf16_mode
        self.dt = np.float32 if bf16_mode else np.float64

    def r(self, a):
        return bf16(a) if self.bf16_mode else np.asarray(a, dtype=np.float64)

    # conv with zero padding 3: out[o, i] = b[o] + sum_{c,k} W[o, c, k] in[c, i + k - 3]
    def conv(self, x, W, b):
        cin, n = x.shape
        xp = np.zeros((cin, n + K - 1), dtype=self.dt)
        xp[:, 3:3 + n] = x
        out = np.zeros((W.shape[0], n), dtype=self.dt)
        for k in range(K):
            out += W[:, :, k].astype(self.dt) @ xp[:, k:k + n]
        return out + b.astype(self.dt)[:, None]

    def conv_back_data(self, g, W, n):
        # d in[c, j] = sum_{o,k} W[o, c, k] g[o, j - k + 3]
        gp = np.zeros((g.shape[0], n + K - 1), dtype=self.dt)
        gp[:, 3:3 + n] = g
        out = np.zeros((W.shape[1], n), dtype=self.dt)
        for k in range(K):
            out += W[:, :, k].T.astype(self.dt) @ gp[:, 6 - k:6 - k + n]
        return out

    def conv_back_weight(self, g, x):
        # dW[o, c, k] = sum_i g[o, i] in[c, i + k - 3]
        cin, n = x.shape
        xp = np.zeros((cin, n + K - 1), dtype=self.dt)
        xp[:, 3:3 + n] = x
        return np.stack([g @ xp[:, k:k + n].T for k in range(K)], axis=2)

    def forward(self, p: dict, x: np.ndarray) -> dict:
        """x: [CIN, n] (already padded).  Returns scores, restart and the saved values."""
        r = self.r
        W = {k: r(v) for k, v in p.items() if k.startswith(("W", "w"))}
        x = r(x)
        a1 = r(np.maximum(self.conv(x, W["W1"], p["b1"]), 0))
        a2 = r(np.maximum(self.conv(a1, W["W2"], p["b2"]), 0))
        a3 = r(np.maximum(self.conv(a2, W["W3"], p["b3"]), 0))
        h = r(np.maximum(W["W4"].astype(self.dt) @ a3 + p["b4"].astype(self.dt)[:, None], 0))
        score = W["w5"].astype(self.dt) @ h + self.dt(p["b5"][0])
        pooled = a3.mean(axis=1)
        restart = self.dt(W["w6"].astype(self.dt) @ pooled + p["b6"][0])
        return {"x": x, "a1": a1, "a2": a2, "a3": a3, "h": h, "score": score, "pooled": pooled,
                "restart": restart, "W": W}

    def loss_grads(self, fw: dict, target: int, y: float, wf: float, scale: float):
        """Loss of one sample and the gradients of scale*loss w.r.t. score and restart."""
        s = fw["score"]
        m = s.max()
        e = np.exp(s - m)
        z = e.sum()
        ce = float(np.log(z) + m - s[target])
        prob = e / z
        ds = prob.copy()
        ds[target] -= 1.0
        ds *= wf * scale
        dr = (fw["restart"] - y) * scale
        loss = wf * ce + 0.5 * float((fw["restart"] - y) ** 2)
        return loss, ds.astype(self.dt), self.dt(dr)

    def backward(self, p: dict, fw: dict, ds: np.ndarray, dr) -> dict:
        r = self.r
        W = fw["W"]
        n = ds.shape[0]
        g = {}
        h, a3 = fw["h"], fw["a3"]
        g["w5"] = h @ ds
        g["b5"] = np.array([ds.sum()])
        g["w6"] = fw["pooled"] * dr
        g["b6"] = np.array([dr])
        dh = r(np.outer(W["w5"], ds) * (h > 0))
        g["W4"] = dh @ a3.T
        g["b4"] = dh.sum(axis=1)
        da3 = W["W4"].T.astype(self.dt) @ dh + (W["w6"].astype(self.dt) * dr / n)[:, None]
        da3 = r(da3 * (a3 > 0))
        g["W3"] = self.conv_back_weight(da3, fw["a2"])
        g["b3"] = da3.sum(axis=1)
        da2 = r(self.conv_back_data(da3, W["W3"], n) * (fw["a2"] > 0))
        g["W2"] = self.conv_back_weight(da2, fw["a1"])
        g["b2"] = da2.sum(axis=1)
        da1 = r(self.conv_back_data(da2, W["W2"], n) * (fw["a1"] > 0))
        g["W1"] = self.conv_back_weight(da1, fw["x"])
        g["b1"] = da1.sum(axis=1)
        return g

    def batch_loss_and_grads(self, p, xs, targets, ys, wfs):
        """Mean loss over the batch and its gradients (dict)."""
        B = len(xs)
        tot = 0.0
        grads = {name: np.zeros(shape, dtype=self.dt) for name, shape in PARAM_SHAPES}
        for b in range(B):
            fw = self.forward(p, xs[b])
            loss, ds, dr = self.loss_grads(fw, int(targets[b]), float(ys[b]), float(wfs[b]), 1.0 / B)
            tot += loss / B
            for k, v in self.backward(p, fw, ds, dr).items():
                grads[k] += v
        return tot, grads


def adamw(params: dict, grads: dict, m: dict, v: dict, t: int, lr: float, beta1=0.9, beta2=0.999,
          eps=1e-8, wd=0.01):
    """One AdamW step (float32), t counted from 1."""
    out = {}
    for name, _ in PARAM_SHAPES:
        g = grads[name].astype(np.float32)
        m[name] = (beta1 * m[name] + (1 - beta1) * g).astype(np.float32)
        v[name] = (beta2 * v[name] + (1 - beta2) * g * g).astype(np.float32)
        mh = m[name] / (1 - beta1 ** t)
        vh = v[name] / (1 - beta2 ** t)
        decay = wd if name.startswith(("W", "w")) else 0.0
        out[name] = (params[name] - lr * (mh / (np.sqrt(vh) + eps) + decay * params[name])).astype(np.float32)
    return out


def features(seq: np.ndarray, C_even: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """[CIN, n] input of one state: s_i, C_{2(i+1)}/sqrt(L) (0 past the last lag),
    dISL_i/(8L); channels 3..15 zero."""
    L = seq.size
    n = (L + 1) // 2
    x = np.zeros((CIN, n), dtype=np.float32)
    x[0] = seq[:n]
    c = np.zeros(n, dtype=np.float32)
    c[:n - 1] = C_even[:n - 1]
    x[1] = c / np.sqrt(np.float32(L))
    x[2] = np.asarray(delta, dtype=np.float32) / np.float32(8 * L)
    return x
