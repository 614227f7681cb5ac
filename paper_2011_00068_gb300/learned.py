"""Training of the learned proposal network from the walk's own log.

Data: a plain walk with the log armed writes one record per walker and chunk (the
state at the chunk start, the flip it took, the lowest ISL it reached before its first
restart).  Labels (labs_log_labels) and inputs (labs_features) are built on the GPU;
each training step runs the library's forward/backward kernels (labs_net_gradients)
and its AdamW kernel.  PyTorch only allocates memory and shuffles the record buffer.
"""
from __future__ import annotations

import ctypes

import torch

from . import LOG_RECORD_WORDS, Search, _check, _ptr, _stream_handle, features, library, log_labels


def param_count(n: int = 128) -> int:
    pc = ctypes.c_size_t()
    _check(library().labs_net_sizes(n, 1, ctypes.byref(pc), None), library())
    return int(pc.value)


def init_params(seed: int, device=None) -> torch.Tensor:
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    p = torch.empty(param_count(), dtype=torch.float32, device=dev)
    _check(library().labs_net_init(_ptr(p), int(seed), _stream_handle(torch.cuda.current_stream(dev))), library())
    return p


def collect(L: int, walkers: int, chunks: int, seed: int, chunk_steps: int = 256, device=None, **cfg) -> torch.Tensor:
    """Walk `walkers` walkers of length L for `chunks` chunks with the log armed; returns
    the records (uint8 [walkers*chunks, 64])."""
    s = Search(L, walkers, seed, device=device, chunk_steps=chunk_steps, **cfg)
    rec = s.log(walkers * chunks)
    s.walk(chunk_steps * chunks)
    s.sync()
    out = rec.clone()
    s.close()
    return out


class Trainer:
    """AdamW training of the network on walk-log records, batch by batch."""

    def __init__(self, L: int, batch: int, seed: int, device=None, lr: float = 1e-3, weight_decay: float = 0.01):
        self.lib = library()
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.L, self.n, self.B = L, (L + 1) // 2, batch
        self.lr, self.wd = lr, weight_decay
        self.params = init_params(seed, self.dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        wb = ctypes.c_size_t()
        _check(self.lib.labs_net_sizes(self.n, batch, None, ctypes.byref(wb)), self.lib)
        self.ws = torch.empty(int(wb.value), dtype=torch.uint8, device=self.dev)
        self.ws_bytes = int(wb.value)
        self.t = 0

    def step(self, records: torch.Tensor) -> torch.Tensor:
        """One AdamW step on a batch of records; returns the loss (device tensor)."""
        s = _stream_handle(torch.cuda.current_stream(self.dev))
        B = records.shape[0]
        x = features(self.L, records, LOG_RECORD_WORDS, B)
        target, y, wf = log_labels(records)
        _check(self.lib.labs_net_gradients(_ptr(self.params), _ptr(x), _ptr(target), _ptr(y), _ptr(wf), B, self.n,
                                           _ptr(self.grads), _ptr(self.loss), _ptr(self.ws), self.ws_bytes, s),
               self.lib)
        self.t += 1
        _check(self.lib.labs_net_adamw(_ptr(self.params), _ptr(self.grads), _ptr(self.m), _ptr(self.v), self.t,
                                       ctypes.c_float(self.lr), ctypes.c_float(self.wd), s), self.lib)
        self._keep = (x, target, y, wf)
        return self.loss.clone()

    def fit(self, records: torch.Tensor, steps: int, seed: int = 0) -> list:
        """`steps` steps over the records, reshuffled each epoch; returns the losses."""
        N = records.shape[0]
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        losses, pos, perm = [], N, None
        for _ in range(steps):
            if pos + self.B > N:
                perm = records[torch.randperm(N, device=self.dev, generator=g)]
                pos = 0
            losses.append(self.step(perm[pos:pos + self.B]))
            pos += self.B
        return [float(v.item()) for v in losses]
