"""GB300-native search for skew-symmetric binary sequences with a high merit factor
(Brest & Boskovic, "Computational Search of Long Skew-symmetric Binary Sequences with
High Merit Factors", arXiv 2011.00068).

This package is the Python face of liblabs (C ABI in include/labs.h, CUDA sources in
csrc/).  It marshals arguments only: PyTorch provides device memory and streams, and
every step of the search runs in liblabs's sm_103a kernels.  There is no CPU path:
when the library cannot be loaded every call raises.

    import torch, paper_2011_00068_gb300 as labs
    s = labs.Search(201, walkers=16384, seed=7)      # Algorithm 1, one run per walker
    s.walk(10_000)
    print(s.best())                                   # {'isl': ..., 'F': ..., 'hex': ...}
    labs.isl(rows)               # Eq. 2 for int8 [B, L] rows on the GPU
    labs.neighbor_delta(rows)    # dISL of every free-variable flip, int32 [B, n]
    labs.enumerate_skew(41)      # exhaustive skew-symmetric optimum
"""
from __future__ import annotations

import atexit
import ctypes
from typing import Sequence

import numpy as np
import torch

from . import _native
from ._native import LabsConfig, LabsCounters, LabsError  # noqa: F401

__all__ = ["Search", "isl", "neighbor_delta", "enumerate_skew", "config", "LabsError", "library", "features",
           "log_labels", "close_rows"]

LOG_RECORD_WORDS = 16  # a labs_log_record is 16 32-bit words


def library():
    """The loaded liblabs (ctypes.CDLL), built on first use."""
    return _native.load()


def _err(lib, ctx) -> str:
    msg = lib.labs_last_error(ctx)
    return msg.decode() if msg else ""


def _check(rc: int, lib, ctx=None):
    if rc != _native.LABS_OK:
        raise LabsError(rc, _err(lib, ctx) if ctx else "")


def config(**kw) -> LabsConfig:
    """labs_config with the library defaults, then the given fields."""
    cfg = LabsConfig()
    library().labs_default_config(ctypes.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError("unknown config field %r" % k)
        setattr(cfg, k, int(v))
    return cfg


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream) -> ctypes.c_void_p:
    return ctypes.c_void_p(stream.cuda_stream)


class Search:
    """A set of independent walkers (one run of Algorithm 1 each) on one GPU.

    ``L`` and ``walkers`` are an int each, or equal-length sequences for a context that
    mixes lengths (walker ids then run length by length).  Extra keyword arguments are
    labs_config fields (tabu_log2, probe_cap, patience, target_num, target_den,
    chunk_steps, warps_per_cta, flags).  ``objective="psl"`` sets LABS_FLAG_PSL: the
    walkers minimise (PSL, ISL) pairs instead of ISL."""

    def __init__(self, L, walkers, seed: int, *, device=None, stream=None, objective: str = "isl", **cfg):
        if objective not in ("isl", "psl"):
            raise ValueError("objective is 'isl' or 'psl'")
        if objective == "psl":
            cfg["flags"] = int(cfg.get("flags", 0)) | _native.LABS_FLAG_PSL
        self.lib = library()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.type != "cuda":
            raise ValueError("liblabs runs on CUDA devices only")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.cfg = config(**cfg)
            self.psl = bool(self.cfg.flags & _native.LABS_FLAG_PSL)
            self.ctx = ctypes.c_void_p()
            if isinstance(L, (list, tuple)):
                self.Ls = [int(x) for x in L]
                counts = [int(x) for x in walkers]
                Ls_a = (ctypes.c_int32 * len(self.Ls))(*self.Ls)
                W_a = (ctypes.c_int64 * len(counts))(*counts)
                rc = self.lib.labs_init_multi(ctypes.byref(self.ctx), Ls_a, W_a, len(self.Ls), seed,
                                              ctypes.byref(self.cfg), _stream_handle(self.stream))
            else:
                self.Ls = [int(L)]
                counts = [int(walkers)]
                rc = self.lib.labs_init(ctypes.byref(self.ctx), int(L), int(walkers), seed, ctypes.byref(self.cfg),
                                        _stream_handle(self.stream))
            if rc != 0:
                msg = _err(self.lib, self.ctx)
                self.lib.labs_destroy(self.ctx)
                self.ctx = None
                raise LabsError(rc, msg)
            self.counts = counts
            self.first = list(np.cumsum([0] + counts[:-1]))
            self.W = int(sum(counts))
            self.seed = seed
            nbytes = ctypes.c_size_t()
            _check(self.lib.labs_workspace_bytes(self.ctx, ctypes.byref(nbytes)), self.lib, self.ctx)
            self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
            _check(self.lib.labs_bind_workspace(self.ctx, _ptr(self.workspace), nbytes.value), self.lib, self.ctx)
        self._trace_bufs = None

    # ------------------------------------------------------------------ control
    def _c(self, rc):
        _check(rc, self.lib, self.ctx)

    def reset(self):
        self._c(self.lib.labs_reset(self.ctx))

    def walk(self, steps: int):
        """Advance every walker by ``steps`` steps (asynchronous)."""
        self._c(self.lib.labs_walk(self.ctx, int(steps)))

    def sync(self):
        self._c(self.lib.labs_sync(self.ctx))

    def set_deadline(self, ns_from_now: int):
        self._c(self.lib.labs_set_deadline(self.ctx, int(ns_from_now)))

    def cancel(self):
        self._c(self.lib.labs_cancel(self.ctx))

    def clear_stop(self):
        self._c(self.lib.labs_clear_stop(self.ctx))

    # ------------------------------------------------------------------ results
    def best(self, L: int = 0) -> dict:
        Lmax = max(self.Ls)
        seq = np.zeros(Lmax, dtype=np.int8)
        isl_ = ctypes.c_int32()
        F = ctypes.c_double()
        Lo = ctypes.c_int32()
        hexbuf = ctypes.create_string_buffer((Lmax + 3) // 4 + 1)
        self._c(self.lib.labs_best(self.ctx, int(L), seq.ctypes.data_as(ctypes.c_void_p), ctypes.byref(isl_),
                                   ctypes.byref(F), ctypes.byref(Lo), hexbuf))
        out = {"L": Lo.value, "isl": isl_.value, "F": F.value, "seq": seq[:Lo.value].copy(),
               "hex": hexbuf.value.decode()}
        if self.psl:
            psl_ = ctypes.c_int32()
            self._c(self.lib.labs_best_psl(self.ctx, int(L), None, ctypes.byref(psl_), None, None, None))
            out["psl"] = psl_.value
        return out

    def results(self, first: int = 0, count: int | None = None, seqs: bool = False) -> dict:
        count = self.W - first if count is None else count
        out = {"isl": np.zeros(count, np.int32), "best_isl": np.zeros(count, np.int32),
               "target_step": np.zeros(count, np.int64)}
        args = [out["isl"].ctypes.data_as(ctypes.c_void_p), out["best_isl"].ctypes.data_as(ctypes.c_void_p)]
        if seqs:
            g = int(np.searchsorted(np.cumsum(self.counts), first, side="right"))
            Lw = self.Ls[g]
            out["seq"] = np.zeros((count, Lw), np.int8)
            out["best_seq"] = np.zeros((count, Lw), np.int8)
            args += [out["seq"].ctypes.data_as(ctypes.c_void_p), out["best_seq"].ctypes.data_as(ctypes.c_void_p)]
        else:
            args += [None, None]
        args.append(out["target_step"].ctypes.data_as(ctypes.c_void_p))
        self._c(self.lib.labs_walker_results(self.ctx, int(first), int(count), *args))
        if self.psl:
            out["psl"] = np.zeros(count, np.int32)
            out["best_psl"] = np.zeros(count, np.int32)
            self._c(self.lib.labs_walker_psl(self.ctx, int(first), int(count),
                                             out["psl"].ctypes.data_as(ctypes.c_void_p),
                                             out["best_psl"].ctypes.data_as(ctypes.c_void_p)))
        return out

    def stats(self, L: int = 0) -> dict:
        c = LabsCounters()
        self._c(self.lib.labs_stats(self.ctx, int(L), ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in LabsCounters._fields_}

    def trace(self, walker_ids: Sequence[int], capacity: int):
        """Arm per-step tracing; returns the device logs (code, isl), int32 [k, capacity]."""
        k = len(walker_ids)
        ids = np.asarray(walker_ids, dtype=np.int64)
        code = torch.full((max(k, 1), max(capacity, 1)), -7, dtype=torch.int32, device=self.device)
        isl_ = torch.full((max(k, 1), max(capacity, 1)), -7, dtype=torch.int32, device=self.device)
        self._c(self.lib.labs_trace(self.ctx, ids.ctypes.data_as(ctypes.c_void_p), k, int(capacity), _ptr(code),
                                    _ptr(isl_)))
        self._trace_bufs = (code, isl_)
        return code[:k], isl_[:k]

    def log(self, capacity: int) -> torch.Tensor:
        """Arm the walk log: returns the record buffer (uint8 [capacity, 64]); record
        k*W + w is walker w's k-th chunk from now (see labs_log_record)."""
        buf = torch.zeros((max(capacity, 1), _native.LOG_RECORD_BYTES), dtype=torch.uint8, device=self.device)
        self._c(self.lib.labs_log(self.ctx, _ptr(buf), int(capacity)))
        self._log_buf = buf
        return buf[:capacity]

    def learned(self, params: torch.Tensor | None, tau: int = 0, candidates: int = 4):
        """Turn the learned mode on with network parameters (float32 CUDA tensor) or off."""
        if params is None:
            self._c(self.lib.labs_learned(self.ctx, None, 0, 1, None, 0))
            self._learned_ws = None
            return
        nbytes = ctypes.c_size_t()
        self._c(self.lib.labs_learned_workspace_bytes(self.ctx, int(candidates), ctypes.byref(nbytes)))
        self._learned_ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self._learned_params = params
        self._c(self.lib.labs_learned(self.ctx, _ptr(params), int(tau), int(candidates), _ptr(self._learned_ws),
                                      nbytes.value))

    def trace_learned(self, k: int, capacity: int, n_max: int) -> dict:
        """Replay dumps of the k walkers armed by trace() (learned mode)."""
        d = {"scores": torch.zeros((k, capacity, n_max), dtype=torch.float32, device=self.device),
             "score_step": torch.zeros((k, capacity), dtype=torch.int64, device=self.device),
             "score_count": torch.zeros(k, dtype=torch.int32, device=self.device),
             "restart": torch.zeros((k, capacity, 8), dtype=torch.int32, device=self.device),
             "restart_idx": torch.zeros((k, capacity), dtype=torch.int64, device=self.device),
             "restart_count": torch.zeros(k, dtype=torch.int32, device=self.device)}
        self._c(self.lib.labs_trace_learned(self.ctx, int(capacity), _ptr(d["scores"]), _ptr(d["score_step"]),
                                            _ptr(d["score_count"]), _ptr(d["restart"]), _ptr(d["restart_idx"]),
                                            _ptr(d["restart_count"])))
        self._dumps = d
        return d

    def checkpoint(self, with_tabu: bool = True) -> bytearray:
        n = ctypes.c_size_t()
        self._c(self.lib.labs_checkpoint(self.ctx, int(with_tabu), None, ctypes.byref(n)))
        buf = bytearray(n.value)
        cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
        self._c(self.lib.labs_checkpoint(self.ctx, int(with_tabu), cbuf, ctypes.byref(n)))
        return buf

    def restore(self, buf: bytearray):
        cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
        self._c(self.lib.labs_restore(self.ctx, cbuf, len(buf)))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.labs_destroy(self.ctx)
            self.ctx = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_row_ctx: dict = {}


def close_rows():
    """Destroys the contexts that isl() and neighbor_delta() keep per (length, device,
    stream); the next call creates them again.  Runs at interpreter exit."""
    lib = _native._lib
    while _row_ctx:
        _, ctx = _row_ctx.popitem()
        if lib is not None:
            lib.labs_destroy(ctx)


atexit.register(close_rows)


def _rows_ctx(L: int, device: torch.device, stream):
    key = (L, device.index, stream.cuda_stream)
    c = _row_ctx.get(key)
    if c is None:
        lib = library()
        ctx = ctypes.c_void_p()
        with torch.cuda.device(device):
            rc = lib.labs_init(ctypes.byref(ctx), int(L), 0, 0, None, _stream_handle(stream))
        if rc != 0:
            msg = _err(lib, ctx)
            lib.labs_destroy(ctx)
            raise LabsError(rc, msg)
        c = _row_ctx[key] = ctx
    return c


def _rows(seqs: torch.Tensor):
    if seqs.dtype != torch.int8 or seqs.dim() != 2 or not seqs.is_cuda:
        raise TypeError("need an int8 CUDA tensor [batch, L]")
    return seqs.contiguous()


def isl(seqs: torch.Tensor, stream=None) -> torch.Tensor:
    """Eq. 2 for every row of an int8 [batch, L] +-1 tensor; -1 for rows that are not +-1."""
    seqs = _rows(seqs)
    stream = stream or torch.cuda.current_stream(seqs.device)
    L = seqs.shape[1]
    out = torch.empty(seqs.shape[0], dtype=torch.int32, device=seqs.device)
    lib = library()
    ctx = _rows_ctx(L, seqs.device, stream)
    with torch.cuda.device(seqs.device):
        _check(lib.labs_isl(ctx, _ptr(seqs), seqs.shape[0], _ptr(out)), lib, ctx)
    return out


def neighbor_delta(seqs: torch.Tensor, stream=None) -> torch.Tensor:
    """dISL of flipping each free variable (and its mirror) of every skew-symmetric row:
    int32 [batch, n]; rows that are not +-1 / skew-symmetric are filled with INT32_MIN."""
    seqs = _rows(seqs)
    stream = stream or torch.cuda.current_stream(seqs.device)
    L = seqs.shape[1]
    out = torch.empty((seqs.shape[0], (L + 1) // 2), dtype=torch.int32, device=seqs.device)
    lib = library()
    ctx = _rows_ctx(L, seqs.device, stream)
    with torch.cuda.device(seqs.device):
        _check(lib.labs_neighbor_delta(ctx, _ptr(seqs), seqs.shape[0], _ptr(out)), lib, ctx)
    return out


def enumerate_skew(L: int, device=None, stream=None) -> tuple[int, int, int]:
    """Exhaustive skew-symmetric search (centre +1): (min ISL, #minimisers, lowest
    minimising assignment)."""
    lib = library()
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    nbytes = ctypes.c_size_t()
    _check(lib.labs_enumerate_scratch_bytes(int(L), ctypes.byref(nbytes)), lib)
    scratch = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
    m, cnt, first = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    with torch.cuda.device(device):
        stream = stream or torch.cuda.current_stream(device)
        _check(lib.labs_enumerate(int(L), _ptr(scratch), nbytes.value, ctypes.byref(m), ctypes.byref(cnt),
                                  ctypes.byref(first), _stream_handle(stream)), lib)
    return m.value, cnt.value, first.value


def log_labels(records: torch.Tensor, stream=None):
    """(target int32, y float32, wf float32) of walk-log records (uint8 [N, 64])."""
    lib = library()
    N = records.shape[0]
    dev = records.device
    target = torch.empty(N, dtype=torch.int32, device=dev)
    y = torch.empty(N, dtype=torch.float32, device=dev)
    wf = torch.empty(N, dtype=torch.float32, device=dev)
    stream = stream or torch.cuda.current_stream(dev)
    _check(lib.labs_log_labels(_ptr(records), N, _ptr(target), _ptr(y), _ptr(wf), _stream_handle(stream)), lib)
    return target, y, wf


def features(L: int, bits: torch.Tensor, stride_words: int, count: int, stream=None) -> torch.Tensor:
    """Network inputs float32 [count, 3, n] of states given as free-variable bit words."""
    lib = library()
    n = (L + 1) // 2
    x = torch.empty((count, 3, n), dtype=torch.float32, device=bits.device)
    stream = stream or torch.cuda.current_stream(bits.device)
    _check(lib.labs_features(int(L), _ptr(bits), int(stride_words), int(count), _ptr(x), _stream_handle(stream)), lib)
    return x
