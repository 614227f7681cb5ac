"""Failure paths of the walk, made on the host: a walker state corrupted in the
workspace between two labs_walk calls (LABS_ESTATE), and a workspace that is missing
or one byte short (LABS_ENOMEM).  Nothing here faults the GPU: the corruption is an
ordinary write of a wrong ISL into device memory the caller owns, which the next
chunk start detects by rebuilding the walker's rows and table from its stored bits."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2011_00068_gb300 as labs
from paper_2011_00068_gb300 import _native

pytestmark = pytest.mark.gpu

STATE_BYTES = 160  # sizeof(WalkerState)
STEPS_OFFSET = 64  # WalkerState.steps_done (int64), after cur[8] and best[8] (uint32)
ISL_OFFSET = 96    # WalkerState.isl, then best_isl (int32)
CKPT_HEADER = 64


def states_offset(s) -> int:
    """Byte offset of the WalkerState array in the workspace tensor: the array is the
    body of a checkpoint without HT (after its 64-byte header), found in the workspace
    by its content."""
    ck = bytes(s.checkpoint(with_tabu=False))
    states = ck[CKPT_HEADER:CKPT_HEADER + STATE_BYTES * s.W]
    ws = s.workspace.cpu().numpy().tobytes()
    off = ws.find(states)
    assert off >= 0 and ws.find(states, off + 1) < 0
    return off


@pytest.mark.parametrize("L,W,bad", [(41, 8, 5), (201, 6, 3), (351, 4, 2)])
def test_corrupted_walker_state_raises_estate(L, W, bad):
    seed, chunk = 3, 64
    s = labs.Search(L, W, seed, tabu_log2=10, chunk_steps=chunk)
    s.walk(chunk)
    s.sync()
    base = states_offset(s)
    off = base + STATE_BYTES * bad + ISL_OFFSET
    isl = int(np.frombuffer(s.workspace[off:off + 4].cpu().numpy().tobytes(), np.int32)[0])
    assert isl == s.results(bad, 1)["isl"][0]
    s.workspace[off:off + 4] = torch.from_numpy(np.array([isl + 8], np.int32).view(np.uint8)).to(s.device)
    s.walk(chunk)
    with pytest.raises(labs.LabsError) as err:
        s.sync()
    assert err.value.code == _native.LABS_ESTATE
    assert "walker %d" % bad in str(err.value)
    # the other walkers took their steps; the corrupted one stopped before its chunk.
    # (Result calls report the error until labs_reset: read the states directly.)
    raw = s.workspace[base:base + STATE_BYTES * W].cpu().numpy().tobytes()
    field = lambda w, o, dt: int(np.frombuffer(raw, dt, 1, STATE_BYTES * w + o)[0])
    o = oracle.walk(L, seed, W, 2 * chunk, tabu_log2=10)
    for w in range(W):
        if w == bad:
            assert field(w, STEPS_OFFSET, np.int64) == chunk
            assert field(w, ISL_OFFSET, np.int32) == isl + 8
            continue
        assert field(w, STEPS_OFFSET, np.int64) == 2 * chunk, w
        assert field(w, ISL_OFFSET, np.int32) == o["final_isl"][w], w
        assert field(w, ISL_OFFSET + 4, np.int32) == o["best_isl"][w], w
    # labs_reset clears the error with the states
    s.reset()
    s.walk(chunk)
    s.sync()
    assert s.stats()["steps"] == W * chunk
    s.close()


def test_corrupted_long_walker_state_raises_estate():
    L, W, bad, seed, chunk = 601, 3, 1, 4, 32
    s = labs.Search(L, W, seed, tabu_log2=10, chunk_steps=chunk)
    s.walk(chunk)
    s.sync()
    ck = bytes(s.checkpoint(with_tabu=False))
    ws = s.workspace.cpu().numpy().tobytes()
    # long sequences keep their bits beside the states; the states lead the checkpoint body
    off = ws.find(ck[CKPT_HEADER:CKPT_HEADER + STATE_BYTES * W])
    assert off >= 0
    off += STATE_BYTES * bad + ISL_OFFSET
    isl = int(np.frombuffer(ws[off:off + 4], np.int32)[0])
    assert isl == s.results(bad, 1)["isl"][0]
    s.workspace[off:off + 4] = torch.from_numpy(np.array([isl + 8], np.int32).view(np.uint8)).to(s.device)
    s.walk(chunk)
    with pytest.raises(labs.LabsError) as err:
        s.sync()
    assert err.value.code == _native.LABS_ESTATE
    s.close()


def test_missing_or_short_workspace_is_enomem():
    lib = labs.library()
    cfg = labs.config(tabu_log2=8)
    ctx = ctypes.c_void_p()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.labs_init(ctypes.byref(ctx), 41, 4, 1, ctypes.byref(cfg), stream) == 0
    try:
        need = ctypes.c_size_t()
        assert lib.labs_workspace_bytes(ctx, ctypes.byref(need)) == 0
        # unbound: every call that touches the workspace refuses
        assert lib.labs_walk(ctx, 10) == _native.LABS_ENOMEM
        assert lib.labs_reset(ctx) == _native.LABS_ENOMEM
        assert b"workspace" in lib.labs_last_error(ctx)
        # one byte short
        ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
        assert lib.labs_bind_workspace(ctx, ctypes.c_void_p(ws.data_ptr()), need.value - 1) == _native.LABS_ENOMEM
        assert lib.labs_walk(ctx, 10) == _native.LABS_ENOMEM
        # the full size works
        assert lib.labs_bind_workspace(ctx, ctypes.c_void_p(ws.data_ptr()), need.value) == 0
        assert lib.labs_walk(ctx, 10) == 0
        assert lib.labs_sync(ctx) == 0
    finally:
        lib.labs_destroy(ctx)


def test_learned_flags_reject_bad_combinations():
    lib = labs.library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for flags in (_native.LABS_FLAG_LEARNED | _native.LABS_FLAG_LEARNED_RESTARTS,
                  _native.LABS_FLAG_LEARNED_RESTARTS | _native.LABS_FLAG_BEST_FIRST,
                  _native.LABS_FLAG_LEARNED_RESTARTS | _native.LABS_FLAG_PSL):
        cfg = labs.config(tabu_log2=8, flags=flags)
        ctx = ctypes.c_void_p()
        rc = lib.labs_init(ctypes.byref(ctx), 41, 4, 1, ctypes.byref(cfg), stream)
        assert rc == _native.LABS_EINVAL, flags
        lib.labs_destroy(ctx)
    cfg = labs.config(tabu_log2=8, flags=_native.LABS_FLAG_LEARNED_RESTARTS)
    ctx = ctypes.c_void_p()
    assert lib.labs_init(ctypes.byref(ctx), 1025, 4, 1, ctypes.byref(cfg), stream) == _native.LABS_EINVAL
    lib.labs_destroy(ctx)
