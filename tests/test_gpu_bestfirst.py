"""GPU parity of the best-first search (Algorithm 1 as printed, LABS_FLAG_BEST_FIRST)
against the oracle's statement of it: per-step trace codes (fingerprint bits of each
new S) and ISLs, best and final sequences and counters, bit-exact; independence from
chunking and launch mode; the combinations the library refuses."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2011_00068_gb300 as labs
from paper_2011_00068_gb300 import _native

pytestmark = pytest.mark.gpu

BF = _native.LABS_FLAG_BEST_FIRST
K = _native.LABS_QUEUE_SIZE


def traced(L, walkers, steps, seed, **cfg):
    s = labs.Search(L, walkers, seed, **cfg)
    code, isl = s.trace(list(range(walkers)), steps)
    s.walk(steps)
    s.sync()
    return s, code.cpu().numpy(), isl.cpu().numpy()


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (21, 8, 600, {}),
    (41, 16, 800, {}),
    (21, 6, 500, {"tabu_log2": 4, "probe_cap": 3}),
    (101, 8, 400, {}),
    (201, 6, 300, {}),
    (303, 4, 200, {}),
    (511, 2, 80, {}),
])
def test_bestfirst_trajectory_parity(L, walkers, steps, kw):
    seed = 1
    s, code, isl = traced(L, walkers, steps, seed, flags=BF, **kw)
    o = oracle.bestfirst(L, seed, walkers, steps, pq_size=K, trace=True, **kw)
    assert np.array_equal(code, o["trace_code"])
    assert np.array_equal(isl, o["trace_isl"])
    res = s.results(seqs=True)
    for k in ("best_isl", "target_step"):
        assert np.array_equal(res[k], o[k]), k
    assert np.array_equal(res["isl"], o["final_isl"])
    assert np.array_equal(res["seq"], o["final_seq"])
    assert np.array_equal(res["best_seq"], o["best_seq"])
    st = s.stats()
    assert st["steps"] == walkers * steps and st["walkers_per_warp"] == 1
    assert st["flip_evaluations"] == walkers * steps * ((L + 1) // 2)
    assert st["restarts"] == int(o["restarts"].sum())
    assert st["overflows"] == int(o["overflows"].sum())
    assert st["blocked"] == int((o["trace_code"] == -1).sum())
    s.close()


def test_bestfirst_chunking_graphs_and_mixed_lengths():
    L, W, steps, seed = 61, 12, 700, 5
    ref = None
    for cfg in ({}, {"chunk_steps": 7}, {"chunk_steps": 64, "flags": BF | _native.LABS_FLAG_NO_GRAPH},
                {"warps_per_cta": 3, "chunk_steps": 100}):
        cfg = dict(cfg)
        cfg["flags"] = cfg.get("flags", BF)
        s, code, isl = traced(L, W, steps, seed, **cfg)
        if ref is None:
            ref = (code, isl)
        else:
            assert np.array_equal(code, ref[0]) and np.array_equal(isl, ref[1])
        s.close()
    o = oracle.bestfirst(L, seed, W, steps, pq_size=K, trace=True)
    assert np.array_equal(ref[0], o["trace_code"]) and np.array_equal(ref[1], o["trace_isl"])
    # several calls == one call; lengths mixed in one launch
    Ls, counts = [41, 23, 101], [5, 4, 3]
    s = labs.Search(Ls, counts, 9, flags=BF)
    code, isl = s.trace(list(range(sum(counts))), 400)
    for part in (1, 150, 249):
        s.walk(part)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    first = 0
    for Lg, cnt in zip(Ls, counts):
        o = oracle.bestfirst(Lg, 9, cnt, 400, pq_size=K, first_walker=first, trace=True)
        assert np.array_equal(code[first:first + cnt], o["trace_code"]), Lg
        assert np.array_equal(isl[first:first + cnt], o["trace_isl"]), Lg
        first += cnt


def test_bestfirst_refusals():
    with pytest.raises(labs.LabsError):
        labs.Search(41, 4, 1, flags=BF | _native.LABS_FLAG_LEARNED)
    s = labs.Search(41, 4, 1, flags=BF)
    s.walk(10)
    with pytest.raises(labs.LabsError):
        s.checkpoint()
    with pytest.raises(labs.LabsError):
        s.walk(_native.LABS_BEST_FIRST_MAX_STEPS)
    s.close()


SH = _native.LABS_FLAG_SECOND_HASH


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (21, 6, 500, {}),
    (21, 4, 400, {"tabu_log2": 4, "probe_cap": 3}),
    (41, 8, 600, {}),
    (201, 6, 300, {}),
    (303, 3, 200, {"tabu_log2": 10}),
])
def test_second_table_parity(L, walkers, steps, kw):
    """xLastovka's second table: skipped neighbours, insertions and the emptying at
    restarts give the oracle's trajectory, results and skip count bit for bit."""
    seed = 4
    s, code, isl = traced(L, walkers, steps, seed, flags=BF | SH, **kw)
    o = oracle.bestfirst(L, seed, walkers, steps, pq_size=K, trace=True, second_hash=True, **kw)
    assert np.array_equal(code, o["trace_code"])
    assert np.array_equal(isl, o["trace_isl"])
    res = s.results(seqs=True)
    assert np.array_equal(res["best_isl"], o["best_isl"])
    assert np.array_equal(res["seq"], o["final_seq"])
    assert np.array_equal(res["best_seq"], o["best_seq"])
    st = s.stats()
    assert st["cache_hits"] == int(o["cache_hits"].sum()) > 0
    assert st["restarts"] == int(o["restarts"].sum())
    s.close()


def test_second_table_chunking_and_refusal():
    L, W, steps, seed = 61, 8, 500, 7
    ref = None
    for cfg in ({}, {"chunk_steps": 13}, {"chunk_steps": 100, "warps_per_cta": 2}):
        s, code, isl = traced(L, W, steps, seed, flags=BF | SH, **cfg)
        if ref is None:
            ref = (code, isl, s.stats()["cache_hits"])
        else:
            assert np.array_equal(code, ref[0]) and np.array_equal(isl, ref[1])
            assert s.stats()["cache_hits"] == ref[2]
        s.close()
    o = oracle.bestfirst(L, seed, W, steps, pq_size=K, trace=True, second_hash=True)
    assert np.array_equal(ref[0], o["trace_code"]) and ref[2] == int(o["cache_hits"].sum())
    with pytest.raises(labs.LabsError):
        labs.Search(41, 4, 1, flags=SH)  # the second table belongs to the best-first search
