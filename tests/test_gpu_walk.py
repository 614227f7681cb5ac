"""GPU parity of the walk (labs_walk) against the oracle: per-step trace codes and
ISLs, best ISL and sequence, bit-exact, across lengths, table sizes, chunking and
launch modes; plus checkpoint/resume and stop control."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2011_00068_gb300 as labs
from paper_2011_00068_gb300 import _native

pytestmark = pytest.mark.gpu


def run_traced(L, walkers, steps, seed, ids=None, **cfg):
    s = labs.Search(L, walkers, seed, **cfg)
    ids = list(range(walkers)) if ids is None else ids
    code, isl = s.trace(ids, steps)
    s.walk(steps)
    s.sync()
    return s, code.cpu().numpy(), isl.cpu().numpy()


def oracle_for(L, seed, gid, steps, **kw):
    return oracle.walk(L, seed, 1, steps, first_walker=gid, trace=True, **kw)


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (5, 8, 200, {}),
    (13, 16, 600, {}),
    (41, 64, 2000, {}),
    (21, 16, 800, {"tabu_log2": 4, "probe_cap": 3}),
    (41, 16, 800, {"patience": 5}),
    (127, 16, 500, {}),
    (201, 16, 600, {}),
    (303, 8, 400, {}),
    (511, 4, 200, {}),
])
def test_walk_trajectory_parity(L, walkers, steps, kw):
    seed = 1
    s, code, isl = run_traced(L, walkers, steps, seed, **kw)
    res = s.results(seqs=True)
    okw = {k: v for k, v in kw.items() if k in ("tabu_log2", "probe_cap", "patience")}
    o = oracle.walk(L, seed, walkers, steps, trace=True, **okw)
    assert np.array_equal(code, o["trace_code"])
    assert np.array_equal(isl, o["trace_isl"])
    assert np.array_equal(res["best_isl"], o["best_isl"])
    assert np.array_equal(res["isl"], o["final_isl"])
    assert np.array_equal(res["seq"], o["final_seq"])
    assert np.array_equal(res["best_seq"], o["best_seq"])
    assert np.array_equal(res["target_step"], o["target_step"])
    st = s.stats()
    assert st["steps"] == walkers * steps
    assert st["flip_evaluations"] == walkers * steps * ((L + 1) // 2)
    assert st["restarts"] == int(o["restarts"].sum())
    assert st["overflows"] == int(o["overflows"].sum())
    s.close()


def test_chunking_and_graphs_do_not_change_trajectories():
    L, W, steps = 61, 32, 700
    ref = None
    for cfg in ({}, {"chunk_steps": 7}, {"chunk_steps": 64, "flags": _native.LABS_FLAG_NO_GRAPH},
                {"warps_per_cta": 2}, {"warps_per_cta": 5, "chunk_steps": 100}):
        s, code, isl = run_traced(L, W, steps, 5, **cfg)
        if ref is None:
            ref = (code, isl)
        else:
            assert np.array_equal(code, ref[0]) and np.array_equal(isl, ref[1])
        s.close()
    # several labs_walk calls == one call
    s = labs.Search(L, W, 5)
    code, isl = s.trace(list(range(W)), steps)
    for part in (1, 99, 300, 300):
        s.walk(part)
    s.sync()
    assert np.array_equal(code.cpu().numpy(), ref[0]) and np.array_equal(isl.cpu().numpy(), ref[1])


@pytest.mark.parametrize("L,W", [(41, 13), (151, 10), (61, 6)])
def test_launch_shapes_agree_with_oracle(L, W):
    """Four, two and one walker per warp run the same trajectories; walker counts that
    are not a multiple of the walkers per warp leave partly idle warps."""
    steps, seed = 500, 12
    o = oracle.walk(L, seed, W, steps, trace=True)
    shapes = []
    for flags in (0, _native.LABS_FLAG_TWO_PER_WARP, _native.LABS_FLAG_WARP_PER_WALKER):
        s, code, isl = run_traced(L, W, steps, seed, flags=flags)
        shapes.append(s.stats()["walkers_per_warp"])
        assert np.array_equal(code, o["trace_code"]) and np.array_equal(isl, o["trace_isl"]), flags
        s.close()
    assert shapes == [4, 2, 1]


def test_mixed_short_lengths_four_per_warp():
    """Lengths that change inside a warp of four walkers run group by group."""
    Ls, counts = [41, 23, 61, 5, 101], [5, 6, 7, 3, 2]
    steps, seed = 400, 4
    s = labs.Search(Ls, counts, seed)
    assert s.stats()["walkers_per_warp"] == 4
    code, isl = s.trace(list(range(sum(counts))), steps)
    s.walk(steps)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    first = 0
    for L, cnt in zip(Ls, counts):
        o = oracle.walk(L, seed, cnt, steps, first_walker=first, trace=True)
        assert np.array_equal(code[first:first + cnt], o["trace_code"]), L
        assert np.array_equal(isl[first:first + cnt], o["trace_isl"]), L
        first += cnt


def test_mixed_lengths_one_launch():
    Ls = [201, 23, 303, 41, 255]
    counts = [6, 5, 4, 7, 3]
    steps, seed = 400, 9
    s = labs.Search(Ls, counts, seed)
    code, isl = s.trace(list(range(sum(counts))), steps)
    s.walk(steps)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    first = 0
    for L, cnt in zip(Ls, counts):
        o = oracle.walk(L, seed, cnt, steps, first_walker=first, trace=True)
        assert np.array_equal(code[first:first + cnt], o["trace_code"])
        assert np.array_equal(isl[first:first + cnt], o["trace_isl"])
        r = s.results(first, cnt, seqs=True)
        assert np.array_equal(r["best_seq"], o["best_seq"])
        first += cnt
    b = s.best()
    all_best = []
    first = 0
    for L, cnt in zip(Ls, counts):
        r = s.results(first, cnt)
        all_best += [(int(e), first + j, L) for j, e in enumerate(r["best_isl"])]
        first += cnt
    e, w, Lw = min(all_best)
    assert (b["isl"], b["L"]) == (e, Lw)
    assert oracle.isl(b["seq"]) == e and oracle.hex_encode(b["seq"]) == b["hex"]
    b303 = s.best(303)
    assert b303["L"] == 303 and oracle.isl(b303["seq"]) == b303["isl"]


def test_best_and_hex_match_oracle():
    L, W, steps = 101, 40, 500
    s = labs.Search(L, W, 3)
    s.walk(steps)
    b = s.best()
    o = oracle.walk(L, 3, W, steps)
    w = int(np.argmin(o["best_isl"]))
    assert b["isl"] == o["best_isl"][w]
    assert np.array_equal(b["seq"], o["best_seq"][w])
    assert b["hex"] == oracle.hex_encode(o["best_seq"][w])
    assert abs(b["F"] - oracle.merit(L, b["isl"])) < 1e-12


def test_checkpoint_resume_is_bit_identical():
    L, W = 77, 24
    a = labs.Search(L, W, 21)
    a.walk(350)
    ck = a.checkpoint(with_tabu=True)
    a.walk(450)
    ra = a.results(seqs=True)
    b = labs.Search(L, W, 21)
    b.restore(ck)
    b.walk(450)
    rb = b.results(seqs=True)
    for k in ("isl", "best_isl", "seq", "best_seq", "target_step"):
        assert np.array_equal(ra[k], rb[k])
    o = oracle.walk(L, 21, W, 800)
    assert np.array_equal(ra["isl"], o["final_isl"])


def test_deadline_cancel_and_resume():
    """A passed deadline and a cancel stop the walkers between steps with their state
    saved; after labs_clear_stop, labs_walk(0) brings every walker to the planned step
    count and the trajectories equal an uninterrupted run."""
    L, W, steps = 151, 64, 3000
    s = labs.Search(L, W, 4, chunk_steps=256)
    s.set_deadline(0)
    s.walk(steps)
    with pytest.raises(labs.LabsError) as ei:
        s.sync()
    assert ei.value.code == _native.LABS_ETIMEOUT
    s.clear_stop()
    assert s.stats()["steps"] == 0
    s.walk(0)
    s.sync()
    assert s.stats()["steps"] == W * steps
    s.cancel()
    s.walk(500)
    with pytest.raises(labs.LabsError) as ei:
        s.sync()
    assert ei.value.code == _native.LABS_ECANCELLED
    s.clear_stop()
    s.walk(0)
    s.sync()
    assert s.stats()["steps"] == W * (steps + 500)
    o = oracle.walk(L, 4, W, steps + 500)
    assert np.array_equal(s.results()["isl"], o["final_isl"])
    assert np.array_equal(s.results()["best_isl"], o["best_isl"])


def test_reset_replays():
    s = labs.Search(45, 8, 2)
    s.walk(300)
    r1 = s.results(seqs=True)
    s.reset()
    s.walk(300)
    r2 = s.results(seqs=True)
    assert np.array_equal(r1["seq"], r2["seq"]) and np.array_equal(r1["best_isl"], r2["best_isl"])


def test_bad_arguments_raise():
    with pytest.raises(labs.LabsError):
        labs.Search(200, 4, 1)
    with pytest.raises(labs.LabsError):
        labs.Search(_native.LABS_MAX_L_LONG + 2, 4, 1)
    with pytest.raises(labs.LabsError):
        labs.Search(41, 4, 1, tabu_log2=21)
    with pytest.raises(labs.LabsError):
        labs.Search(41, 4, 1, warps_per_cta=9)
    s = labs.Search(41, 4, 1)
    with pytest.raises(labs.LabsError):
        s.walk(-1)
    with pytest.raises(labs.LabsError):
        s.results(3, 5)


def test_strict_ht_reports_overflows():
    """LABS_FLAG_STRICT_HT: labs_sync returns LABS_ETABU_FULL once an HT insertion found
    no free slot (a 16-slot table with 3 probes at L = 21 overflows within 400 steps, as
    the oracle shows); the walk itself is unchanged.  With the default table no error."""
    o = oracle.walk(21, 9, 2, 400, tabu_log2=4, probe_cap=3, trace=True)
    assert o["overflows"].sum() > 0
    s = labs.Search(21, 2, 9, tabu_log2=4, probe_cap=3, flags=_native.LABS_FLAG_STRICT_HT)
    code, isl = s.trace([0, 1], 400)
    s.walk(400)
    with pytest.raises(labs.LabsError) as err:
        s.sync()
    assert err.value.code == _native.LABS_ETABU_FULL
    assert np.array_equal(code.cpu().numpy(), o["trace_code"])
    assert s.stats()["overflows"] == int(o["overflows"].sum())
    # labs_reset empties HT and the counters: the error is gone, and a walk shorter than
    # the first overflow (the oracle's walkers first overflow within 10 steps) syncs
    s.reset()
    assert s.stats()["overflows"] == 0
    s.sync()
    assert oracle.walk(21, 9, 2, 9, tabu_log2=4, probe_cap=3)["overflows"].sum() == 0
    s.walk(9)
    s.sync()
    assert s.stats()["overflows"] == 0
    s.close()
    s = labs.Search(21, 2, 9, flags=_native.LABS_FLAG_STRICT_HT)
    s.walk(400)
    s.sync()
    assert s.stats()["overflows"] == 0
    s.close()
