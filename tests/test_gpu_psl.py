"""GPU parity of the walk under the PSL objective (LABS_FLAG_PSL) against the oracle,
whose every neighbour is rebuilt and measured from Eq. 1: per-step trace codes and
ISLs, best and final sequences with their PSL and ISL, counters, bit-exact;
independence from chunking and launch settings; the best-walker reduction in the
(PSL, ISL) order; checkpoints; the combinations the library refuses."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2011_00068_gb300 as labs
from paper_2011_00068_gb300 import _native

pytestmark = pytest.mark.gpu


def traced(L, walkers, steps, seed, **cfg):
    s = labs.Search(L, walkers, seed, objective="psl", **cfg)
    code, isl = s.trace(list(range(walkers)), steps)
    s.walk(steps)
    s.sync()
    return s, code.cpu().numpy(), isl.cpu().numpy()


def check_results(s, o, walkers, steps, L, flags=0):
    res = s.results(seqs=True)
    for k in ("best_isl", "best_psl", "target_step"):
        assert np.array_equal(res[k], o[k]), k
    assert np.array_equal(res["isl"], o["final_isl"])
    assert np.array_equal(res["psl"], o["final_psl"])
    assert np.array_equal(res["seq"], o["final_seq"])
    assert np.array_equal(res["best_seq"], o["best_seq"])
    st = s.stats()
    # two walkers per warp up to n = 128 unless LABS_FLAG_WARP_PER_WALKER asks for one
    pair = (L + 1) // 2 <= 128 and not flags & _native.LABS_FLAG_WARP_PER_WALKER
    assert st["steps"] == walkers * steps and st["walkers_per_warp"] == (2 if pair else 1)
    assert st["flip_evaluations"] == walkers * steps * ((L + 1) // 2)
    assert st["restarts"] == int(o["restarts"].sum())
    assert st["overflows"] == int(o["overflows"].sum())
    assert st["blocked"] == int((o["trace_code"] == -1).sum())
    # best walker: lowest (best PSL, best ISL), ties to the lowest id
    order = sorted(range(walkers), key=lambda g: (o["best_psl"][g], o["best_isl"][g], g))
    g = order[0]
    assert (st["best_psl"], st["best_isl"], st["best_walker"]) == (o["best_psl"][g], o["best_isl"][g], g)
    b = s.best()
    assert (b["psl"], b["isl"]) == (o["best_psl"][g], o["best_isl"][g])
    assert np.array_equal(b["seq"], o["best_seq"][g])
    assert oracle.psl(b["seq"]) == b["psl"] and oracle.isl(b["seq"]) == b["isl"]


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (3, 4, 40, {}),
    (5, 4, 60, {}),
    (13, 8, 300, {}),
    (21, 6, 400, {"tabu_log2": 4, "probe_cap": 3}),
    (21, 6, 300, {"patience": 5}),
    (41, 16, 500, {}),
    (63, 8, 300, {}),
    (101, 8, 300, {}),
    (201, 6, 200, {}),
    (303, 4, 120, {}),
    (511, 2, 40, {}),
])
def test_psl_trajectory_parity(L, walkers, steps, kw):
    seed = 3
    s, code, isl = traced(L, walkers, steps, seed, **kw)
    o = oracle.walk(L, seed, walkers, steps, trace=True, objective="psl", **kw)
    assert np.array_equal(code, o["trace_code"])
    assert np.array_equal(isl, o["trace_isl"])
    check_results(s, o, walkers, steps, L)
    s.close()


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (41, 7, 400, {}),
    (101, 5, 300, {"tabu_log2": 5, "probe_cap": 9}),
    (201, 9, 250, {}),
    (255, 4, 200, {"patience": 40}),
])
def test_psl_two_walkers_per_warp_matches_one(L, walkers, steps, kw):
    """Two walkers per warp (lockstep PSL step) and one walker per warp
    (LABS_FLAG_WARP_PER_WALKER) give the same trajectories, results and counters, and
    both match the oracle; odd walker counts leave a lone walker in the last warp, and a
    small table with a probe cap above the 8 slots of a round takes the full probes."""
    seed = 13
    o = oracle.walk(L, seed, walkers, steps, trace=True, objective="psl", **kw)
    for flags in (0, _native.LABS_FLAG_WARP_PER_WALKER):
        s, code, isl = traced(L, walkers, steps, seed, flags=flags, **kw)
        assert np.array_equal(code, o["trace_code"]), flags
        assert np.array_equal(isl, o["trace_isl"]), flags
        check_results(s, o, walkers, steps, L, flags)
        s.close()


def test_psl_chunking_graphs_and_mixed_lengths():
    L, W, steps, seed = 61, 12, 600, 5
    ref = None
    for cfg in ({}, {"chunk_steps": 7}, {"chunk_steps": 64, "flags": _native.LABS_FLAG_NO_GRAPH},
                {"warps_per_cta": 3, "chunk_steps": 100}):
        s, code, isl = traced(L, W, steps, seed, **cfg)
        if ref is None:
            ref = (code, isl)
        else:
            assert np.array_equal(code, ref[0]) and np.array_equal(isl, ref[1])
        s.close()
    o = oracle.walk(L, seed, W, steps, trace=True, objective="psl")
    assert np.array_equal(ref[0], o["trace_code"]) and np.array_equal(ref[1], o["trace_isl"])
    # several calls == one call; lengths mixed in one launch (lane blocks 5 and 3)
    Ls, counts = [41, 23, 201, 101], [5, 4, 2, 3]
    s = labs.Search(Ls, counts, 9, objective="psl")
    code, isl = s.trace(list(range(sum(counts))), 300)
    for part in (1, 120, 179):
        s.walk(part)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    first = 0
    for Lg, cnt in zip(Ls, counts):
        o = oracle.walk(Lg, 9, cnt, 300, first_walker=first, trace=True, objective="psl")
        assert np.array_equal(code[first:first + cnt], o["trace_code"]), Lg
        assert np.array_equal(isl[first:first + cnt], o["trace_isl"]), Lg
        assert np.array_equal(s.results(first, cnt)["best_psl"], o["best_psl"]), Lg
        first += cnt
    s.close()


def test_psl_checkpoint_round_trip():
    L, W, seed = 81, 6, 2
    a = labs.Search(L, W, seed, objective="psl")
    a.walk(150)
    buf = a.checkpoint(with_tabu=True)
    a.walk(200)
    ra = a.results(seqs=True)
    b = labs.Search(L, W, seed, objective="psl")
    b.restore(buf)
    b.walk(200)
    rb = b.results(seqs=True)
    for k in ("isl", "best_isl", "psl", "best_psl", "seq", "best_seq"):
        assert np.array_equal(ra[k], rb[k]), k
    o = oracle.walk(L, seed, W, 350, objective="psl")
    assert np.array_equal(ra["best_psl"], o["best_psl"]) and np.array_equal(ra["seq"], o["final_seq"])
    # a checkpoint of the PSL walk does not restore into an ISL context
    c = labs.Search(L, W, seed)
    with pytest.raises(labs.LabsError):
        c.restore(buf)
    for x in (a, b, c):
        x.close()


def test_psl_refusals():
    for f in (_native.LABS_FLAG_BEST_FIRST, _native.LABS_FLAG_LEARNED):
        with pytest.raises(labs.LabsError):
            labs.Search(41, 4, 1, objective="psl", flags=f)
    s = labs.Search(41, 4, 1, objective="psl")
    with pytest.raises(labs.LabsError):
        s.log(16)
    s.close()
    plain = labs.Search(41, 4, 1)
    plain.walk(5)
    for fn, args in ((plain.lib.labs_best_psl, (0, None, None, None, None, None)),
                     (plain.lib.labs_walker_psl, (0, 4, None, None))):
        assert fn(plain.ctx, *args) == _native.LABS_EINVAL
    assert plain.stats()["best_psl"] == -1
    plain.close()
