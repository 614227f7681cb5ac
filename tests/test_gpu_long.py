"""GPU parity of the long-sequence walk (LABS_MAX_L < L <= LABS_MAX_L_LONG, one walker
per CTA) against the oracle, whose walk has no length limit: per-step trace codes and
ISLs, best and final sequences, counters, bit-exact; chunking, graphs and mixed long
lengths; checkpoints; the long row kernels (ISL, neighbourhood) including the rows
outside the exact range; the combinations the library refuses."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import labs_inputs
import oracle
import paper_2011_00068_gb300 as labs
from paper_2011_00068_gb300 import _native

pytestmark = pytest.mark.gpu


def traced(L, walkers, steps, seed, **cfg):
    s = labs.Search(L, walkers, seed, **cfg)
    code, isl = s.trace(list(range(walkers)), steps)
    s.walk(steps)
    s.sync()
    return s, code.cpu().numpy(), isl.cpu().numpy()


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (513, 6, 400, {}),
    (601, 4, 300, {"tabu_log2": 4, "probe_cap": 3}),
    (1025, 4, 300, {"patience": 40}),
    (2047, 3, 120, {}),
    (4095, 2, 60, {}),
    (8191, 2, 16, {}),
    (11263, 1, 4, {}),
])
def test_long_trajectory_parity(L, walkers, steps, kw):
    seed = 6
    s, code, isl = traced(L, walkers, steps, seed, **kw)
    o = oracle.walk(L, seed, walkers, steps, trace=True, **kw)
    assert np.array_equal(code, o["trace_code"])
    assert np.array_equal(isl, o["trace_isl"])
    res = s.results(seqs=True)
    for k in ("best_isl", "target_step"):
        assert np.array_equal(res[k], o[k]), k
    assert np.array_equal(res["isl"], o["final_isl"])
    assert np.array_equal(res["seq"], o["final_seq"])
    assert np.array_equal(res["best_seq"], o["best_seq"])
    st = s.stats()
    assert st["walkers_per_warp"] == 0  # one walker per CTA
    assert st["steps"] == walkers * steps
    assert st["restarts"] == int(o["restarts"].sum())
    assert st["overflows"] == int(o["overflows"].sum())
    assert st["blocked"] == int((o["trace_code"] == -1).sum())
    g = int(np.argmin(o["best_isl"]))
    b = s.best()
    assert b["isl"] == o["best_isl"][g] and np.array_equal(b["seq"], o["best_seq"][g])
    assert b["hex"] == oracle.hex_encode(o["best_seq"][g])
    s.close()


def test_long_chunking_graphs_and_mixed_lengths():
    L, W, steps, seed = 1025, 4, 200, 5
    ref = None
    for cfg in ({}, {"chunk_steps": 7}, {"chunk_steps": 50, "flags": _native.LABS_FLAG_NO_GRAPH}):
        s, code, isl = traced(L, W, steps, seed, **cfg)
        if ref is None:
            ref = (code, isl)
        else:
            assert np.array_equal(code, ref[0]) and np.array_equal(isl, ref[1])
        s.close()
    o = oracle.walk(L, seed, W, steps, trace=True)
    assert np.array_equal(ref[0], o["trace_code"]) and np.array_equal(ref[1], o["trace_isl"])
    # several calls == one call; long lengths mixed in one launch
    Ls, counts = [601, 2001, 1025], [3, 2, 3]
    s = labs.Search(Ls, counts, 9)
    code, isl = s.trace(list(range(sum(counts))), 150)
    for part in (1, 70, 79):
        s.walk(part)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    first = 0
    for Lg, cnt in zip(Ls, counts):
        o = oracle.walk(Lg, 9, cnt, 150, first_walker=first, trace=True)
        assert np.array_equal(code[first:first + cnt], o["trace_code"]), Lg
        assert np.array_equal(isl[first:first + cnt], o["trace_isl"]), Lg
        first += cnt
    s.close()


def exact_limit(L):
    """The long kernels' exact-range bound on ISL: every value of the fp32 dISL
    assembly stays below 2^24 (restated from the library's derivation)."""
    n = (L + 1) // 2
    room = ((1 << 24) - 8 * L - 32 * n - 32) / 16
    return int(min(room * room / (n - 1), 2 ** 29)) - 1


@pytest.mark.parametrize("L", [513, 1025, 4095, 8191, 11263])
def test_long_rows(L):
    n = (L + 1) // 2
    xs = labs_inputs.random_free_vars(5, L, seed=L)
    rows = [oracle.skew_expand(x, L) for x in xs]
    rows.append(oracle.skew_expand(np.ones(n, np.int8), L))            # degenerate
    rows.append(oracle.skew_expand(np.array([(-1) ** i for i in range(n)], np.int8), L))
    bad = rows[0].copy()
    bad[L - 1] = -bad[L - 1]                                            # breaks Eq. 4
    rows.append(bad)
    R = np.stack(rows)
    dev = torch.from_numpy(R).cuda()
    d = labs.neighbor_delta(dev).cpu().numpy()
    e = labs.isl(dev).cpu().numpy()
    over = 0
    for k, r in enumerate(rows[:-1]):
        want = oracle.isl(r)
        assert e[k] == (want if want <= 2 ** 31 - 1 else -2), k
        if want > exact_limit(L):
            over += 1
            assert (d[k] == np.iinfo(np.int32).min).all(), k
        else:
            assert np.array_equal(d[k], oracle.neighbor_delta(r)), k
    assert (d[-1] == np.iinfo(np.int32).min).all()
    assert e[-1] == oracle.isl(bad)  # any +-1 row has an ISL
    if L >= 4095:
        assert over == 2  # both degenerate rows lie outside the exact range


def test_long_checkpoint_round_trip():
    L, W, seed = 1025, 3, 2
    a = labs.Search(L, W, seed)
    a.walk(60)
    buf = a.checkpoint(with_tabu=True)
    a.walk(90)
    ra = a.results(seqs=True)
    b = labs.Search(L, W, seed)
    b.restore(buf)
    b.walk(90)
    rb = b.results(seqs=True)
    for k in ("isl", "best_isl", "seq", "best_seq"):
        assert np.array_equal(ra[k], rb[k]), k
    o = oracle.walk(L, seed, W, 150)
    assert np.array_equal(ra["seq"], o["final_seq"]) and np.array_equal(ra["best_isl"], o["best_isl"])
    # a long checkpoint does not restore into a context of short walkers
    c = labs.Search(511, W, seed)
    with pytest.raises(labs.LabsError):
        c.restore(buf)
    for x in (a, b, c):
        x.close()


def test_long_refusals():
    with pytest.raises(labs.LabsError):
        labs.Search([201, 1025], [2, 2], 1)  # short and long lengths in one context
    with pytest.raises(labs.LabsError):
        labs.Search(_native.LABS_MAX_L_LONG + 2, 2, 1)
    BF = _native.LABS_FLAG_BEST_FIRST
    for f in (_native.LABS_FLAG_LEARNED, BF | _native.LABS_FLAG_SECOND_HASH):
        with pytest.raises(labs.LabsError):
            labs.Search(1025, 2, 1, flags=f)
    s = labs.Search(1025, 2, 1)
    with pytest.raises(labs.LabsError):
        s.log(4)
    s.close()
    s = labs.Search(1025, 2, 1, flags=BF)
    s.walk(3)
    with pytest.raises(labs.LabsError):
        s.checkpoint()
    with pytest.raises(labs.LabsError):
        s.walk(_native.LABS_BEST_FIRST_MAX_STEPS_LONG)
    s.close()


def test_long_walker_outside_exact_range_stops_with_erange():
    """A walker put (through a checkpoint) on a state whose ISL is above the exact-range
    bound stops before evaluating it and labs_sync reports LABS_ERANGE; the other walker
    is unaffected.  Checkpoint layout: 64-byte header, then the walker states (160 bytes
    each, ISL at byte 96), then the rows of current and best bits (176 words per walker,
    each array 256-byte aligned; n = 2048 here, so walker 0's bits are the row's first
    64 words)."""
    import struct

    L, W, seed = 4095, 2, 5
    s = labs.Search(L, W, seed)
    buf = s.checkpoint(with_tabu=False)
    hdr, state_bytes = 64, 160
    cur = hdr + ((W * state_bytes + 255) // 256) * 256
    buf[cur:cur + 256] = bytes(256)                       # walker 0: every free variable +1
    struct.pack_into("<i", buf, hdr + 96, 2 ** 31 - 1)    # its ISL as the kernel finds it (saturated)
    assert oracle.isl(oracle.skew_expand(np.ones((L + 1) // 2, np.int8), L)) > 2 ** 31 - 1
    s.restore(buf)
    s.walk(4)
    with pytest.raises(labs.LabsError) as err:
        s.sync()
    assert err.value.code == _native.LABS_ERANGE
    s.clear_stop()  # errors are sticky until cleared
    r = s.results(1, 1)
    o = oracle.walk(L, seed, 1, 4, first_walker=1)
    assert r["isl"][0] == o["final_isl"][0]
    s.close()


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (513, 3, 60, {}),
    (601, 2, 50, {"tabu_log2": 4, "probe_cap": 3}),
    (1025, 2, 12, {}),
])
def test_long_psl_parity(L, walkers, steps, kw):
    """The walk under the PSL objective for long sequences (one walker per CTA) against
    the oracle, which rebuilds every neighbour: traces, final and best sequences with
    their PSL and ISL, the best walker in the (PSL, ISL) order."""
    seed = 8
    s, code, isl = traced(L, walkers, steps, seed, objective="psl", **kw)
    o = oracle.walk(L, seed, walkers, steps, trace=True, objective="psl", **kw)
    assert np.array_equal(code, o["trace_code"])
    assert np.array_equal(isl, o["trace_isl"])
    res = s.results(seqs=True)
    for k, ok in (("best_isl", "best_isl"), ("best_psl", "best_psl"), ("isl", "final_isl"), ("psl", "final_psl")):
        assert np.array_equal(res[k], o[ok]), k
    assert np.array_equal(res["best_seq"], o["best_seq"])
    g = min(range(walkers), key=lambda j: (o["best_psl"][j], o["best_isl"][j], j))
    b = s.best()
    assert (b["psl"], b["isl"]) == (o["best_psl"][g], o["best_isl"][g])
    assert s.stats()["walkers_per_warp"] == 0
    s.close()


def test_long_psl_chunking_and_mixed_lengths():
    Ls, counts = [601, 1025], [2, 2]
    s = labs.Search(Ls, counts, 4, objective="psl", chunk_steps=5)
    code, isl = s.trace(list(range(4)), 14)
    for part in (3, 11):
        s.walk(part)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    first = 0
    for Lg, cnt in zip(Ls, counts):
        o = oracle.walk(Lg, 4, cnt, 14, first_walker=first, trace=True, objective="psl")
        assert np.array_equal(code[first:first + cnt], o["trace_code"]), Lg
        assert np.array_equal(isl[first:first + cnt], o["trace_isl"]), Lg
        first += cnt
    s.close()


@pytest.mark.parametrize("L,walkers,steps,kw", [
    (513, 3, 80, {}),
    (601, 2, 60, {"tabu_log2": 4, "probe_cap": 3}),
    (1025, 2, 40, {}),
    (2049, 1, 20, {}),
    (3001, 1, 12, {}),
    (4801, 1, 6, {}),
    (11263, 1, 3, {}),
])
def test_long_bestfirst_parity(L, walkers, steps, kw):
    """The best-first search (Algorithm 1 as printed) for long sequences, one walker per
    CTA (128 threads up to L = 2303, 256 at L = 3001, 512 at 4801 and 11263), against the
    oracle: per-step trace codes and ISLs, best and final sequences, counters."""
    seed = 3
    s, code, isl = traced(L, walkers, steps, seed, flags=_native.LABS_FLAG_BEST_FIRST, **kw)
    o = oracle.bestfirst(L, seed, walkers, steps, pq_size=_native.LABS_QUEUE_SIZE, trace=True, **kw)
    assert np.array_equal(code, o["trace_code"])
    assert np.array_equal(isl, o["trace_isl"])
    res = s.results(seqs=True)
    for k, ok in (("best_isl", "best_isl"), ("target_step", "target_step"), ("isl", "final_isl")):
        assert np.array_equal(res[k], o[ok]), k
    assert np.array_equal(res["seq"], o["final_seq"])
    assert np.array_equal(res["best_seq"], o["best_seq"])
    st = s.stats()
    assert st["steps"] == walkers * steps and st["walkers_per_warp"] == 0
    assert st["restarts"] == int(o["restarts"].sum())
    assert st["overflows"] == int(o["overflows"].sum())
    assert st["blocked"] == int((o["trace_code"] == -1).sum())
    s.close()


def test_long_bestfirst_chunking_and_mixed_lengths():
    """The queue survives the ends of chunks and of labs_walk calls: the same traces
    with 5-step chunks over three calls, two lengths in one launch."""
    Ls, counts = [601, 1025], [2, 2]
    s = labs.Search(Ls, counts, 6, flags=_native.LABS_FLAG_BEST_FIRST, chunk_steps=5)
    code, isl = s.trace(list(range(4)), 30)
    for part in (3, 11, 16):
        s.walk(part)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    first = 0
    for Lg, cnt in zip(Ls, counts):
        o = oracle.bestfirst(Lg, 6, cnt, 30, pq_size=_native.LABS_QUEUE_SIZE, first_walker=first, trace=True)
        assert np.array_equal(code[first:first + cnt], o["trace_code"]), Lg
        assert np.array_equal(isl[first:first + cnt], o["trace_isl"]), Lg
        first += cnt
    s.close()


@pytest.mark.parametrize("mode", ["walk", "psl", "bestfirst"])
@pytest.mark.parametrize("L_long,R", [(2311, 5), (11263, 11)])
def test_long_kernels_on_short_walkers(mode, L_long, R):
    """The kernels chosen for a context's longest length run all its walkers, so the
    L = 601 walkers of a context whose longest length is 2311 (256-thread CTAs, lane
    block 5) or 11263 (512 threads, lane block 11) exercise those kernels at a length
    where the oracle is fast (under the PSL objective it rebuilds every neighbour in
    O(L^2)): their traces against the oracle, and the long walker's final and best
    values against the oracle's Eq. 2 and PSL of its sequences."""
    Ls, counts, seed, steps = [601, L_long], [2, 1], 12, 16
    cfg = {"objective": "psl"} if mode == "psl" else {}
    if mode == "bestfirst":
        cfg["flags"] = _native.LABS_FLAG_BEST_FIRST
    s = labs.Search(Ls, counts, seed, **cfg)
    assert s.stats()["lane_block"] == R
    code, isl = s.trace([0, 1], steps)
    s.walk(steps)
    s.sync()
    code, isl = code.cpu().numpy(), isl.cpu().numpy()
    if mode == "bestfirst":
        o = oracle.bestfirst(601, seed, 2, steps, pq_size=_native.LABS_QUEUE_SIZE, trace=True)
    else:
        o = oracle.walk(601, seed, 2, steps, trace=True, objective="psl" if mode == "psl" else "isl")
    assert np.array_equal(code, o["trace_code"]) and np.array_equal(isl, o["trace_isl"])
    r = s.results(0, 2, seqs=True)
    assert np.array_equal(r["seq"], o["final_seq"]) and np.array_equal(r["best_isl"], o["best_isl"])
    r = s.results(2, 1, seqs=True)
    assert r["isl"][0] == oracle.isl(r["seq"][0]) and r["best_isl"][0] == oracle.isl(r["best_seq"][0])
    if mode == "psl":
        assert r["psl"][0] == oracle.psl(r["seq"][0]) and r["best_psl"][0] == oracle.psl(r["best_seq"][0])
        assert (r["best_psl"][0], r["best_isl"][0]) <= (r["psl"][0], r["isl"][0])
    else:
        assert r["best_isl"][0] <= r["isl"][0]
    s.close()
