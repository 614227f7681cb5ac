"""Pins of the oracle's walk (Algorithm 1, self-avoiding form with restarts).

The paper prints no trajectory, so the walk is pinned against a second statement of
the same rules in tests/pyref.py, whose dISL comes from flip-and-recompute (numpy)
instead of the oracle's two-position formula, and against invariants that any
correct walk keeps.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import pyref


@pytest.mark.parametrize("L,steps,log2,cap,patience",
                         [(13, 300, 16, 32, 0), (21, 400, 16, 32, 0), (21, 300, 4, 3, 7),
                          (5, 60, 16, 32, 0), (41, 250, 16, 32, 0), (601, 40, 16, 32, 0)])
def test_walk_matches_python_statement(L, steps, log2, cap, patience):
    seed = 1
    out = oracle.walk(L, seed, 3, steps, tabu_log2=log2, probe_cap=cap, patience=patience,
                      trace=True, nthreads=2)
    for g in range(3):
        codes, isls, best, restarts = pyref.walk(L, seed, g, steps, log2, cap, patience)
        assert list(out["trace_code"][g]) == codes
        assert list(out["trace_isl"][g]) == isls
        assert out["best_isl"][g] == best
        assert out["restarts"][g] == restarts


def test_small_table_exercises_overflow_and_full_neighbourhood():
    """A 16-slot HT with 3 probes overflows and blocks whole neighbourhoods, so both
    restart paths (-1 codes and the restart bit) occur and still agree."""
    out = oracle.walk(21, 9, 2, 400, tabu_log2=4, probe_cap=3, trace=True, nthreads=1)
    codes = out["trace_code"]
    assert (out["overflows"] > 0).any()
    assert ((codes & oracle.TRACE_RESTART) != 0).any()
    for g in range(2):
        c, i, b, r = pyref.walk(21, 9, g, 400, 4, 3, 0)
        assert list(codes[g]) == c and list(out["trace_isl"][g]) == i


def test_walk_invariants_L201():
    """L = 201: every ISL in the trace is the recomputed ISL of a skew state (checked
    at the end), best <= every traced ISL, best sequence reproduces best ISL, the
    walk is reproducible and independent of the thread count."""
    L, steps = 201, 600
    a = oracle.walk(L, 7, 4, steps, trace=True, nthreads=4)
    b = oracle.walk(L, 7, 4, steps, trace=True, nthreads=1)
    for k in ("trace_code", "trace_isl", "best_isl", "final_isl", "best_seq"):
        assert np.array_equal(a[k], b[k])
    n = (L + 1) // 2
    for g in range(4):
        assert a["best_isl"][g] <= a["trace_isl"][g].min()
        assert oracle.isl(a["best_seq"][g]) == a["best_isl"][g]
        assert oracle.isl(a["final_seq"][g]) == a["final_isl"][g] == a["trace_isl"][g][-1]
        assert oracle.is_skew(a["final_seq"][g])
        assert (a["trace_isl"][g] % 8 == (n - 1) % 8).all()
        flips = a["trace_code"][g]
        moved = flips[flips >= 0] & 0xFFFF
        assert (moved < n).all()
    # walkers are independent: walker 2 alone equals walker 2 of the batch
    c = oracle.walk(L, 7, 1, steps, first_walker=2, trace=True)
    assert np.array_equal(c["trace_isl"][0], a["trace_isl"][2])


def test_stagnation_restart_interval():
    """With patience P and a large HT (no overflow), a step ends in a restart exactly
    when it is the P-th consecutive step without a new best since the last restart."""
    L, P, steps = 21, 9, 500
    out = oracle.walk(L, 3, 1, steps, patience=P, trace=True)
    assert out["overflows"][0] == 0
    codes, isls = out["trace_code"][0], out["trace_isl"][0]
    since = oracle.isl(oracle.skew_expand(oracle.random_start(3, 0, 0, L), L))
    stag = 0
    saw_restart = False
    for t in range(steps):
        c = int(codes[t])
        if c == -1:  # whole neighbourhood visited: restart without a move
            since, stag = int(isls[t]), 0
            continue
        if c & oracle.TRACE_RESTART:
            # the move did not improve (else stag resets) and it was the P-th such step
            assert stag == P - 1
            since, stag = int(isls[t]), 0
            saw_restart = True
            continue
        e = int(isls[t])
        if e < since:
            since, stag = e, 0
        else:
            stag += 1
        assert stag < P
    assert saw_restart


# ------------------------------------------------------ best-first search (Alg. 1)

@pytest.mark.parametrize("L,steps,K,log2,cap", [(13, 300, 3, 16, 32), (21, 300, 32, 16, 32), (21, 400, 5, 4, 3),
                                                (41, 200, 32, 16, 32), (5, 80, 2, 16, 32), (601, 25, 32, 16, 32)])
def test_bestfirst_matches_python_statement(L, steps, K, log2, cap):
    """The queue rules (order, eviction of the last entry, discarding entries that
    became S, restarts) against the Python statement, whose dISL is flip-and-recompute."""
    seed = 2
    out = oracle.bestfirst(L, seed, 3, steps, pq_size=K, tabu_log2=log2, probe_cap=cap, trace=True, nthreads=2)
    for g in range(3):
        codes, isls, best, restarts, overflows, _ = pyref.bestfirst(L, seed, g, steps, K, log2, cap)
        assert list(out["trace_code"][g]) == codes
        assert list(out["trace_isl"][g]) == isls
        assert out["best_isl"][g] == best
        assert out["restarts"][g] == restarts and out["overflows"][g] == overflows


@pytest.mark.parametrize("L", [21, 41, 61])
def test_bestfirst_with_a_queue_of_one_is_the_walk(L):
    """With K = 1 the queue holds only the best neighbour not in HT, which is what the
    walk moves to: the two searches coincide when the walk never restarts on stagnation."""
    a = oracle.walk(L, 3, 6, 1500, patience=1 << 30, trace=True)
    b = oracle.bestfirst(L, 3, 6, 1500, pq_size=1, trace=True)
    for k in ("trace_isl", "final_seq", "best_seq", "best_isl", "restarts", "overflows"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["trace_code"] == -1, b["trace_code"] == -1)


def test_bestfirst_with_an_unbounded_queue_expands_every_state_once():
    """L = 21 (2^11 skew states) with K >= 2^11: no entry is ever dropped, so every
    state becomes S exactly once, the queue runs empty after step 2^11, and the best
    found is the exhaustive optimum."""
    L, n = 21, 11
    opt = oracle.enumerate_skew(L)[0]
    out = oracle.bestfirst(L, 5, 2, 2 ** n + 10, pq_size=4096, trace=True)
    for g in range(2):
        codes = out["trace_code"][g]
        assert int(np.argmax(codes == -1)) + 1 == 2 ** n
        assert (codes[: 2 ** n - 1] >= 0).all()
        assert out["best_isl"][g] == opt
        assert oracle.isl(out["best_seq"][g]) == opt


def test_bestfirst_invariants_L201():
    L, steps = 201, 300
    a = oracle.bestfirst(L, 7, 4, steps, pq_size=32, trace=True, nthreads=4)
    b = oracle.bestfirst(L, 7, 4, steps, pq_size=32, trace=True, nthreads=1)
    n = (L + 1) // 2
    for k in ("trace_code", "trace_isl", "best_isl", "final_isl", "best_seq"):
        assert np.array_equal(a[k], b[k])
    for g in range(4):
        assert a["best_isl"][g] <= a["trace_isl"][g].min()
        assert oracle.isl(a["best_seq"][g]) == a["best_isl"][g]
        assert oracle.isl(a["final_seq"][g]) == a["final_isl"][g] == a["trace_isl"][g][-1]
        assert (a["trace_isl"][g] % 8 == (n - 1) % 8).all()
        assert (oracle.fingerprint(a["final_seq"][g]) & 0xFFFF) == a["trace_code"][g][-1]


# ------------------------------------------------------------ PSL objective walk

@pytest.mark.parametrize("L,steps,log2,cap,patience",
                         [(13, 200, 16, 32, 0), (21, 250, 16, 32, 0), (21, 300, 4, 3, 7),
                          (5, 60, 16, 32, 0), (3, 20, 16, 32, 0), (41, 150, 16, 32, 0), (601, 12, 16, 32, 0)])
def test_psl_walk_matches_python_statement(L, steps, log2, cap, patience):
    """Candidate order (PSL, ISL, i), best and stagnation on (PSL, ISL) pairs, against
    the Python statement, whose PSL and ISL come from numpy's correlate."""
    seed = 4
    out = oracle.walk(L, seed, 3, steps, tabu_log2=log2, probe_cap=cap, patience=patience,
                      trace=True, nthreads=2, objective="psl")
    for g in range(3):
        codes, isls, best, restarts = pyref.walk_psl(L, seed, g, steps, log2, cap, patience)
        assert list(out["trace_code"][g]) == codes
        assert list(out["trace_isl"][g]) == isls
        assert (out["best_psl"][g], out["best_isl"][g]) == best
        assert out["restarts"][g] == restarts


def test_psl_walk_reaches_barker_13():
    """The Barker sequence of length 13 is skew-symmetric with PSL 1, the lowest PSL any
    sequence can have; an exhaustive pass over the 2^7 skew states finds exactly it, its
    reversal and their negations, and every PSL walker ends at one of them."""
    L, n = 13, 7
    barker = np.array([1 if ch == "+" else -1 for ch in "+++++--++-+-+"], dtype=np.int8)
    family = [barker, -barker, barker[::-1].copy(), -barker[::-1]]
    psl1 = []
    for a in range(1 << n):
        x = np.array([-1 if (a >> i) & 1 else 1 for i in range(n)], dtype=np.int8)
        s = oracle.skew_expand(x, L)
        if oracle.psl(s) == 1:
            psl1.append(s)
    assert len(psl1) == 4
    assert all(any(np.array_equal(s, b) for b in family) for s in psl1)
    out = oracle.walk(L, 11, 4, 300, objective="psl")
    for g in range(4):
        assert out["best_psl"][g] == 1
        assert oracle.psl(out["best_seq"][g]) == 1
        assert any(np.array_equal(out["best_seq"][g], s) for s in psl1)


def test_psl_walk_invariants_L101():
    L, steps = 101, 120
    a = oracle.walk(L, 7, 3, steps, trace=True, nthreads=3, objective="psl")
    b = oracle.walk(L, 7, 3, steps, trace=True, nthreads=1, objective="psl")
    for k in ("trace_code", "trace_isl", "best_isl", "best_psl", "final_isl", "best_seq"):
        assert np.array_equal(a[k], b[k])
    n = (L + 1) // 2
    for g in range(3):
        assert oracle.psl(a["best_seq"][g]) == a["best_psl"][g]
        assert oracle.isl(a["best_seq"][g]) == a["best_isl"][g]
        assert oracle.psl(a["final_seq"][g]) == a["final_psl"][g]
        assert oracle.isl(a["final_seq"][g]) == a["final_isl"][g] == a["trace_isl"][g][-1]
        assert oracle.is_skew(a["final_seq"][g])
        assert (a["trace_isl"][g] % 8 == (n - 1) % 8).all()
    # the PSL walk ends at a lower PSL than the ISL walk's best sequences, on average
    c = oracle.walk(L, 7, 3, steps)
    assert a["best_psl"].mean() < c["best_psl"].mean()


# ------------------------------------------ best-first search with xLastovka's second table

@pytest.mark.parametrize("L,steps,K,log2", [(21, 300, 32, 16), (21, 300, 5, 4), (41, 200, 32, 16),
                                            (13, 300, 3, 6)])
def test_bestfirst_second_table_matches_python_statement(L, steps, K, log2):
    """Skipping the neighbours the second table holds, inserting every evaluated one with
    the larger-word rule, and emptying it with HT at restarts, against the Python
    statement; the skips happen (cycles are frequent on the skew-symmetric space)."""
    seed = 3
    out = oracle.bestfirst(L, seed, 3, steps, pq_size=K, tabu_log2=log2, trace=True, second_hash=True)
    for g in range(3):
        codes, isls, best, restarts, overflows, hits = pyref.bestfirst(L, seed, g, steps, K, log2, 32, second=True)
        assert list(out["trace_code"][g]) == codes
        assert list(out["trace_isl"][g]) == isls
        assert out["best_isl"][g] == best and out["restarts"][g] == restarts
        assert out["overflows"][g] == overflows and out["cache_hits"][g] == hits
    assert out["cache_hits"].sum() > 0


def test_bestfirst_second_table_without_hits_is_the_search():
    """A neighbour is only ever skipped when the table holds it, so when no skip occurs
    (a single step from each start, i.e. before anything was inserted) the two searches
    agree; over a run the table changes the trajectory and saves evaluations."""
    L = 41
    a = oracle.bestfirst(L, 5, 4, 1, trace=True)
    b = oracle.bestfirst(L, 5, 4, 1, trace=True, second_hash=True)
    assert (b["cache_hits"] == 0).all()
    for k in ("trace_code", "trace_isl", "best_isl"):
        assert np.array_equal(a[k], b[k])
    c = oracle.bestfirst(L, 5, 4, 400, second_hash=True)
    assert (c["cache_hits"] > 0).all()


@pytest.mark.parametrize("objective", ["isl", "psl"])
@pytest.mark.parametrize("L,walkers,steps,log2,cap", [(21, 4, 600, 4, 3), (41, 4, 800, 16, 32),
                                                       (101, 3, 600, 6, 9), (201, 2, 500, 16, 32)])
def test_walk_never_moves_straight_back(objective, L, walkers, steps, log2, cap):
    """The state a walker has just left is in HT (every state since the walker's start is
    inserted, and a failed insertion restarts it), so the walk never flips the same free
    variable twice in a row within one run between restarts: the fact that lets the GPU's
    lockstep steps leave that move out without probing it.  Small tables, whose
    insertions overflow and whose neighbourhoods fill, keep it too."""
    out = oracle.walk(L, 5, walkers, steps, tabu_log2=log2, probe_cap=cap, trace=True, nthreads=2,
                      objective=objective)
    codes = out["trace_code"]
    moves_back = 0
    pairs = 0
    for g in range(walkers):
        for t in range(1, steps):
            a, b = int(codes[g, t - 1]), int(codes[g, t])
            if a < 0 or (a & oracle.TRACE_RESTART) or b < 0:
                continue  # the step before ended in a restart: a fresh state, no move to undo
            pairs += 1
            moves_back += (a & 0xFFFF) == (b & 0xFFFF)
    assert pairs > steps // 2 and moves_back == 0
