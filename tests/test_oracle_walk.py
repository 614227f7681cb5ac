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
                          (5, 60, 16, 32, 0), (41, 250, 16, 32, 0)])
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
