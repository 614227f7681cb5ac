"""Parity at the workload sizes the benchmark runs, in the launch configuration it
times, on walkers the oracle can replay one by one (bit-exact integers).

config 1: L=41, 64 walkers x 1e5 steps, seed 1: every step of every walker.
config 2: L=201, 16384 walkers x 1e4 steps, seed 7 (the bench step): 48 walkers
          spread over the batch, final/best ISL, best sequence, time-to-target step.
config 3: the 52 odd lengths 201..303, 2048 walkers each, 5e3 steps, one launch:
          64 walkers per length (3,328 oracle walkers; LABS_PARITY_PER_L sets
          another count).
largest length: L=501 (the largest length of the scale-up configuration), 8192
          walkers x 2000 steps.
best-first search: the config-2 workload with LABS_FLAG_BEST_FIRST (bench.py
          --search bestfirst), 24 walkers spread over the batch.
short lengths: L=151 (four walkers per warp), 16384 walkers x 1e4 steps, 24 walkers.
PSL objective: the config-2 workload with LABS_FLAG_PSL, 3 walkers.
long sequences: L=4095, 608 walkers x 512 steps (bench.py --config long), 3 walkers.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import paper_2011_00068_gb300 as labs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def oracle_walkers(jobs):
    """Oracle runs of single walkers (L, seed, steps, walker id), one per host thread
    (the oracle releases the interpreter lock while it runs)."""
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(lambda j: oracle.walk(j[0], j[1], 1, j[2], first_walker=j[3], nthreads=1), jobs))


def check_sample(s, L, seed, steps, ids, bestfirst=False):
    if bestfirst:
        with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
            outs = list(ex.map(lambda g: oracle.bestfirst(L, seed, 1, steps, first_walker=g, nthreads=1), ids))
    else:
        outs = oracle_walkers([(L, seed, steps, gid) for gid in ids])
    for gid, o in zip(ids, outs):
        r = s.results(gid, 1, seqs=True)
        assert r["isl"][0] == o["final_isl"][0], gid
        assert r["best_isl"][0] == o["best_isl"][0], gid
        assert np.array_equal(r["best_seq"][0], o["best_seq"][0]), gid
        assert r["target_step"][0] == o["target_step"][0], gid


def test_config1_L41_full_trajectories():
    L, W, steps, seed = 41, 64, 100_000, 1
    s = labs.Search(L, W, seed)
    code, isl = s.trace(list(range(W)), steps)
    s.walk(steps)
    s.sync()
    o = oracle.walk(L, seed, W, steps, trace=True)
    assert np.array_equal(code.cpu().numpy(), o["trace_code"])
    assert np.array_equal(isl.cpu().numpy(), o["trace_isl"])
    assert int(o["best_isl"].min()) == 108  # the walk reaches the L=41 optimum


def test_config2_L201_bench_shape():
    L, W, steps, seed = 201, 16384, 10_000, 7
    s = labs.Search(L, W, seed)
    s.walk(steps)
    s.sync()
    st = s.stats()
    assert st["steps"] == W * steps and st["overflows"] == 0
    ids = sorted({0, 1, W - 1} | set(list(range(97, W, 353))[:45]))
    check_sample(s, L, seed, steps, ids)
    b = s.best()
    assert oracle.isl(b["seq"]) == b["isl"] == st["best_isl"]


def test_config3_mixed_lengths_one_launch():
    Ls = list(range(201, 304, 2))
    per, steps, seed = 2048, 5000, 7
    s = labs.Search(Ls, [per] * len(Ls), seed)
    s.walk(steps)
    s.sync()
    k = int(os.environ.get("LABS_PARITY_PER_L", "64"))
    rng = np.random.default_rng(3)
    jobs = []
    for g, L in enumerate(Ls):
        jobs += [(L, seed, steps, g * per + int(j)) for j in rng.choice(per, k, replace=False)]
    outs = oracle_walkers(jobs)
    for (L, _, _, gid), o in zip(jobs, outs):
        r = s.results(gid, 1, seqs=True)
        assert r["isl"][0] == o["final_isl"][0], (L, gid)
        assert r["best_isl"][0] == o["best_isl"][0], (L, gid)
        assert np.array_equal(r["best_seq"][0], o["best_seq"][0]), (L, gid)


def test_largest_length_L501():
    L, W, steps, seed = 501, 8192, 2000, 42
    s = labs.Search(L, W, seed)
    s.walk(steps)
    s.sync()
    check_sample(s, L, seed, steps, [0, 4095, W - 1])


def test_bestfirst_L201_bench_shape():
    from paper_2011_00068_gb300 import _native

    L, W, steps, seed = 201, 16384, 10_000, 7
    s = labs.Search(L, W, seed, flags=_native.LABS_FLAG_BEST_FIRST)
    s.walk(steps)
    s.sync()
    st = s.stats()
    assert st["steps"] == W * steps
    ids = sorted({0, W - 1} | set(list(range(211, W, 719))[:22]))
    check_sample(s, L, seed, steps, ids, bestfirst=True)
    b = s.best()
    assert oracle.isl(b["seq"]) == b["isl"] == st["best_isl"]


def test_four_walkers_per_warp_L151_bench_shape():
    L, W, steps, seed = 151, 16384, 10_000, 7
    s = labs.Search(L, W, seed)
    s.walk(steps)
    s.sync()
    st = s.stats()
    assert st["steps"] == W * steps and st["walkers_per_warp"] == 4
    ids = sorted({0, 3, W - 1} | set(list(range(5, W, 701))[:21]))
    check_sample(s, L, seed, steps, ids)


def test_psl_L201_bench_shape():
    """The PSL-objective walk on the config-2 workload (bench.py --search psl): walkers
    0, 8191 and 16383 against the oracle, which rebuilds every neighbour (about 20 s of
    host time per walker for 1e4 steps)."""
    L, W, steps, seed = 201, 16384, 10_000, 7
    s = labs.Search(L, W, seed, objective="psl")
    s.walk(steps)
    s.sync()
    ids = [0, 8191, W - 1]
    with ThreadPoolExecutor(max_workers=len(ids)) as ex:
        outs = list(ex.map(lambda g: oracle.walk(L, seed, 1, steps, first_walker=g, nthreads=1, objective="psl"),
                           ids))
    for gid, o in zip(ids, outs):
        r = s.results(gid, 1, seqs=True)
        for k, ok in (("isl", "final_isl"), ("psl", "final_psl"), ("best_isl", "best_isl"),
                      ("best_psl", "best_psl")):
            assert r[k][0] == o[ok][0], (gid, k)
        assert np.array_equal(r["best_seq"][0], o["best_seq"][0]), gid
    b = s.best()
    assert oracle.psl(b["seq"]) == b["psl"] and oracle.isl(b["seq"]) == b["isl"]


def test_long_L4095_bench_shape():
    """Long sequences at the size bench.py --config long runs (608 walkers x 512 steps
    of L=4095, 256-thread CTAs): walkers 0, 303 and 607 against the oracle."""
    L, W, steps, seed = 4095, 608, 512, 42
    s = labs.Search(L, W, seed)
    s.walk(steps)
    s.sync()
    assert s.stats()["steps"] == W * steps
    check_sample(s, L, seed, steps, [0, 303, W - 1])
