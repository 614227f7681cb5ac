"""The candidate rounds of the lockstep walk steps, restated in Python and checked against
the sequential rule of Algorithm 1's visited-set test on random and adversarial tables.

The sequential rule (the oracle's, and walk_psl's): take the candidates in ascending key
order; probe each one's HT chain from its home slot, up to `cap` slots, stopping at the
first slot that is empty, of an older generation, or holds the candidate's tag; the
candidate is visited when that slot holds its tag; the first candidate that is not
visited is taken, and its insertion slot is the slot where its probe stopped (none when
the probe found no stopping slot within `cap`, an overflow).

The lockstep kernels (walk_lockstep, walk_psl_lockstep) take the two lowest keys above a
floor per round and probe the first S slots of each with one load per lane; a candidate
whose first S slots hold no stopping slot gets a full probe when cap > S (the second one
only when the first is visited), and is free without a slot when cap <= S; when both are
visited the floor moves to the second key.  This test checks, for every table, that the
rounds take the same key and the same insertion slot as the sequential rule.
"""
from __future__ import annotations

import numpy as np
import pytest

GEN_MASK = 0xFFFFF


def tag(f, gen):
    return (f & ~GEN_MASK) | gen


def stops(e, f, gen):
    return (e & GEN_MASK) != gen or e == tag(f, gen)


def probe_full(T, f, gen, cap):
    """Sequential linear probe: (visited, slot or -1)."""
    m = len(T)
    for s in range(cap):
        e = T[(f + s) % m]
        if stops(e, f, gen):
            return e == tag(f, gen), (f + s) % m
    return False, -1


def sequential(keys, fps, T, gen, cap):
    for k in sorted(keys):
        visited, slot = probe_full(T, fps[k], gen, cap)
        if not visited:
            return k, slot
    return None, -1


def rounds(keys, fps, T, gen, cap, S):
    """The kernel's rounds for one walker (the lanes' work written out per candidate)."""
    m = len(T)
    floor = -1
    while True:
        above = sorted(k for k in keys if k > floor)
        k0 = above[0] if above else None
        k1 = above[1] if len(above) > 1 else None

        def partial(k):
            # lanes 0..S-1 (or S..2S-1) each load one of the first S slots (those < cap)
            hits = [s for s in range(min(S, cap)) if stops(T[(fps[k] + s) % m], fps[k], gen)]
            if hits:
                first = hits[0]
                e = T[(fps[k] + first) % m]
                return ("visited" if e == tag(fps[k], gen) else "free"), (fps[k] + first) % m
            return ("unknown" if cap > S else "free"), -1

        st0, sl0 = partial(k0) if k0 is not None else ("none", -1)
        st1, sl1 = partial(k1) if k1 is not None else ("none", -1)
        if st0 == "unknown":
            v, sl0 = probe_full(T, fps[k0], gen, cap)
            st0 = "visited" if v else "free"
        if st0 == "visited" and st1 == "unknown":
            v, sl1 = probe_full(T, fps[k1], gen, cap)
            st1 = "visited" if v else "free"
        if st0 == "free":
            return k0, sl0
        if st0 == "none" or st1 == "none":
            return None, -1
        if st1 == "free":
            return k1, sl1
        floor = k1


def random_case(rng, n, m, cap, density, adversarial):
    gen = int(rng.integers(1, GEN_MASK))
    keys = [int(x) for x in rng.choice(1 << 20, size=n, replace=False)]
    fps = {k: int(rng.integers(0, 1 << 62)) << 1 for k in keys}
    T = [0] * m
    # other states of this generation, older generations, and empty slots
    for s in range(m):
        r = rng.random()
        if r < density:
            T[s] = tag(int(rng.integers(0, 1 << 62)) << 1, gen)
        elif r < density + 0.1:
            T[s] = tag(int(rng.integers(0, 1 << 62)) << 1, max(1, gen - 1))
    # some candidates visited: their tag in their chain, behind occupied slots
    for k in keys:
        if rng.random() < (0.8 if adversarial else 0.3):
            depth = int(rng.integers(0, min(cap, 3 * 8)))
            home = fps[k] % m
            for d in range(depth):
                if (T[(home + d) % m] & GEN_MASK) != gen:
                    T[(home + d) % m] = tag(int(rng.integers(0, 1 << 62)) << 1, gen)
            T[(home + depth) % m] = tag(fps[k], gen)
    return keys, fps, T, gen


@pytest.mark.parametrize("S", [4, 8, 16])
@pytest.mark.parametrize("cap", [1, 3, 8, 9, 16, 32])
def test_rounds_equal_sequential_rule(S, cap):
    rng = np.random.default_rng(1000 * S + cap)
    for trial in range(150):
        n = int(rng.integers(1, 40))
        m = int(rng.choice([16, 64, 256]))
        density = float(rng.choice([0.0, 0.3, 0.7, 0.95]))
        keys, fps, T, gen = random_case(rng, n, m, cap, density, adversarial=trial % 3 == 0)
        assert rounds(keys, fps, T, gen, cap, S) == sequential(keys, fps, T, gen, cap), (S, cap, trial)


def test_every_neighbour_visited_blocks():
    """All candidates in HT: no key is taken, in both forms."""
    rng = np.random.default_rng(5)
    keys = list(range(10, 30))
    fps = {k: int(rng.integers(0, 1 << 40)) << 1 for k in keys}
    T = [0] * 64
    gen = 3
    for k in keys:
        home = fps[k] % 64
        s = 0
        while (T[(home + s) % 64] & GEN_MASK) == gen:
            s += 1
        T[(home + s) % 64] = tag(fps[k], gen)
    assert sequential(keys, fps, T, gen, 32)[0] is None
    for S in (4, 8, 16):
        assert rounds(keys, fps, T, gen, 32, S) == (None, -1)


def test_model_tells_rules_apart():
    """A planted slip, probing only the best candidate per round and taking it when its
    first slot is taken by another state, disagrees with the sequential rule: the model
    comparison can fail."""
    keys = [1, 2]
    fps = {1: 2 << 20, 2: (6 << 20) | 8}   # home slots 0 and 8
    gen = 5
    T = [0] * 16
    home1 = fps[1] % 16
    T[home1] = tag(12345 << 21, gen)       # another state of this generation
    T[(home1 + 1) % 16] = tag(fps[1], gen)  # candidate 1 visited, one slot deep
    assert sequential(keys, fps, T, gen, 32) == (2, 8)
    assert rounds(keys, fps, T, gen, 32, 8) == (2, 8)

    def slip(keys, fps, T, gen, cap):
        k = min(keys)
        e = T[fps[k] % len(T)]
        return (k, fps[k] % len(T)) if e != tag(fps[k], gen) else (max(keys), -1)

    assert slip(keys, fps, T, gen, 32) != sequential(keys, fps, T, gen, 32)
