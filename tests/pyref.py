"""Second, pure-Python statements of a few oracle parts, written independently of
oracle/labs_oracle.c, used only to pin the oracle in the CPU tests.

* ISL through numpy's correlate (a library routine) instead of Eq. 1 loops.
* Philox4x32-10 in Python integers (Salmon et al., SC'11).
* The walk of Algorithm 1 (self-avoiding form) with dISL by flip-and-recompute, not
  by the two-position formula the oracle uses.
* The same walk under the PSL objective, with PSL and ISL of every neighbour from
  numpy's correlate.
"""
from __future__ import annotations

import numpy as np

MASK32 = 0xFFFFFFFF


def isl_np(s) -> int:
    s = np.asarray(s, dtype=np.int64)
    L = s.size
    full = np.correlate(s, s, mode="full")  # index L-1+k holds C_k
    side = full[L:]
    return int(np.dot(side, side))


def psl_np(s) -> int:
    s = np.asarray(s, dtype=np.int64)
    L = s.size
    side = np.correlate(s, s, mode="full")[L:]
    return int(np.abs(side).max()) if side.size else 0


def philox(ctr, key):
    x = [int(v) & MASK32 for v in ctr]
    k = [int(v) & MASK32 for v in key]
    for r in range(10):
        if r:
            k = [(k[0] + 0x9E3779B9) & MASK32, (k[1] + 0xBB67AE85) & MASK32]
        p0 = 0xD2511F53 * x[0]
        p1 = 0xCD9E8D57 * x[2]
        x = [((p1 >> 32) ^ x[1] ^ k[0]) & MASK32, p1 & MASK32,
             ((p0 >> 32) ^ x[3] ^ k[1]) & MASK32, p0 & MASK32]
    return x


def skew(x, L):
    n = (L + 1) // 2
    c = n - 1
    s = np.zeros(L, dtype=np.int64)
    s[:n] = x
    for j in range(1, n):
        s[c + j] = -s[c - j] if j % 2 else s[c - j]
    return s


def start_vars(seed, g, r, L):
    n = (L + 1) // 2
    x = np.zeros(n, dtype=np.int64)
    for i in range(n):
        blk = philox([g, r, i // 128, 0], [seed & MASK32, seed >> 32])
        w = blk[(i // 32) % 4]
        x[i] = -1 if (w >> (i % 32)) & 1 else 1
    return x


def zkey(L, i):
    o = philox([i, L, 0, 2], [0x1BADB002, 0x2011A068])
    return o[0] | (o[1] << 32)


GEN = 0xFFFFF


class HT:
    def __init__(self, log2, cap):
        self.size = 1 << log2
        self.slot = [0] * self.size
        self.cap = min(cap, self.size)
        self.gen = 1

    def contains(self, fp):
        tag = (fp & ~GEN & 0xFFFFFFFFFFFFFFFF) | self.gen
        for p in range(self.cap):
            e = self.slot[(fp + p) % self.size]
            if e & GEN != self.gen:
                return False
            if e == tag:
                return True
        return False

    def insert(self, fp):
        tag = (fp & ~GEN & 0xFFFFFFFFFFFFFFFF) | self.gen
        for p in range(self.cap):
            j = (fp + p) % self.size
            e = self.slot[j]
            if e & GEN != self.gen:
                self.slot[j] = tag
                return True
            if e == tag:
                return True
        return False

    def new_generation(self):
        self.gen += 1
        if self.gen > GEN:
            self.slot = [0] * self.size
            self.gen = 1


def walk(L, seed, g, steps, tabu_log2=16, cap=32, patience=0):
    """Returns (trace_code, trace_isl, best_isl, restarts) for walker g."""
    n = (L + 1) // 2
    patience = patience or 2 * n
    keys = [zkey(L, i) for i in range(n)]
    ht = HT(tabu_log2, cap)
    st = {"r": 0, "best": None, "restarts": 0}

    def fp_of(s):
        f = 0
        for i in range(n):
            if s[i] < 0:
                f ^= keys[i]
        return f

    def begin():
        s = skew(start_vars(seed, g, st["r"], L), L)
        e = isl_np(s)
        f = fp_of(s)
        ht.insert(f)
        if st["best"] is None or e < st["best"]:
            st["best"] = e
        return s, e, f, e, 0

    s, e, f, since, stag = begin()
    codes, isls = [], []
    for _ in range(steps):
        deltas = []
        for i in range(n):
            t = s.copy()
            t[i] = -t[i]
            if L - 1 - i != i:
                t[L - 1 - i] = -t[L - 1 - i]
            deltas.append(isl_np(t) - e)
        order = sorted(range(n), key=lambda i: (deltas[i], i))
        chosen = None
        for i in order:
            if not ht.contains(f ^ keys[i]):
                chosen = i
                break
        if chosen is None:
            st["r"] += 1
            st["restarts"] += 1
            ht.new_generation()
            s, e, f, since, stag = begin()
            codes.append(-1)
            isls.append(e)
            continue
        s[chosen] = -s[chosen]
        if L - 1 - chosen != chosen:
            s[L - 1 - chosen] = -s[L - 1 - chosen]
        e += deltas[chosen]
        f ^= keys[chosen]
        stored = ht.insert(f)
        if e < st["best"]:
            st["best"] = e
        if e < since:
            since, stag = e, 0
        else:
            stag += 1
        code = chosen
        if stag >= patience or not stored:
            st["r"] += 1
            st["restarts"] += 1
            ht.new_generation()
            s, e, f, since, stag = begin()
            code |= 0x10000
        codes.append(code)
        isls.append(e)
    return codes, isls, st["best"], st["restarts"]


def bestfirst(L, seed, g, steps, K, tabu_log2=16, cap=32, second=False):
    """Algorithm 1 with a queue of K entries (the readings of the oracle's best-first
    search); returns (trace_code, trace_isl, best_isl, restarts, overflows, cache_hits).
    second: xLastovka's second table of evaluated neighbours, a list of slots holding
    (generation << 40) | (~fingerprint mod 2^40), the larger word kept on insertion."""
    n = (L + 1) // 2
    keys = [zkey(L, i) for i in range(n)]
    ht = HT(tabu_log2, cap)
    cache = [0] * ht.size if second else None
    st = {"r": 0, "best": None, "restarts": 0, "overflows": 0, "hits": 0}
    low = (1 << 40) - 1

    def tag(f):
        return (ht.gen << 40) | (~f & low)

    def fp_of(s):
        f = 0
        for i in range(n):
            if s[i] < 0:
                f ^= keys[i]
        return f

    def begin():
        s = skew(start_vars(seed, g, st["r"], L), L)
        e = isl_np(s)
        f = fp_of(s)
        ht.insert(f)
        if st["best"] is None or e < st["best"]:
            st["best"] = e
        return s, e, f

    def again():
        nonlocal cache
        st["r"] += 1
        st["restarts"] += 1
        g0 = ht.gen
        ht.new_generation()
        if cache is not None and ht.gen < g0:
            cache = [0] * ht.size
        return begin()

    s, e, f = begin()
    queue = []  # entries (isl, born, i, fp, state)
    codes, isls = [], []
    for t in range(steps):
        cands = []
        held = set()
        if cache is not None:
            held = {i for i in range(n) if cache[(f ^ keys[i]) % ht.size] == tag(f ^ keys[i])}
            st["hits"] += len(held)
        for i in range(n):
            if i in held:
                continue
            u = s.copy()
            u[i] = -u[i]
            if L - 1 - i != i:
                u[L - 1 - i] = -u[L - 1 - i]
            cands.append((isl_np(u), t, i, f ^ keys[i], u))
        cands.sort(key=lambda c: c[:3])
        for c in cands:
            if len(queue) == K and c[:3] > max(q[:3] for q in queue):
                break
            if ht.contains(c[3]):
                continue
            if len(queue) == K:
                queue.remove(max(queue, key=lambda q: q[:3]))
            queue.append(c)
            st["best"] = min(st["best"], c[0])
        if cache is not None:
            for c in cands:
                j = c[3] % ht.size
                cache[j] = max(cache[j], tag(c[3]))
        code = None
        while queue:
            top = min(queue, key=lambda q: q[:3])
            queue.remove(top)
            if ht.contains(top[3]):
                continue
            s, e, f = top[4], top[0], top[3]
            code = f & 0xFFFF
            if not ht.insert(f):
                st["overflows"] += 1
                queue = []
                s, e, f = again()
                code |= 0x10000
            break
        if code is None:
            queue = []
            s, e, f = again()
            code = -1
        codes.append(code)
        isls.append(e)
    return codes, isls, st["best"], st["restarts"], st["overflows"], st["hits"]


def walk_psl(L, seed, g, steps, tabu_log2=16, cap=32, patience=0):
    """The walk with (PSL, ISL) as the objective, compared as pairs; returns
    (trace_code, trace_isl, (best_psl, best_isl), restarts)."""
    n = (L + 1) // 2
    patience = patience or 2 * n
    keys = [zkey(L, i) for i in range(n)]
    ht = HT(tabu_log2, cap)
    st = {"r": 0, "best": None, "restarts": 0}

    def begin():
        s = skew(start_vars(seed, g, st["r"], L), L)
        obj = (psl_np(s), isl_np(s))
        f = 0
        for i in range(n):
            if s[i] < 0:
                f ^= keys[i]
        ht.insert(f)
        if st["best"] is None or obj < st["best"]:
            st["best"] = obj
        return s, obj, f, obj, 0

    def again():
        st["r"] += 1
        st["restarts"] += 1
        ht.new_generation()
        return begin()

    s, obj, f, since, stag = begin()
    codes, isls = [], []
    for _ in range(steps):
        cand = []
        for i in range(n):
            t = s.copy()
            t[i] = -t[i]
            if L - 1 - i != i:
                t[L - 1 - i] = -t[L - 1 - i]
            cand.append(((psl_np(t), isl_np(t)), i))
        chosen = None
        for o, i in sorted(cand):
            if not ht.contains(f ^ keys[i]):
                chosen, new = i, o
                break
        if chosen is None:
            s, obj, f, since, stag = again()
            codes.append(-1)
            isls.append(obj[1])
            continue
        s[chosen] = -s[chosen]
        if L - 1 - chosen != chosen:
            s[L - 1 - chosen] = -s[L - 1 - chosen]
        obj = new
        f ^= keys[chosen]
        stored = ht.insert(f)
        if obj < st["best"]:
            st["best"] = obj
        if obj < since:
            since, stag = obj, 0
        else:
            stag += 1
        code = chosen
        if stag >= patience or not stored:
            s, obj, f, since, stag = again()
            code |= 0x10000
        codes.append(code)
        isls.append(obj[1])
    return codes, isls, st["best"], st["restarts"]
