"""Shared-memory bounds of every walker layout, checked on the CPU.

tests/layout/layout_dump.cpp compiles the layout functions of labs_internal.cuh for the
host and prints each layout (row padding and length, table padding and length, bit
vectors, lane block).  For every length the kernels serve and every lane block the
launch code can pick, the extreme index of every family of shared-memory accesses (the
rows, the table, the bit vectors, in the walk, the best-first search, the PSL walk, the
row kernels and the long-sequence kernels, plain, PSL and best-first) must fall inside its region.  The index
families are restated here from the kernels; the lane and output indices enter them
monotonically, so the first and last lane of each parity class bound them.
"""
from __future__ import annotations

import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def layouts(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("layout") / "layout_dump")
    src = os.path.join(ROOT, "tests", "layout", "layout_dump.cpp")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_2011_00068_gb300", "csrc"), src, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    warp, long_, row = {}, {}, {}
    for line in out.splitlines():
        f = line.split()
        v = list(map(int, f[1:]))
        if f[0] == "row":
            row[(v[0], v[1])] = dict(apad=v[2], alen=v[3], gpad=v[4], glen=v[5], bvec=v[6], boff=v[7], poff=v[8],
                                     words=v[9], R=v[10], roff=v[11], xp=v[12], hoff=v[13], hlen=v[14], hpad=v[15])
        elif f[0] in ("warp", "warpp"):
            tile, n = v[0], v[1]
            warp[(tile if f[0] == "warp" else "psl16", n)] = dict(apad=v[2], alen=v[3], gpad=v[4], glen=v[5], bvec=v[6], xoff=v[7], words=v[8],
                                   R=v[9], xp=v[10], hoff=v[11], hlen=v[12], hpad=v[13], roff=v[14])
        else:
            nt, n = v[0], v[1]
            long_[(nt, n)] = dict(nt=nt, apad=v[2], alen=v[3], gpad=v[4], glen=v[5], bvec=v[6], xoff=v[7],
                                  words=v[8], R=v[9], limit=v[10], psl_only=v[11], xp=v[12], hoff=v[13],
                                  hlen=v[14], hpad=v[15], roff=v[16])
    return warp, long_, row


def conflict_free_R(R, tile):
    while 16 // min(R & -R, 16) < tile // 2:
        R += 1
    return R


class Region:
    def __init__(self, S):
        self.S, self.bad = S, []

    def a(self, idx, what):
        if not (-self.S["apad"] <= idx < self.S["alen"] - self.S["apad"]):
            self.bad.append(("A", what, idx))

    def g(self, y, what):
        if not (-self.S["gpad"] <= y < self.S["glen"] - self.S["gpad"]):
            self.bad.append(("G", what, y))

    def h(self, idx, what):                 # FP16 rows (tensor-core layouts)
        if not (-self.S["hpad"] <= idx < 2 * self.S["hlen"] - self.S["hpad"]):
            self.bad.append(("H", what, idx))

    def b(self, word, what):
        if not (0 <= word < self.S["bvec"]):
            self.bad.append(("B", what, word))


def common(reg, n, tile, R, valid_only, bits=True):
    """Rows, Toeplitz window, assembly, table and (bits) bit vectors."""
    c = n - 1
    half = tile // 2
    v0max = (half - 1) * R
    nu = (n + 7) & ~7
    reg.a(n - 1, "row")                     # s_j -> A_{j&1}[j>>1], j < L
    reg.a(0, "toe A0")
    reg.a(nu - 1, "toe A")                  # float4 rows A[u .. u+7], u < round8(n)
    reg.g(-v0max - (R - 1), "toe win0")     # initial window G[-v0 - r]
    reg.g(nu, "toe top")                    # G[u + 2q + 2 - v0] at v0 = 0
    reg.g(1 - v0max, "toe low")
    for p in (0, 1):
        nv = (n >> 1) if p else ((n + 1) >> 1)
        vmax = (nv - 1) if valid_only else (v0max + R - 1)
        for v in (0, vmax):
            i = 2 * v + p
            reg.a(v, "asm v")
            reg.a(n - 1 - v - p, "asm q")
            reg.a(3 * v + p - n + 1, "asm t")
            reg.g(c - i, "asm G")
    for m in (1, n - 1):                    # set_E
        reg.g(m, "E")
        reg.g(m - 1, "E.y")
        if m <= reg.S["gpad"]:
            reg.g(-m, "mirror E")
        if m < reg.S["gpad"]:
            reg.g(-m - 1, "mirror E.y")
    if not bits:
        return
    for p in (0, 1):                        # shifted mismatch counts (table) and P
        np_ = n - 1 if p else n
        for m in (1, 2, 31, 32, 33, n - 2, n - 1):
            if 1 <= m < n:                  # both classes run over the even class's words
                reg.b((n - m - 1) // 32 + (m >> 5) + 1, "table")
        nv = (n >> 1) if p else ((n + 1) >> 1)
        for v in range(max(1, nv - 40), nv):
            k = (v - 1) // 32
            reg.b(k + ((v + 1) >> 5) + 1, "P x")
            reg.b(k + ((np_ - v) >> 5) + 1, "P xr")
    reg.b(((n + 31) // 32), "bits zero word")


def tensor_core_reads(reg, S, n, R, half=8):
    """Every table, FP16-row and scratch index of the tensor-core Toeplitz product
    (toeplitz_tc, toeplitz_tc1): column groups m of 4 output blocks per class, block
    diagonals d = -min(4m+3, T-1) .. S-1-4m; `half` lanes per class read R outputs each."""
    nS = (n + 15) >> 4
    nT = (((n + 1) >> 1) + 15) >> 4
    for m in range((nT + 3) // 4):
        dlo = -min(4 * m + 3, nT - 1)
        nd = nS - 4 * m - dlo
        ys = [16 * dlo + 2 * tq - g for tq in range(4) for g in range(8)]
        reg.g(min(ys) - 8, "tc table first")
        for k in (0, nd - 1):
            reg.g(min(ys) + 16 * k, "tc table")
            reg.g(max(ys) + 16 * k + 8 + 1, "tc table + 8")
            for tb in range(4):
                for tq in (0, 3):
                    u = 16 * (tb + 4 * m + dlo + k) + 2 * tq
                    reg.h(u, "tc rows")
                    reg.h(u + 9, "tc rows + 9")
        for tx in (0, 2):
            for t in (tx + 4 * m, tx + 4 * m + 1):
                if t < nT and not 16 * t + 15 < S["xp"]:
                    reg.bad.append(("X write", t))
    if not ((S["xp"] & 31) == 16 and half * R <= S["xp"]):
        reg.bad.append(("X scratch", S["roff"], S["xp"]))
    if not ((S["hlen"] & 7) == 4 and (S["hpad"] & 1) == 0):
        reg.bad.append(("FP16 rows", S["hlen"], S["hpad"]))


def test_warp_layouts(layouts):
    warp, _, _ = layouts
    bad = []
    for tile in (8, 16, 32):
        for n_max in range(2, 257):
            S = warp[(tile, n_max)]
            RMAX = S["R"]
            for n in range(2, n_max + 1):
                need = warp[(tile, n)]["R"]
                if tile in (8, 16):   # walk_group's choice
                    R = need if need >= RMAX - 3 else conflict_free_R(RMAX - 3, tile)
                    R = min(R, RMAX)
                else:                 # walk_chunk_kernel's choice
                    R = RMAX if (RMAX <= 2 or need >= RMAX) else RMAX - 2
                assert R >= need
                reg = Region(S)
                c = n - 1
                common(reg, n, tile, R, valid_only=(tile == 8))
                half = tile // 2
                v0max = (half - 1) * R
                # lockstep lag update: lane l covers m = 1 + lR .. (l+1)R, no bounds test
                # (tile 8: reads above stay inside the class)
                for i in (0, 1, c - 1, c):
                    if i < 0:
                        continue
                    vb, pb = i >> 1, i & 1
                    vq = vb if i == c else n - 1 - vb - pb
                    reg.a(vq, "vq")
                    npc = n - 1 if pb else n
                    top = vb + tile * R
                    reg.a(min(top, npc - 1) if tile == 8 else top, "up")
                    reg.a(vb - tile * R, "dn")
                    reg.a(2 * v0max + 2 * (R - 1) - vb, "p1")
                    reg.a(-vq, "p2")
                    if tile == 32:      # strided lags (learned mode, PSL and best-first moves)
                        reg.a(vb + n - 1, "up32")
                        reg.a(vb - (n - 1), "dn32")
                reg.g(tile * R, "E load")
                if tile != 8 or 1 + (tile - 1) * R + R <= S["gpad"]:
                    reg.g(-(1 + (tile - 1) * R) - R, "mirror E load")
                if tile == 8:           # the mirror half of the table as deep as the window reads
                    covered = set()
                    for l in range(8):
                        m0 = 1 + l * R
                        if m0 + R <= S["gpad"]:
                            covered.update(range(m0, m0 + R))
                    if not set(range(1, min(n, 4 * R))) <= covered:
                        reg.bad.append(("mirror coverage", n, R))
                if tile == 16 and n_max <= 128 and not S["xp"]:
                    reg.bad.append(("no tensor-core regions", n_max))
                if S["xp"]:             # the Toeplitz product on the tensor cores
                    if tile == 8:
                        reg.bad.append(("tensor-core regions with four walkers per warp", n_max))
                    tensor_core_reads(reg, S, n, R, tile // 2)
                    if not (S["roff"] + 2 * S["xp"] <= S["hoff"] and S["hoff"] + 2 * S["hlen"] <= S["words"]):
                        reg.bad.append(("regions", S["roff"], S["hoff"], S["words"]))
                    reg.h(n - 1, "row copy")
                    if tile == 32 and S["words"] * 4 * 16 > 226 * 1024:
                        reg.bad.append(("two 8-warp CTAs do not fit", S["words"]))
                if tile == 32:          # the PSL neighbourhood
                    psl_reads(reg, n, R, v0max)
                if reg.bad:
                    bad.append((tile, n_max, n, R, reg.bad[:3]))
    assert not bad, bad[:5]


def psl_passes(R):
    """The ring passes of psl_eval: one up to R = 6, two from R = 8 (R = 7 takes the
    compare-and-select form)."""
    if R >= 8:
        h = (R + 1) // 2
        return [(0, h), (h, R - h)]
    return [(0, R)]


def psl_reads(reg, n, R, v0max):
    """The PSL neighbourhood (psl_eval): each ring pass over outputs C0 .. C0+RC-1 of a
    lane (block start w0 = v0 + C0) runs its lags 2 RC - 2 past n - 1; the select form
    reads the class from -(n-1) up to v0 + n + R - 2."""
    if R == 7:
        reg.a(-(n - 1), "psl sel a")
        reg.a(v0max + n + R - 2, "psl sel b")
        reg.a(v0max + R - 1, "psl sel init")
        return
    for C0, RC in psl_passes(R):
        P = 3 * RC - 2
        tend = n - 1 + 2 * (RC - 1)
        for w0 in (C0, v0max + C0):
            reg.a(w0 + RC - 1, "psl cs")
            reg.a(w0 + P - 1, "psl ring init hi")
            reg.a(w0 + 1 - P, "psl ring init lo")
            reg.a(w0 - tend, "psl a")
            reg.a(w0 + tend, "psl b")
        reg.g(1 - P, "psl ring init G")
        reg.g(tend, "psl C")


def test_psl_pair_layouts(layouts):
    """The PSL walk with two walkers per warp (n_max <= 128): every access of the plain
    lockstep step with two walkers per warp (rows, table, bit vectors, lag update, the
    tensor-core product) and the PSL neighbourhood's reads for the lane blocks that
    walk_group picks, inside the layout warp_smem(n_max, 16, psl)."""
    warp, _, _ = layouts
    bad = []
    for n_max in range(2, 129):
        S = warp[("psl16", n_max)]
        plain = warp[(16, n_max)]
        RMAX = S["R"]
        if RMAX != plain["R"] or not S["xp"] or S["words"] < plain["words"]:
            bad.append((n_max, "layout", RMAX, S["xp"], S["words"]))
        for n in range(2, n_max + 1):
            need = warp[(16, n)]["R"]
            R = need if need >= RMAX - 3 else conflict_free_R(RMAX - 3, 16)
            R = min(R, RMAX)
            assert R >= need
            reg = Region(S)
            c = n - 1
            common(reg, n, 16, R, valid_only=False)
            v0max = 7 * R
            for i in (0, 1, c - 1, c):
                if i < 0:
                    continue
                vb, pb = i >> 1, i & 1
                vq = vb if i == c else n - 1 - vb - pb
                reg.a(vq, "vq")
                reg.a(vb + 16 * R, "up")
                reg.a(vb - 16 * R, "dn")
                reg.a(2 * v0max + 2 * (R - 1) - vb, "p1")
                reg.a(-vq, "p2")
            reg.g(16 * R, "E load")
            reg.g(-(1 + 15 * R) - R, "mirror E load")
            tensor_core_reads(reg, S, n, R, 8)
            if not (S["roff"] + 2 * S["xp"] <= S["hoff"] and S["hoff"] + 2 * S["hlen"] <= S["words"]):
                reg.bad.append(("regions", S["roff"], S["hoff"], S["words"]))
            reg.h(n - 1, "row copy")
            psl_reads(reg, n, R, v0max)
            if reg.bad:
                bad.append((n_max, n, R, reg.bad[:3]))
        # two 8-warp CTAs of 16 walkers each fit on an SM
        if S["words"] * 4 * 16 * 2 > 226 * 1024:
            bad.append((n_max, "two CTAs", S["words"]))
    assert not bad, bad[:5]


def test_long_layouts(layouts):
    _, long_, _ = layouts
    bad = []
    # lane blocks compiled for each CTA width (the dispatch in labs_long.cu)
    compiled = {128: {3, 5, 7, 9}, 256: {3, 5, 7, 9}, 512: {5, 7, 9, 11}}
    assert {n for _, n in long_} == set(range(257, 5633))
    for (nt, n_max), S in sorted(long_.items(), key=lambda kv: kv[0][1]):
        R = S["R"]
        assert R in compiled[nt], (nt, n_max, R)
        # scratch (nt words), bits (kBitWordsLong = 176 words), then the best-first search's
        # 32 queue keys, nt / 32 warps x 32 candidate keys, 32 entered keys (all 64-bit, so
        # 8-byte aligned), two words of round state and 32 places
        q = S["xoff"] + nt + 176
        end = q + 2 * 32 + 2 * nt + 2 * 32 + 4 + 32
        assert nt * R >= n_max and S["words"] >= end
        assert q % 2 == 0
        assert S["words"] * 4 <= {512: 227, 256: 113, 128: 56}[nt] * 1024  # one, two or four CTAs per SM
        if S["xp"]:
            # FP16 rows between the bit vectors and the scratch (cleared with the rows), the
            # product's results after everything else
            assert S["hoff"] + 2 * S["hlen"] <= S["xoff"], (nt, n_max)
            assert S["roff"] >= end and S["roff"] + 2 * S["xp"] <= S["words"], (nt, n_max)
        for n in sorted({257, (257 + n_max) // 2, n_max}):
            reg = Region(S)
            common(reg, n, nt, R, valid_only=True)
            if S["xp"]:
                tensor_core_reads(reg, S, n, R, nt // 2)
                reg.h(n - 1, "row copy")
            c = n - 1
            for vb in (0, c >> 1):
                reg.a(vb + n - 1, "flip up")
                reg.a(vb - (n - 1), "flip dn")
            reg.a(-(n - 1), "p")
            reg.a(2 * ((n + 1) >> 1), "p hi")
            v0max = (nt // 2 - 1) * R        # the PSL neighbourhood (long PSL walk)
            psl_reads(reg, n, R, v0max)
            if reg.bad:
                bad.append((n_max, n, R, reg.bad[:3]))
    assert not bad, bad[:5]


def test_long_exact_range_bound(layouts):
    """The bound on ISL keeps 16 sqrt((n-1) ISL) + 8L + 32n + 32 below 2^24 (Cauchy-Schwarz
    on sum |C_2m|), the condition for the long kernels' fp32 arithmetic to be exact, and
    stays above the ISL of random starts (about L^2/2) by a factor of at least 2."""
    _, long_, _ = layouts
    limit = {n: S["limit"] for (_, n), S in long_.items()}
    for n in (257, 1024, 2048, 4096, 5632):
        L = 2 * n - 1
        lim = limit[n]
        assert 16 * ((n - 1) * lim) ** 0.5 + 8 * L + 32 * n + 32 < 2 ** 24
        assert lim > L * L  # twice the mean ISL of random starts
        assert lim < 2 ** 29


def row_tensor_core(reg, S, n, R):
    """The two-row kernel for n <= 128: FP16 rows only, the tensor-core product, the
    assembly on the FP16 rows and the table, Q overwritten by the product's results."""
    c = n - 1
    vtop = 8 * R
    tensor_core_reads(reg, S, n, R)
    for p in (0, 1):
        reg.h(n - 1 - p, "row load")
        for v in (0, vtop - 1):             # every lane output, existing or not
            reg.h(v, "asm v")
            reg.h(n - 1 - p - v, "asm q")
            reg.h(3 * v + p - n + 1, "asm t")
            reg.g(c - p - 2 * v, "asm G")
    for m in (1, n - 1):                    # the table's writes and mirror writes
        reg.g(m, "E")
        reg.g(m - 1, "E.y")
        reg.g(-m, "mirror E")
        reg.g(-m - 1, "mirror E.y")
    nS = (n + 15) >> 4
    if S["glen"] - S["gpad"] < 16 * nS:     # E is zero from n up to what the product reads
        reg.bad.append(("table top", S["glen"] - S["gpad"]))
    q = max(n, 2 * S["xp"])
    if not (S["roff"] == S["poff"] >= S["boff"] and S["poff"] + q <= S["words"]):
        reg.bad.append(("Q / X region", S["poff"], S["xp"], S["words"]))
    if not (S["hoff"] + 2 * S["hlen"] <= S["boff"] - 2 * S["glen"]):   # rows, then the table
        reg.bad.append(("FP16 rows overlap the table", S["hoff"], S["hlen"]))
    if S["apad"] or S["alen"]:
        reg.bad.append(("FP32 rows", S["apad"], S["alen"]))


def test_row_layouts(layouts):
    """The row kernels (labs_neighbor_delta): two rows per warp (16 lanes) up to n = 160,
    one per warp above; rows, Toeplitz window, assembly and table as in the walk, and the
    per-lag P values Q[m], written for m < n and read at max(n_p - 1 - 2v, 0), inside
    their own region after the bit vectors."""
    _, _, row = layouts
    bad = []
    assert {n for _, n in row} == set(range(2, 257))
    for (tile, n), S in sorted(row.items()):
        R = S["R"]
        reg = Region(S)
        if tile == 16 and n <= 128:
            row_tensor_core(reg, S, n, R)
            if reg.bad:
                bad.append((tile, n, R, reg.bad[:3]))
            continue
        # the two-row kernel assembles every lane output; the one-row kernel existing ones
        common(reg, n, tile, R, valid_only=(tile == 32), bits=False)
        for m in (1, n - 1):                    # the table's mirror writes, unconditional
            reg.g(-m, "mirror E (row)")
            reg.g(-m - 1, "mirror E.y (row)")
        for p in (0, 1):                        # row_load writes entries below the class length
            reg.a((n - 1 - p), "row load")
        if S["alen"] - S["apad"] < ((n + 7) & ~7):
            reg.bad.append(("zero padding to round8(n)", S["alen"] - S["apad"]))
        if S["gpad"] < n:                       # the table's mirror writes are unconditional
            reg.bad.append(("gpad below n", S["gpad"]))
        q_words = (n + 3) & ~3
        if not (S["poff"] >= S["boff"] and S["poff"] + q_words <= S["words"]):
            reg.bad.append(("Q region", S["poff"], S["words"]))
        half = tile // 2
        for p in (0, 1):
            np_ = n - p
            for v in (0, (half - 1) * R + R - 1):       # every lane output, existing or not
                idx = max(np_ - 1 - 2 * v, 0)
                if not 0 <= idx < n:
                    reg.bad.append(("Q read", p, v, idx))
        if S["words"] % 4:
            reg.bad.append(("alignment", S["words"]))
        if reg.bad:
            bad.append((tile, n, R, reg.bad[:3]))
    assert not bad, bad[:5]
