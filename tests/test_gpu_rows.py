"""GPU parity of the row kernels (labs_isl, labs_neighbor_delta) and of the exhaustive
skew search (labs_enumerate) against the CPU oracle: bit-exact integers."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import labs_inputs
import oracle
import paper_2011_00068_gb300 as labs
from tests.test_oracle_pins import table1

pytestmark = pytest.mark.gpu

INT32_MIN = -(2**31)


def skew_rows(batch, L, seed):
    xs = labs_inputs.random_free_vars(batch, L, seed)
    return np.stack([oracle.skew_expand(x, L) for x in xs])


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("L", [3, 5, 33, 201, 303, 511])
def test_isl_random_rows(L):
    rows = labs_inputs.random_pm1((67, L), seed=L)
    got = labs.isl(dev(rows)).cpu().numpy()
    want = np.array([oracle.isl(r) for r in rows])
    assert np.array_equal(got, want)


def test_isl_invalid_and_empty_rows():
    L = 21
    rows = labs_inputs.random_pm1((5, L), seed=1)
    rows[2, 7] = 0
    rows[4, 0] = 3
    got = labs.isl(dev(rows)).cpu().numpy()
    assert got[2] == -1 and got[4] == -1
    assert got[0] == oracle.isl(rows[0])
    assert labs.isl(dev(np.zeros((0, L), np.int8))).numel() == 0


@pytest.mark.parametrize("L", [3, 5, 7, 9, 21, 41, 63, 65, 101, 127, 129, 201, 255, 257, 303, 501, 511])
def test_neighbor_delta_random_skew(L):
    rows = skew_rows(37, L, seed=1000 + L)
    got = labs.neighbor_delta(dev(rows)).cpu().numpy()
    for r, g in zip(rows, got):
        assert np.array_equal(g, oracle.neighbor_delta(r))


def test_neighbor_delta_table1_and_degenerate():
    rows = [oracle.hex_decode(h, L) for L, _, _, h, _ in table1()]
    for L in sorted({len(r) for r in rows}):
        sel = np.stack([r for r in rows if len(r) == L])
        got = labs.neighbor_delta(dev(sel)).cpu().numpy()
        for r, g in zip(sel, got):
            assert np.array_equal(g, oracle.neighbor_delta(r))
    for L in (3, 41, 201, 511):
        n = (L + 1) // 2
        sel = np.stack([oracle.skew_expand(np.ones(n, np.int8), L),
                        oracle.skew_expand(-np.ones(n, np.int8), L),
                        oracle.skew_expand(labs_inputs.structured_pm1("alternating", n), L),
                        oracle.skew_expand(labs_inputs.structured_pm1("halves", n), L)])
        got = labs.neighbor_delta(dev(sel)).cpu().numpy()
        for r, g in zip(sel, got):
            assert np.array_equal(g, oracle.neighbor_delta(r))


def test_neighbor_delta_rejects_bad_rows():
    L = 41
    rows = skew_rows(4, L, seed=3)
    rows[1, L - 1] = -rows[1, L - 1]  # breaks Eq. 4
    rows[3, 5] = 0                    # not +-1
    got = labs.neighbor_delta(dev(rows)).cpu().numpy()
    assert (got[1] == INT32_MIN).all() and (got[3] == INT32_MIN).all()
    assert np.array_equal(got[0], oracle.neighbor_delta(rows[0]))
    assert np.array_equal(got[2], oracle.neighbor_delta(rows[2]))


def test_neighbor_delta_every_length():
    """Every odd L = 3..511 (every lane block and word count the row kernels
    instantiate): two random skew rows, a row with one entry negated (breaks Eq. 4 unless
    it is the centre) and, at odd batch sizes, the two-rows-per-warp tail."""
    rng = np.random.default_rng(21)
    for L in range(3, 512, 2):
        n = (L + 1) // 2
        rows = skew_rows(3, L, seed=L)
        j = int(rng.integers(0, L - 1))
        j = j if j < n - 1 else j + 1  # any position but the centre
        rows[2, j] = -rows[2, j]
        got = labs.neighbor_delta(dev(rows)).cpu().numpy()
        for b in (0, 1):
            assert np.array_equal(got[b], oracle.neighbor_delta(rows[b])), (L, b)
        assert (got[2] == INT32_MIN).all(), (L, j)


@pytest.mark.parametrize("L,offset", [(41, 1), (201, 3), (401, 5), (201, 16)])
def test_neighbor_delta_unaligned_input(L, offset):
    """Rows starting off a 16-byte boundary are read from global memory directly (no
    staging copy); offset 16 keeps the staged path with a shifted base."""
    B = 37
    rows = skew_rows(B, L, seed=50 + L)
    buf = torch.zeros(B * L + offset, dtype=torch.int8, device="cuda")
    buf[offset:] = dev(rows.reshape(-1))
    view = buf[offset:].view(B, L)
    assert (view.data_ptr() % 16 == 0) == (offset % 16 == 0)
    got = labs.neighbor_delta(view).cpu().numpy()
    for r, g in zip(rows, got):
        assert np.array_equal(g, oracle.neighbor_delta(r))


@pytest.mark.parametrize("L,B", [(3, 1), (3, 2), (5, 3), (41, 1), (201, 1), (401, 1)])
def test_neighbor_delta_tiny_batches(L, B):
    """Inputs shorter than one 16-byte block (nothing staged) and single rows."""
    rows = skew_rows(B, L, seed=7 + L + B)
    got = labs.neighbor_delta(dev(rows)).cpu().numpy()
    for r, g in zip(rows, got):
        assert np.array_equal(g, oracle.neighbor_delta(r))


def test_neighbor_delta_many_rows_per_warp():
    """About ten row pairs per warp (both staging buffers in turn), an odd batch whose
    byte count is not a multiple of 16 (the last bytes come from global memory), every
    row checked."""
    L, B = 41, 150001
    rows = skew_rows(B, L, seed=77)
    assert (B * L) % 16 != 0
    got = labs.neighbor_delta(dev(rows)).cpu().numpy()
    bad = [b for b in range(B) if not np.array_equal(got[b], oracle.neighbor_delta(rows[b]))]
    assert not bad, bad[:10]


def test_neighbor_delta_large_batch_sampled():
    """The launch shape used for throughput (many rows per warp slot): sampled rows."""
    L, B = 201, 20000
    xs = labs_inputs.random_free_vars(B, L, seed=11)
    n = (L + 1) // 2
    c = n - 1
    # Eq. 4 expansion of the free variables, in torch, for the big batch
    x = torch.from_numpy(xs).cuda()
    j = torch.arange(1, n, device="cuda")
    sign = torch.where(j % 2 == 1, -1, 1).to(torch.int8)
    right = x[:, c - j] * sign
    rows = torch.cat([x, right], dim=1).contiguous()
    got = labs.neighbor_delta(rows).cpu().numpy()
    rng = np.random.default_rng(0)
    for b in list(rng.choice(B, 48, replace=False)) + [0, B - 1]:
        r = rows[b].cpu().numpy()
        assert oracle.is_skew(r)
        assert np.array_equal(got[b], oracle.neighbor_delta(r))


@pytest.mark.parametrize("L", [3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27])
def test_enumerate_small(L):
    m, cnt, first, _ = oracle.enumerate_skew(L)
    assert labs.enumerate_skew(L) == (m, cnt, first)


def test_enumerate_L41():
    m, cnt, first, seq = oracle.enumerate_skew(41)
    assert (m, cnt) == (108, 2)
    assert labs.enumerate_skew(41) == (m, cnt, first)
