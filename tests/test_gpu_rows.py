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
