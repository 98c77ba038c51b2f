"""Pins for the oracle's random streams and per-cell grouping (CPU only).

Philox4x32-10 is pinned to published known-answer vectors; the grouping to
numpy's stable sort; the pairing order to brute force over an independent
pure-Python Philox.
"""
import os

import numpy as np
import pytest
from scipy import stats

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")

M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def py_philox(ctr, key):
    """Independent pure-Python Philox4x32-10 (Salmon et al. 2011) for brute-force checks."""
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
    return [c0, c1, c2, c3]


def kat_rows():
    rows = []
    with open(GOLD) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", kat_rows())
def test_philox_known_answers(orc, ctr, key, expect):
    assert [int(x) for x in orc.philox(ctr, key)] == expect
    assert py_philox(ctr, key) == expect


def test_philox_uniformity_chi2(orc):
    # 4 words x 20000 counters; top byte histogram must look uniform.
    words = np.array([orc.draw(12345, i, 7, orc.TAG_PARTICLE) for i in range(20000)], dtype=np.uint64)
    for col in range(4):
        h = np.bincount((words[:, col] >> 24).astype(np.int64), minlength=256)
        p = stats.chisquare(h).pvalue
        assert p > 1e-4, (col, p)


def test_uniform_range(orc):
    assert orc.uniform(0) == 0.5 / 2**32
    assert orc.uniform(0xFFFFFFFF) == (2**32 - 0.5) / 2**32
    assert 0.0 < orc.uniform(0) < orc.uniform(0xFFFFFFFF) < 1.0


def test_group_matches_numpy(orc):
    rng = np.random.default_rng(3)
    M = 50
    cell = rng.integers(0, M, 5000).astype(np.int32)
    cell[cell == 7] = 8  # an empty cell
    counts, cs, perm = orc.group(cell, M)
    assert np.array_equal(counts, np.bincount(cell, minlength=M))
    assert np.array_equal(cs[1:], np.cumsum(np.bincount(cell, minlength=M)))
    assert cs[0] == 0
    assert np.array_equal(perm, np.argsort(cell, kind="stable"))


def test_group_rejects_bad_cell(orc):
    with pytest.raises(RuntimeError):
        orc.group(np.array([0, 3, 1], np.int32), 3)


def test_pair_order_brute_force(orc):
    rng = np.random.default_rng(11)
    M = 9
    counts = [0, 1, 2, 3, 4, 7, 16, 33, 5]
    cell = np.repeat(np.arange(M), counts).astype(np.int32)
    p = rng.permutation(cell.size)
    cell = cell[p]
    seed, step = 0xDEADBEEF12345678, 41
    cs, order = orc.pair_order(cell, M, seed, step)
    key = [seed & MASK, seed >> 32]
    for j in range(M):
        members = [l for l in range(cell.size) if cell[l] == j]
        want = sorted(members, key=lambda l: (py_philox([l, step, 1, 0], key)[0], l))
        assert list(order[cs[j]:cs[j + 1]]) == want


def test_pair_order_changes_with_step(orc):
    cell = np.zeros(64, np.int32)
    _, o1 = orc.pair_order(cell, 1, 0, 1)
    _, o2 = orc.pair_order(cell, 1, 0, 2)
    assert sorted(o1) == list(range(64)) and sorted(o2) == list(range(64))
    assert not np.array_equal(o1, o2)


def test_pair_partner_uniform(orc):
    # Over many steps the partner of particle 0 in a 6-particle cell is uniform over the other 5.
    cell = np.zeros(6, np.int32)
    hits = np.zeros(6, np.int64)
    for s in range(3000):
        _, o = orc.pair_order(cell, 1, 5, s)
        pos = int(np.where(o == 0)[0][0])
        hits[int(o[pos ^ 1])] += 1
    assert hits[0] == 0
    assert stats.chisquare(hits[1:]).pvalue > 1e-3
