"""Pins of the oracle's bijection pairing mode (cells of at least 4097 particles).

The mode pairs the particle of id rank r with the one whose rank shares its
pairing slot under a keyed bijection pi of [0, n).  Nothing in the paper fixes
pi, so it is pinned against what a uniformly random perfect matching must
satisfy:
  * pi is a bijection of [0, n) and the inverse undoes it, for many sizes;
  * positions, partners and the particle left out of an odd cell are uniform
    (chi^2 over coarse bins);
  * pairs of ranks at a fixed distance d (d = 1, 2, the mixed radix b, ...) occur
    at the rate of a random matching, (n - d) / (n - 1) per matching -- a
    four-round version of the same network pairs neighbouring ranks 1.33 times
    too often and fails this;
  * a block of "hot" ranks (the last 5 %, as a loader that writes each cell's
    hot tail last would produce) is paired within itself at the random rate;
  * the pairing depends on the ids, not on the storage order;
  * small cells keep the key sort;
  * the neutral step's candidate count is floor(P_null N + U): its mean is
    P_null N and each particle is selected with the same frequency.
"""
import math

import numpy as np
import pytest
from scipy.stats import chi2

from paper_2508_06771_gb300 import workloads as W

P_MIN = 1e-3     # chi^2 p-value floor (fixed seeds: the values are deterministic)


def _chi2_p(counts):
    counts = np.asarray(counts, float)
    e = counts.sum() / counts.size
    return chi2.sf(((counts - e) ** 2 / e).sum(), counts.size - 1)


@pytest.mark.parametrize("n", list(range(1, 200)) + [4095, 4096, 4097, 4098, 5000, 8191, 9999, 10000, 12289,
                                                     30001, 65535, 65536])
def test_bijection_and_inverse(orc, n):
    for cell, step in ((0, 0), (7, 3), (123456, 99999)):
        fwd, prm = orc.bij_table(11, cell, step, n)
        inv, _ = orc.bij_table(11, cell, step, n, inverse=True)
        assert np.array_equal(np.sort(fwd), np.arange(n))
        assert np.array_equal(inv[fwd], np.arange(n))
        a, b = int(prm[0]), int(prm[1])
        assert a * a >= n and (a - 1) * (a - 1) < n and a * b >= n and a * (b - 1) < n


@pytest.fixture(scope="module")
def tables(orc):
    """pi for 2000 (cell, step) keys at n = 4097 (odd) and n = 10000."""
    out = {}
    for n in (4097, 10000):
        out[n] = [orc.bij_table(5, t % 97, t // 97, n) for t in range(2000)]
    return out


def _matching(fwd, n):
    inv = np.empty(n, np.int64)
    inv[fwd] = np.arange(n)
    m = n - n % 2
    return inv[0:m:2], inv[1:m:2], inv


@pytest.mark.parametrize("n", [4097, 10000])
def test_positions_and_partners_uniform(tables, n):
    bins = 50
    pos = {r: np.zeros(bins, np.int64) for r in (0, n // 2, n - 1)}
    part = {r: np.zeros(bins, np.int64) for r in (0, n - 2)}
    for fwd, _ in tables[n]:
        for r in pos:
            pos[r][fwd[r] * bins // n] += 1
        _, _, inv = _matching(fwd, n)
        for r in part:
            q = fwd[r] ^ 1
            if q < n - n % 2:
                part[r][inv[q] * bins // n] += 1
    for r, c in pos.items():
        assert _chi2_p(c) > P_MIN, ("position", r)
    for r, c in part.items():
        assert _chi2_p(c) > P_MIN, ("partner", r)


def test_odd_cell_left_out_uniform(tables):
    n, bins = 4097, 50
    c = np.zeros(bins, np.int64)
    for fwd, _ in tables[n]:
        _, _, inv = _matching(fwd, n)
        c[inv[n - 1] * bins // n] += 1
    assert _chi2_p(c) > P_MIN


@pytest.mark.parametrize("n", [4097, 10000])
def test_rank_distance_pairs_at_random_rate(tables, n):
    """Pairs (r, r + d): a uniformly random matching holds (n - d)/(n - 1) of them on average."""
    b = int(tables[n][0][1][1])
    for d in (1, 2, 3, b - 1, b, b + 1, 2 * b):
        tot = 0
        for fwd, _ in tables[n]:
            pa, pb, _ = _matching(fwd, n)
            tot += int(np.sum(np.abs(pa - pb) == d))
        keys = len(tables[n])
        exp = keys * (n - d) / (n - 1)
        assert abs(tot - exp) < 4.0 * math.sqrt(exp), (d, tot, exp)


def test_four_round_network_would_fail_the_neighbour_pin():
    """The same mixed-radix network with four rounds (a plausible cheaper variant) pairs
    neighbouring ranks about 1.3-1.45 times too often; the test above would catch it."""
    M1, M2 = 0x9E3779B1, 0x85EBCA6B

    def f(r, k, m):
        w = ((r ^ k) * M1) & 0xFFFFFFFF
        u = w ^ (w >> 16)
        return (((u * M2) & 0xFFFFFFFF) * m) >> 32

    n = 4096
    a = b = 64
    rng = np.random.default_rng(3)
    tot = 0
    keys = 400
    for _ in range(keys):
        K = [int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)]
        x = np.arange(n)
        L, R = x // b, x % b
        for i in range(4):
            m = a if i % 2 == 0 else b
            L, R = R, (L + np.array([f(int(r), K[i], m) for r in R])) % m
        fwd = L * b + R
        pa, pb, _ = _matching(fwd, n)
        tot += int(np.sum(np.abs(pa - pb) == 1))
    exp = keys * (n - 1) / (n - 1)
    assert tot > exp + 4.0 * math.sqrt(exp)


def test_hot_block_mixes(tables):
    """The last 5 % of ranks pair among themselves at the random-matching rate
    C(h, 2) / (n - 1) per matching."""
    n = 10000
    h = n // 20
    tot = 0
    for fwd, _ in tables[n]:
        pa, pb, _ = _matching(fwd, n)
        tot += int(np.sum((pa >= n - h) & (pb >= n - h)))
    exp = len(tables[n]) * h * (h - 1) / 2 / (n - 1)
    assert abs(tot - exp) < 4.0 * math.sqrt(exp), (tot, exp)


def _cells_wl(counts, seed=2, shuffled=True):
    counts = np.asarray(counts)
    rng = np.random.default_rng(seed)
    n = int(counts.sum())
    cell = np.repeat(np.arange(counts.size, dtype=np.int32), counts)
    if shuffled:
        cell = cell[rng.permutation(n)]
    return cell


def test_pairing_follows_ids_not_storage(orc):
    """Two storage orders of the same particles (same ids) give the same matching of ids."""
    counts = [4097, 100, 6000]
    cell = _cells_wl(counts, shuffled=False)
    wl = W._base(len(counts), seed=9)
    P = orc.make_params(wl, pairing_mode=orc.PAIR_BIJECTION)
    rng = np.random.default_rng(4)
    ids = rng.permutation(cell.size).astype(np.uint32)     # arbitrary distinct ids
    p = rng.permutation(cell.size)
    cs1, o1 = orc.pair_order_mode(cell, len(counts), P, 17, ids)
    cs2, o2 = orc.pair_order_mode(cell[p], len(counts), P, 17, ids[p])
    assert np.array_equal(cs1, cs2)
    assert np.array_equal(ids[o1], ids[p][o2])


def test_small_cells_keep_the_key_sort(orc):
    counts = [4096, 3, 2000, 4097]
    cell = _cells_wl(counts)
    wl = W._base(len(counts), seed=9)
    P = orc.make_params(wl, pairing_mode=orc.PAIR_BIJECTION)
    cs, ob = orc.pair_order_mode(cell, len(counts), P, 5)
    _, ok = orc.pair_order(cell, len(counts), 9, 5)
    for j in range(3):
        a, b = int(cs[j]), int(cs[j + 1])
        assert np.array_equal(ob[a:b], ok[a:b])
    a, b = int(cs[3]), int(cs[4])
    assert not np.array_equal(ob[a:b], ok[a:b])
    # the large cell: rank r (ascending storage index, the ids here) sits at position pi(r)
    fwd, _ = orc.bij_table(9, 3, 5, 4097)
    members = np.sort(np.nonzero(cell == 3)[0])
    assert np.array_equal(ob[a:b][fwd], members)


def test_candidate_count_law_and_uniform_selection(orc):
    """Bijection mode neutral step on 8 cells x 5000 electrons over 60 steps: each cell's
    candidate count is floor or ceil of P_null N with mean P_null N, and every particle
    is selected about equally often."""
    ncell, ppc, steps = 8, 5000, 60
    rng = np.random.default_rng(12)
    vt = math.sqrt(5.0 * W.E_CHARGE / W.M_E)
    n = ncell * ppc
    wl = W._base(ncell, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt,
                 vz=rng.standard_normal(n) * vt, cell=np.repeat(np.arange(ncell, dtype=np.int32), ppc),
                 inv_vol=np.full(ncell, 1e17), dt_cell=np.full(ncell, 4e-11), lnlam_cell=np.full(ncell, 10.0),
                 seed=21, capacity=4 * n, sigma_ion=0.0)
    P = orc.make_params(wl, pairing_mode=orc.PAIR_BIJECTION)
    sel = np.zeros(n, np.int64)
    dev = []
    for s in range(steps):
        st = orc.State(wl)
        vx, vy, vz, cl = st.views()
        vmax2 = np.array([np.max(vx[cl == j] ** 2 + vy[cl == j] ** 2 + vz[cl == j] ** 2) for j in range(ncell)])
        numax = wl["n_neutral"] * (wl["sigma_el"] + wl["sigma_ion"]) * np.sqrt(vmax2)
        pnull = -np.expm1(-numax * wl["dt_cell"])
        out = orc.neutral(st, P, s, with_decisions=True)
        cand = out["decision"] > 0
        sel += cand
        for j in range(ncell):
            c = int(cand[j * ppc:(j + 1) * ppc].sum())
            t = pnull[j] * ppc
            assert c in (math.floor(t), math.ceil(t)), (s, j, c, t)
            dev.append(c - t)
    dev = np.array(dev)
    # the rounding uniform makes each count's error a zero-mean variable bounded by 1
    assert abs(dev.mean()) < 4.0 * 0.5 / math.sqrt(dev.size)
    # within each cell (the cells' P_null differ), selections spread evenly over 25 bins of ids
    bins = 25
    x2 = 0.0
    for j in range(ncell):
        c = sel[j * ppc:(j + 1) * ppc].reshape(bins, -1).sum(axis=1).astype(float)
        e = c.sum() / bins
        x2 += ((c - e) ** 2 / e).sum()
    assert chi2.sf(x2, ncell * (bins - 1)) > P_MIN
