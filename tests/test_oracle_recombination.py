"""Pins of the oracle's recombination C5 (Table 1; RS0-RS5 of Table 4, Sec. 4.3).

* Count law: each cell removes floor or ceil of P_rec N primaries, P_rec N on
  average, and never more than N / 2 (every primary needs its own catalyte).
* Matching: every removed primary has exactly one catalyte in its own cell,
  no catalyte serves two primaries and no primary is a catalyte -- per cell, the
  particles whose velocity changed are as many as the removed ones and disjoint
  from them.
* Energy bookkeeping: per cell, the kinetic energy of the live particles after
  the step equals the energy of all before plus dE_rec per recombination (the
  primary's energy passes to its catalyte).
* The catalytes' new directions are isotropic.
* Cells of fewer than two particles are left alone; removed particles no
  longer count in the moments.
"""
import math

import numpy as np

from paper_2508_06771_gb300 import workloads as W


def _wl(counts, seed=4, T=2.0, dens=1e20):
    counts = np.asarray(counts)
    rng = np.random.default_rng(seed)
    n = int(counts.sum())
    vt = math.sqrt(T * W.E_CHARGE / W.M_E)
    M = counts.size
    return W._base(M, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt,
                   vz=rng.standard_normal(n) * vt, cell=np.repeat(np.arange(M, dtype=np.int32), counts),
                   inv_vol=np.full(M, dens / 1000.0), dt_cell=np.full(M, 1e-10), lnlam_cell=np.full(M, 10.0),
                   seed=seed, capacity=2 * n)


def _prec(wl, counts, k_rec):
    nj = wl["weight"] * np.asarray(counts) * wl["inv_vol"]
    return -np.expm1(-wl["dt_cell"] * k_rec * nj * nj)


def _energy(st, sel):
    return 0.5 * W.M_E * (st.vx[sel] ** 2 + st.vy[sel] ** 2 + st.vz[sel] ** 2) / W.E_CHARGE


def test_count_law_matching_and_energy(orc):
    counts = [1, 2, 3, 1000, 2500, 4097, 5000]
    k_rec, de = 1e-32, 4.21
    tot_dev, n_obs = 0.0, 0
    for step in range(30):
        wl = _wl(counts, seed=step)
        P = orc.make_params(wl)
        st = orc.State(wl)
        before = (st.vx[:st.n].copy(), st.vy[:st.n].copy(), st.vz[:st.n].copy())
        e_before = np.array([_energy(st, np.nonzero(st.cell[:st.n] == j)[0]).sum() for j in range(len(counts))])
        gone = orc.recombine(st, P, step, k_rec, de)
        cell_after = st.cell[:st.n]
        dead = cell_after < 0
        assert int(dead.sum()) == gone
        changed = (st.vx[:st.n] != before[0]) | (st.vy[:st.n] != before[1]) | (st.vz[:st.n] != before[2])
        assert not np.any(changed & dead)
        pr = _prec(wl, counts, k_rec)
        for j, c in enumerate(counts):
            members = np.nonzero(wl["cell"] == j)[0]
            nd = int(dead[members].sum())
            nc = int(changed[members].sum())
            assert nc == nd, (step, j, nc, nd)
            if c < 2:
                assert nd == 0
                continue
            t = pr[j] * c
            assert nd in (min(math.floor(t), c // 2), min(math.ceil(t), c // 2)), (step, j, nd, t)
            if t < c // 2 - 1:
                tot_dev += nd - t
                n_obs += 1
            live = members[~dead[members]]
            e_after = _energy(st, live).sum()
            assert abs(e_after - (e_before[j] + nd * de)) <= 1e-12 * max(e_before[j], 1.0), (step, j)
        mom, _ = orc.moments(st, P)
        assert int(mom[:, 0].sum()) == st.n - gone
    assert n_obs > 50 and abs(tot_dev / n_obs) < 4 * 0.5 / math.sqrt(n_obs)


def test_cap_at_half_the_cell(orc):
    counts = [10, 11, 4098]
    wl = _wl(counts, seed=7)
    P = orc.make_params(wl)
    st = orc.State(wl)
    gone = orc.recombine(st, P, 0, 1e-20, 4.21)         # P_rec = 1
    assert gone == sum(c // 2 for c in counts)


def test_catalyte_directions_isotropic(orc):
    counts = [5000] * 8
    dirs = []
    for step in range(10):
        wl = _wl(counts, seed=100 + step, T=0.01)           # cold: the new speed is mostly dE_rec
        P = orc.make_params(wl)
        st = orc.State(wl)
        v0 = st.vx[:st.n].copy()
        orc.recombine(st, P, step, 1e-32, 4.21)
        ch = (st.vx[:st.n] != v0) & (st.cell[:st.n] >= 0)
        v = np.stack([st.vx[:st.n][ch], st.vy[:st.n][ch], st.vz[:st.n][ch]], 1)
        dirs.append(v / np.linalg.norm(v, axis=1, keepdims=True))
    d = np.concatenate(dirs)
    n = d.shape[0]
    assert n > 500
    assert np.abs(d.mean(0)).max() < 4 * math.sqrt(1 / 3 / n)
    assert np.abs((d ** 2).mean(0) - 1 / 3).max() < 4 * math.sqrt(4 / 45 / n)


def test_bijection_mode_uses_its_pairing_order(orc):
    """The primaries are the last positions of the cell's pairing order, whichever the mode."""
    counts = [6000]
    wl = _wl(counts, seed=9)
    for mode in (orc.PAIR_KEY, orc.PAIR_BIJECTION):
        P = orc.make_params(wl, pairing_mode=mode)
        st = orc.State(wl)
        _, order = orc.pair_order_mode(wl["cell"], 1, P, 3)
        gone = orc.recombine(st, P, 3, 1e-32, 4.21)
        assert gone > 0
        assert np.array_equal(np.sort(np.nonzero(st.cell[:st.n] < 0)[0]), np.sort(order[-gone:]))
