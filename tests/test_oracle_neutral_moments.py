"""Pins for the oracle's electron-neutral null-collision step, moments and Coulomb logarithm.

Checked against analytic collision counts (binomial, within 4 sigma), the
Maxwellian mean collision frequency, the mean elastic energy loss 2m/M per
collision, exact particle and energy bookkeeping, numpy bincount sums, and
hand-evaluated formulary values.
"""
import math

import numpy as np
import pytest

from paper_2508_06771_gb300 import workloads as W


def _maxwell_cell(n, T_eV, seed, M=1):
    rng = np.random.default_rng(seed)
    vt = math.sqrt(T_eV * W.E_CHARGE / W.M_E)
    wl = W.ragged(M=M, mean_ppc=n, seed=seed, with_empty=False)
    cell = np.repeat(np.arange(M, dtype=np.int32), n)
    wl.update(vx=rng.standard_normal(n * M) * vt, vy=rng.standard_normal(n * M) * vt,
              vz=rng.standard_normal(n * M) * vt, cell=cell, capacity=3 * n * M,
              dt_cell=np.full(M, 2e-12), counts=np.full(M, n))
    return wl


def _speed(st, n):
    return np.sqrt(st.vx[:n] ** 2 + st.vy[:n] ** 2 + st.vz[:n] ** 2)


def test_null_collision_counts_match_expectation(orc):
    n = 200_000
    wl = _maxwell_cell(n, 20.0, seed=2)
    P = orc.make_params(wl)
    st = orc.State(wl)
    v = _speed(st, n)
    numax = wl["n_neutral"] * (wl["sigma_el"] + wl["sigma_ion"]) * v.max()
    pnull = -math.expm1(-numax * wl["dt_cell"][0])
    E = 0.5 * W.M_E * v * v / W.E_CHARGE
    nu_el = wl["n_neutral"] * wl["sigma_el"] * v
    nu_ion = np.where(E >= wl["e_ion"], wl["n_neutral"] * wl["sigma_ion"] * v, 0.0)
    out = orc.neutral(st, P, step=3, with_decisions=True)
    for key, rate in (("elastic", nu_el), ("ionization", nu_ion)):
        p = pnull * rate / numax
        mean, sd = p.sum(), math.sqrt((p * (1 - p)).sum())
        assert abs(out[key] - mean) < 4 * sd, (key, out[key], mean, sd)
    mean, sd = n * pnull, math.sqrt(n * pnull * (1 - pnull))
    assert abs(out["candidates"] - mean) < 4 * sd
    # bookkeeping: N grows by exactly the ionizations, decisions agree with counts
    assert st.n == n + out["ionization"]
    assert int((out["decision"] == 3).sum()) == out["ionization"]
    assert int((out["decision"] == 2).sum()) == out["elastic"]
    assert int((out["decision"] >= 1).sum()) == out["candidates"]


def test_maxwellian_mean_collision_frequency(orc):
    # <nu_el> = n_n sigma_el sqrt(8 kT / (pi m)) for a Maxwellian; sigma_ion switched off.
    n, T = 400_000, 2.0
    wl = _maxwell_cell(n, T, seed=4)
    wl["sigma_ion"] = 0.0
    P = orc.make_params(wl)
    st = orc.State(wl)
    v = _speed(st, n)
    numax = wl["n_neutral"] * wl["sigma_el"] * v.max()
    pnull = -math.expm1(-numax * wl["dt_cell"][0])
    out = orc.neutral(st, P, step=0)
    nu_mean = wl["n_neutral"] * wl["sigma_el"] * math.sqrt(8 * T * W.E_CHARGE / (math.pi * W.M_E))
    expect = n * pnull * nu_mean / numax
    assert abs(out["elastic"] - expect) < 4 * math.sqrt(expect) + 3 * expect * math.sqrt(1.0 / n)


def test_elastic_energy_loss_and_bookkeeping(orc):
    n = 300_000
    wl = _maxwell_cell(n, 5.0, seed=6)
    wl["dt_cell"] = np.full(1, 5e-11)   # many collisions
    P = orc.make_params(wl)
    st = orc.State(wl)
    v0 = np.stack([st.vx[:n].copy(), st.vy[:n].copy(), st.vz[:n].copy()], 1)
    E0 = 0.5 * W.M_E * (v0 ** 2).sum(1) / W.E_CHARGE
    out = orc.neutral(st, P, step=9, with_decisions=True)
    dec = out["decision"]
    v1 = np.stack([st.vx[:n], st.vy[:n], st.vz[:n]], 1)
    E1 = 0.5 * W.M_E * (v1 ** 2).sum(1) / W.E_CHARGE
    el = dec == 2
    # fractional loss off a cold heavy target averages 2 m/M over isotropic scattering
    frac = (E0[el] - E1[el]) / E0[el]
    want = 2 * W.M_E / wl["mass_neutral"]
    assert abs(frac.mean() - want) < 4 * frac.std() / math.sqrt(el.sum())
    # untouched particles keep their velocity bit-for-bit
    assert np.array_equal(v1[dec <= 1], v0[dec <= 1])
    # energy bookkeeping: total drops by E_ion per ionization plus the elastic losses
    n1 = st.n
    Esec = 0.5 * W.M_E * (st.vx[n:n1] ** 2 + st.vy[n:n1] ** 2 + st.vz[n:n1] ** 2) / W.E_CHARGE
    total_after = E1.sum() + Esec.sum()
    expect = E0.sum() - wl["e_ion"] * out["ionization"] - (E0[el] - E1[el]).sum()
    assert math.isclose(total_after, expect, rel_tol=1e-12)


def test_secondaries_appended_in_cell_then_pairing_order(orc):
    M, n = 5, 20_000
    wl = _maxwell_cell(n, 30.0, seed=8, M=M)
    # interleave cells so parent order differs from cell order
    rng = np.random.default_rng(1)
    p = rng.permutation(n * M)
    for k in ("vx", "vy", "vz", "cell"):
        wl[k] = wl[k][p]
    wl["x"] = np.arange(n * M, dtype=np.float64)          # carried position = original index
    wl["dt_cell"] = np.full(M, 2e-11)
    P = orc.make_params(wl)
    st = orc.State(wl)
    out = orc.neutral(st, P, step=1, with_decisions=True)
    N0 = n * M
    parents = np.where(out["decision"] == 3)[0]
    cells = wl["cell"][parents]
    keys = np.array([orc.draw(wl["seed"], int(l), 1, orc.TAG_PARTICLE)[0] for l in parents], np.uint64)
    want = parents[np.lexsort((parents, keys, cells))]   # cell, then (pairing key, index)
    assert st.n == N0 + parents.size
    assert np.array_equal(st.cell[N0:st.n], wl["cell"][want])
    assert np.array_equal(st.x[N0:st.n], wl["x"][want])


def test_capacity_overflow_reported(orc):
    wl = _maxwell_cell(5000, 40.0, seed=10)
    wl["dt_cell"] = np.full(1, 1e-10)
    P = orc.make_params(wl)
    st = orc.State(wl, capacity=5000)
    with pytest.raises(OverflowError):
        orc.neutral(st, P, step=0)


def test_moments_match_numpy(orc):
    wl = W.ragged(M=23, mean_ppc=50, seed=12, shuffled=True)
    P = orc.make_params(wl)
    st = orc.State(wl)
    mom, hist = orc.moments(st, P)
    vx, vy, vz, cell = st.views()
    M = wl["M"]
    bc = lambda w: np.bincount(cell, weights=w, minlength=M)
    v = np.sqrt(vx ** 2 + vy ** 2 + vz ** 2)
    E = 0.5 * W.M_E * v * v / W.E_CHARGE
    cols = [np.bincount(cell, minlength=M).astype(float), bc(np.full(cell.size, wl["weight"])),
            bc(vx), bc(vy), bc(vz), bc(vx * vx), bc(vy * vy), bc(vz * vz), bc(wl["sigma_el"] * v),
            bc(np.where(E >= wl["e_ion"], wl["sigma_ion"], 0.0) * v)]
    np.testing.assert_allclose(mom, np.stack(cols, 1), rtol=1e-12, atol=0)
    edges = np.logspace(-2, 3, 65)
    b = np.clip(np.searchsorted(edges, E, side="right") - 1, 0, 63)
    want = np.zeros((M, 64), np.int64)
    np.add.at(want, (cell, b), 1)
    near = np.abs(np.log10(E)[:, None] - np.log10(edges)[None, :]).min(1) < 1e-9
    assert not near.any()
    assert np.array_equal(hist, want)


def test_energy_bin_edges(orc):
    for b in range(64):
        e = 10 ** (-2 + 5 * b / 64)
        assert orc.energy_bin(e * (1 + 1e-9)) == b
        if b:
            assert orc.energy_bin(e * (1 - 1e-9)) == b - 1
    assert orc.energy_bin(0.0) == 0 and orc.energy_bin(1e-9) == 0 and orc.energy_bin(1e9) == 63


def test_nrl_lnlambda_values(orc):
    # 23.5 - ln(n^1/2 T^-5/4) - sqrt(1e-5 + (ln T - 2)^2 / 16), n in cm^-3, T in eV
    assert math.isclose(orc.nrl_lnlambda(1e18, 1.0), 23.5 - math.log(1e6) - math.sqrt(1e-5 + 0.25),
                        rel_tol=1e-14)
    T = math.exp(2.0)
    assert math.isclose(orc.nrl_lnlambda(1e20, T), 23.5 - math.log(1e7 * T ** -1.25) - math.sqrt(1e-5),
                        rel_tol=1e-14)
    assert orc.nrl_lnlambda(1e40, 0.01) == 2.0
