"""Pins of the oracle's push and re-binning (steps S2b/S2c of Table 2, CS6/CS7 of Table 3).

* Free flight: with no field, K periodic pushes put every particle at
  (x0 + K dt v) mod L, the closed form, and leave the velocities unchanged.
* Uniform field: for the update x+ = x + dt v, v+ = v + dt a, the kinetic energy
  per unit mass grows by a (x+ - x) + a^2 dt^2 / 2 per step (an algebraic
  identity of this update; a dropped or doubled term fails it).
* Re-binning: the cells after a push equal numpy's floor(x / dx) and the counts
  numpy's bincount.
* Absorbing walls: the particles that leave [0, L) are numpy's count, they take
  part in nothing afterwards (grouping, collisions, moments).
"""
import math

import numpy as np

from paper_2508_06771_gb300 import workloads as W


def _wl(M=16, ppc=200, seed=3, T=3.0, dx=1e-4):
    rng = np.random.default_rng(seed)
    n = M * ppc
    vt = math.sqrt(T * W.E_CHARGE / W.M_E)
    x = (np.repeat(np.arange(M), ppc) + rng.random(n)) * dx
    wl = W._base(M, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt,
                 vz=rng.standard_normal(n) * vt, cell=np.repeat(np.arange(M, dtype=np.int32), ppc), x=x,
                 inv_vol=np.full(M, 1e18 / ppc), dt_cell=np.full(M, 2e-11), lnlam_cell=np.full(M, 10.0), seed=seed,
                 capacity=2 * n)
    return wl, dx


def test_free_flight_closed_form(orc):
    wl, dx = _wl()
    M, L, K = wl["M"], wl["M"] * dx, 25
    st = orc.State(wl)
    x0, v0 = st.x[:st.n].copy(), (st.vx[:st.n].copy(), st.vy[:st.n].copy(), st.vz[:st.n].copy())
    for _ in range(K):
        assert orc.push(st, np.zeros(M), dx) == 0
    dt = wl["dt_cell"][0]
    ref = np.mod(x0 + K * dt * v0[2], L)
    d = np.abs(st.x[:st.n] - ref)
    d = np.minimum(d, L - d)                      # the seam: 0 and L are the same point
    assert d.max() <= 1e-12 * L * K
    for a, b in zip((st.vx, st.vy, st.vz), v0):
        assert np.array_equal(a[:st.n], b)
    assert np.all((st.x[:st.n] >= 0) & (st.x[:st.n] < L))


def test_uniform_field_energy_identity(orc):
    wl, dx = _wl(M=64, ppc=50)
    M = wl["M"]
    st = orc.State(wl)
    st.x[:st.n] = st.x[:st.n] * 0.01 + 0.4 * M * dx    # far from the walls: no particle leaves
    a = np.full(M, 3e14)                               # m/s^2
    dt = wl["dt_cell"][0]
    e0 = 0.5 * (st.vx[:st.n] ** 2 + st.vy[:st.n] ** 2 + st.vz[:st.n] ** 2)
    x0 = st.x[:st.n].copy()
    K = 10
    for _ in range(K):
        assert orc.push(st, a, dx, orc.BOUNDARY_ABSORB) == 0
    e1 = 0.5 * (st.vx[:st.n] ** 2 + st.vy[:st.n] ** 2 + st.vz[:st.n] ** 2)
    gain = a[0] * (st.x[:st.n] - x0) + K * 0.5 * a[0] ** 2 * dt ** 2
    assert np.abs((e1 - e0) - gain).max() <= 1e-9 * e0.mean()
    assert np.allclose(st.vz[:st.n], wl["vz"] + K * dt * a[0], rtol=0, atol=1e-9 * np.abs(wl["vz"]).max())


def test_rebinning_matches_numpy(orc):
    wl, dx = _wl(M=32, ppc=300, T=40.0)
    M, L = wl["M"], wl["M"] * dx
    st = orc.State(wl)
    orc.push(st, np.linspace(-1e15, 1e15, M), dx)
    cells = np.floor(st.x[:st.n] / dx).astype(np.int64)
    assert np.array_equal(st.cell[:st.n], np.clip(cells, 0, M - 1))
    counts, cs, perm = orc.group(st.cell[:st.n], M)
    assert np.array_equal(counts, np.bincount(cells, minlength=M))
    assert np.array_equal(cs[1:], np.cumsum(counts))
    assert orc.bin_position(L * (1 - 1e-17), dx, M) == M - 1


def test_absorbing_walls(orc):
    wl, dx = _wl(M=8, ppc=400, T=200.0)
    M, L = wl["M"], wl["M"] * dx
    wl["dt_cell"] = np.full(M, 1e-10)
    st = orc.State(wl)
    dt = wl["dt_cell"][0]
    x1 = st.x[:st.n] + dt * st.vz[:st.n]
    out = (x1 < 0) | (x1 >= L)
    assert out.sum() > 0
    gone = orc.push(st, np.zeros(M), dx, orc.BOUNDARY_ABSORB)
    assert gone == int(out.sum())
    assert np.array_equal(st.cell[:st.n] < 0, out)
    # removed particles take part in nothing: moments count the live ones, Coulomb conserves
    P = orc.make_params(wl)
    mom0, _ = orc.moments(st, P)
    assert int(mom0[:, 0].sum()) == st.n - gone
    dead_v = st.vx[:st.n][out].copy()
    orc.coulomb(st, P, 1)
    mom1, _ = orc.moments(st, P)
    assert np.array_equal(st.vx[:st.n][out], dead_v)
    np.testing.assert_allclose(mom1[:, 2:5], mom0[:, 2:5], rtol=0, atol=1e-9 * np.abs(mom0[:, 2:5]).max())
    e0, e1 = mom0[:, 5:8].sum(1), mom1[:, 5:8].sum(1)
    assert np.abs(e1 - e0).max() <= 1e-12 * e0.max()
    assert orc.push(st, np.zeros(M), dx, orc.BOUNDARY_ABSORB) >= 0
    assert np.all(st.cell[:st.n][out] == -1)
    # the neutral step (with ionization appends) leaves the removed particles alone too
    n_before, dead = st.n, st.cell[:st.n] < 0
    info = orc.neutral(st, P, 2, with_decisions=True)
    assert info["candidates"] > 0 and np.all(info["decision"][dead] == 0)
    assert st.n == n_before + info["ionization"]
    assert np.all(st.cell[n_before:st.n] >= 0)
