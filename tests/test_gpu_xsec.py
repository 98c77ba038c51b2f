"""GPU parity of the tabulated cross sections and per-particle selection (Sec. 4.2) through the C ABI.

The oracle evaluates the same piecewise-cubic tables (binary64, natural log,
one division, Horner).  Bars: FP64 velocities within 1e-12 per particle,
particle count, cell ids and appended secondaries exact, moments (rate sums
sum sigma(E)|v| included) within 1e-12; FP32 moments within 1e-5 in the cells
where no decision of the oracle lies within 1e-5 of its threshold (binary32
evaluates the tables with the hardware logarithm, about 1e-6 relative).
Null-collision selection runs in both pairing modes (the bijection mode's
large cells go through the home-order kernel); per-particle selection in the
key mode, where it is defined.
"""
import math

import numpy as np
import pytest

from paper_2508_06771_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_06771_gb300 import build as B
    from paper_2508_06771_gb300 import ltpc
    B.build()
    ltpc.load_library()
    return ltpc


def _vel_err(v_gpu, v_ref):
    d = np.sqrt(sum((a - b) ** 2 for a, b in zip(v_gpu, v_ref)))
    nrm = np.sqrt(sum(b * b for b in v_ref))
    floor = 1e-3 * np.sqrt(np.mean(nrm * nrm)) if nrm.size else 1.0
    return d / np.maximum(nrm, floor)


def _mom_err(mom, omom):
    """Per-cell relative errors: N exact; sums of v over N v_rms; the rest relative."""
    N = np.maximum(omom[:, :1], 1)
    vscale = np.sqrt(omom[:, 5:8].sum(1, keepdims=True) / N)
    d = np.abs(mom - omom)
    d[:, 2:5] /= np.maximum(vscale * N, 1e-300)
    for k in (1, 5, 6, 7, 8, 9):
        d[:, k] /= np.maximum(np.abs(omom[:, k]), 1e-300)
    return d


def xs_workload(M=29, mean_ppc=300, seed=11, T_eV=15.0, dt=4e-11, selection=0, shuffled=True):
    wl = W.ragged(M=M, mean_ppc=mean_ppc, seed=seed, shuffled=shuffled, T_eV=T_eV)
    wl["dt_cell"] = np.full(wl["M"], dt)
    wl["xs"] = W.argon_like_tables()
    wl["selection"] = selection
    return wl


def big_xs_workload(counts=(4097, 6000, 1500, 9001), seed=21, T_eV=12.0, dt=3e-11):
    counts = np.asarray(counts)
    rng = np.random.default_rng([seed, 5])
    n = int(counts.sum())
    vt = math.sqrt(T_eV * W.E_CHARGE / W.M_E)
    cell = np.repeat(np.arange(counts.size, dtype=np.int32), counts)
    wl = W._base(counts.size, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt,
                 vz=rng.standard_normal(n) * vt, cell=cell, inv_vol=np.full(counts.size, 1e15),
                 dt_cell=np.full(counts.size, dt), lnlam_cell=np.full(counts.size, 10.0), seed=seed,
                 capacity=2 * n)
    wl["xs"] = W.argon_like_tables()
    return wl


@pytest.mark.parametrize("selection", [0, 1])
def test_fp64_neutral_with_tables(L, orc, selection):
    """One S2a pass (elastic, ionization with appends) against the oracle, both selections."""
    wl = xs_workload(selection=selection)
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    col.collide_neutral(col.dt, 5)
    info = orc.neutral(st, P, 5)
    gx, gy, gz, gc, _ = col.read()
    col.sync()
    assert info["ionization"] > 0 and info["elastic"] > 0
    assert gx.size == st.n
    assert np.array_equal(gc, st.cell[:st.n])
    err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
    assert err.max() <= FP64_TOL, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("selection", [0, 1])
def test_fp64_steps_and_rate_sums(L, orc, selection):
    """Three fused steps (Coulomb, neutral, moments): velocities and all ten moments."""
    wl = xs_workload(M=33, mean_ppc=350, seed=13, T_eV=12.0, dt=1e-11, selection=selection, shuffled=False)
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    for s in range(3):
        col.step(col.dt, s)
        omom, ohist, _ = orc.step(st, P, s)
        mom, hist = col.moments()
        col.sync()
        assert np.array_equal(mom[:, 0], omom[:, 0]) and np.array_equal(hist, ohist), s
        d = _mom_err(mom, omom)
        assert d[:, 1:].max() <= FP64_TOL, (s, d.max(), np.unravel_index(d.argmax(), d.shape))
        gx, gy, gz, _, _ = col.read()
        err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        assert err.max() <= FP64_TOL, (s, err.max())
    assert omom[:, 9].sum() > 0 and omom[:, 8].sum() > 0


def test_fp64_bijection_big_cells_with_tables(L, orc):
    """Bijection pairing: cells above 4096 particles take the home-order kernel."""
    wl = big_xs_workload()
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0, pairing_mode=L.PAIR_BIJECTION)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl, pairing_mode=orc.PAIR_BIJECTION)
    for s in range(2):
        col.step(col.dt, s)
        omom, ohist, info = orc.step(st, P, s)
        mom, hist = col.moments()
        col.sync()
        assert np.array_equal(mom[:, 0], omom[:, 0]) and np.array_equal(hist, ohist), s
        d = _mom_err(mom, omom)
        assert d[:, 1:].max() <= FP64_TOL, (s, d.max())
        gx, gy, gz, gc, _ = col.read()
        assert gx.size == st.n and np.array_equal(gc, st.cell[:st.n])
        err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        assert err.max() <= FP64_TOL, (s, err.max())


@pytest.mark.parametrize("selection", [0, 1])
def test_fp32_moments_with_tables(L, orc, selection):
    wl = xs_workload(M=32, mean_ppc=2000, seed=17, T_eV=10.0, dt=1e-11, selection=selection, shuffled=False)
    for k in ("vx", "vy", "vz"):
        wl[k] = wl[k].astype(np.float32).astype(np.float64)
    col = L.Collider.from_workload(wl, precision=L.F32, correction=1)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl, correction=True)
    orc.coulomb(st, P, 0)
    probe = orc.State(wl)
    probe.vx[:], probe.vy[:], probe.vz[:] = st.vx, st.vy, st.vz
    dec = orc.neutral(probe, P, 0, with_decisions=True)
    near = np.zeros(wl["M"], bool)
    near[st.cell[:st.n][dec["margin"] < 1e-5]] = True
    orc.neutral(st, P, 0)
    omom, _ = orc.moments(st, P)
    col.step(col.dt, 0)
    mom, _ = col.moments()
    col.sync()
    ok = ~near
    assert ok.sum() >= wl["M"] - 8, near.sum()
    assert np.array_equal(mom[ok, 0], omom[ok, 0])
    d = _mom_err(mom, omom)
    assert d[ok][:, 2:10].max() <= FP32_TOL, d[ok][:, 2:10].max(axis=0)


def test_constants_restored(L):
    """Tables off again: the pass is bit-identical to one that never had tables."""
    wl = xs_workload(selection=0)
    outs = []
    for with_tables in (False, True):
        w = dict(wl)
        w.pop("xs")
        col = L.Collider.from_workload(w, precision=L.F64, correction=0)
        if with_tables:
            col.set_cross_sections(*wl["xs"], L.SELECT_PER_PARTICLE)
            col.set_cross_sections(None, None, 0.0, L.SELECT_NULL)
        col.load_workload(w)
        col.run(col.dt, 0, 2)
        outs.append(col.read())
        col.sync()
    for a, b in zip(outs[0][:4], outs[1][:4]):
        assert np.array_equal(a, b)


def test_bad_tables_rejected(L):
    wl = xs_workload(selection=0)
    w = dict(wl)
    w.pop("xs")
    el, ion, smax = wl["xs"]
    col = L.Collider.from_workload(w, precision=L.F64)
    with pytest.raises(L.LtpcError) as ei:
        col.set_cross_sections(el, ion, 0.5 * smax)            # sum above sigma_max
    assert ei.value.code == L.EINVAL
    neg = dict(el, coef=el["coef"] * -1.0)
    with pytest.raises(L.LtpcError):
        col.set_cross_sections(neg, None, smax)
    with pytest.raises(L.LtpcError):
        col.set_cross_sections(dict(el, pieces=0), None, smax)
    with pytest.raises(L.LtpcError):
        col.set_cross_sections(dict(el, pieces=L.XS_MAX_PIECES + 1), None, smax)
    with pytest.raises(L.LtpcError):
        col.set_cross_sections(el, ion, smax, 2)
    bij = L.Collider.from_workload(w, precision=L.F64, pairing_mode=L.PAIR_BIJECTION)
    bij.set_cross_sections(el, ion, smax, L.SELECT_NULL)
    with pytest.raises(L.LtpcError) as ei:
        bij.set_cross_sections(el, ion, smax, L.SELECT_PER_PARTICLE)
    assert ei.value.code == L.EINVAL
