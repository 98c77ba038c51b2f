"""GPU parity of steps S2b/S2c (push in a per-cell field, re-binning, walls) through the C ABI.

The oracle runs the same order: S1 Coulomb, S2a neutral (appends), S2b/S2c push
of every particle, S3 moments of the pushed particles in their new cells.  Bars:
FP64 velocities and positions within 1e-12 (relative to the speed / domain
length), cell ids, counts, grouping and pairing order exact; FP32 moments within
1e-5 in the cells no particle crosses within 1e-5 dx of a cell edge.
"""
import math

import numpy as np
import pytest

from paper_2508_06771_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


DX = 1e-4


def push_workload(M=24, mean_ppc=300, seed=5, T_eV=12.0, dt=1e-11, shuffled=True):
    wl = W.ragged(M=M, mean_ppc=mean_ppc, seed=seed, T_eV=T_eV, shuffled=shuffled)
    rng = np.random.default_rng([seed, 3131])
    wl["x"] = (wl["cell"] + rng.random(wl["cell"].size)) * DX
    wl["dt_cell"] = np.full(M, dt)
    wl["accel"] = rng.uniform(-3e15, 3e15, M)
    return wl


def _collider(L, wl, prec, boundary, **kw):
    col = L.Collider.from_workload(wl, precision=L.F32 if prec == "f32" else L.F64, **kw)
    col.set_field(DX, wl["accel"], boundary)
    return col


def test_binning_at_load(L, orc):
    wl = push_workload(shuffled=True)
    col = _collider(L, wl, "f64", L.WALL_PERIODIC)
    col.load(wl["vx"], wl["vy"], wl["vz"], None, wl["x"])
    _, _, _, cell, x = col.read()
    ref = np.array([orc.bin_position(v, DX, wl["M"]) for v in wl["x"]], np.int32)
    assert np.array_equal(cell, ref)
    assert np.array_equal(cell, wl["cell"])
    bad = wl["x"].copy()
    bad[7] = -DX
    with pytest.raises(L.LtpcError) as ei:
        col.load(wl["vx"], wl["vy"], wl["vz"], None, bad)
    assert ei.value.code == L.EINVAL


def _vel_err(v_gpu, v_ref):
    d = np.sqrt(sum((a - b) ** 2 for a, b in zip(v_gpu, v_ref)))
    nrm = np.sqrt(sum(b * b for b in v_ref))
    floor = 1e-3 * np.sqrt(np.mean(nrm * nrm)) if nrm.size else 1.0
    return d / np.maximum(nrm, floor)


@pytest.mark.parametrize("boundary", ["periodic", "absorb"])
def test_fp64_steps_with_push(L, orc, boundary):
    """Three full steps (Coulomb, neutral with appends, push) against the oracle."""
    wl = push_workload(T_eV=15.0 if boundary == "periodic" else 60.0, dt=2e-11)
    wall = L.WALL_PERIODIC if boundary == "periodic" else L.WALL_ABSORB
    col = _collider(L, wl, "f64", wall, correction=0)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    owall = orc.BOUNDARY_PERIODIC if boundary == "periodic" else orc.BOUNDARY_ABSORB
    gone = 0
    Ld = wl["M"] * DX
    for s in range(3):
        col.step(col.dt, s)
        orc.coulomb(st, P, s)
        orc.neutral(st, P, s)
        gone += orc.push(st, wl["accel"], DX, owall)
        omom, ohist = orc.moments(st, P)
        mom, hist = col.moments()
        col.sync()
        gx, gy, gz, gc, gpos = col.read()
        assert gx.size == st.n
        assert np.array_equal(gc, st.cell[:st.n]), s
        assert np.abs(gpos - st.x[:st.n]).max() <= 1e-12 * Ld, s
        err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        assert err.max() <= 1e-12, (s, err.max())
        assert np.array_equal(mom[:, 0], omom[:, 0]) and np.array_equal(hist, ohist), s
    if boundary == "absorb":
        assert gone > 0 and int((gc < 0).sum()) == gone


def test_grouping_and_pairing_after_push(L, orc):
    wl = push_workload(shuffled=False, T_eV=20.0, dt=3e-11)
    col = _collider(L, wl, "f64", L.WALL_PERIODIC)
    col.load_workload(wl)
    for s in range(2):
        col.step(col.dt, s)
    col.sync()
    _, _, _, cell, _ = col.read()
    assert not np.all(np.diff(cell) >= 0), "particles did not change cells"
    cs, perm, cnt = col.grouping()
    ocounts, ocs, operm = orc.group(cell, wl["M"])
    assert np.array_equal(cnt, ocounts) and np.array_equal(cs.astype(np.uint64), ocs)
    for j in range(wl["M"]):
        a, b = int(ocs[j]), int(ocs[j + 1])
        assert np.array_equal(np.sort(perm[a:b]), operm[a:b]), j
    gcs, gorder = col.pair_order(2)
    _, oorder = orc.pair_order(cell, wl["M"], wl["seed"], 2)
    assert np.array_equal(gorder, oorder)


def test_fp32_moments_with_push(L, orc):
    """FP32 Coulomb steps with push against the FP64 oracle from the same binary32 values."""
    wl = push_workload(M=16, mean_ppc=2000, T_eV=5.0, dt=1e-11)
    wl["neutral"] = False
    for k in ("vx", "vy", "vz", "x"):
        wl[k] = wl[k].astype(np.float32).astype(np.float64)
    col = _collider(L, wl, "f32", L.WALL_PERIODIC)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl, correction=True)
    vth = math.sqrt(2.0 * W.E_CHARGE / W.M_E)
    col.step(col.dt, 0)
    orc.coulomb(st, P, 0)
    x_before = st.x[:st.n].copy()
    orc.push(st, wl["accel"], DX, orc.BOUNDARY_PERIODIC)
    omom, _ = orc.moments(st, P)
    mom, _ = col.moments()
    col.sync()
    # cells a particle enters or leaves within 1e-5 dx of an edge may differ by that particle
    frac = st.x[:st.n] / DX - np.floor(st.x[:st.n] / DX)
    edge = (frac < 1e-5) | (frac > 1 - 1e-5)
    near = np.zeros(wl["M"], bool)
    near[st.cell[:st.n][edge]] = True
    near[np.clip(st.cell[:st.n][edge] - 1, 0, None)] = True
    near[np.clip(st.cell[:st.n][edge] + 1, None, wl["M"] - 1)] = True
    ok = ~near
    assert ok.sum() >= wl["M"] - 3
    N = np.maximum(omom[:, 0], 1)
    assert np.array_equal(mom[ok, 0], omom[ok, 0])
    e_mean = np.abs(mom[ok, 2:5] - omom[ok, 2:5]) / (N[ok, None] * vth)
    e_sq = np.abs(mom[ok, 5:8] - omom[ok, 5:8]) / omom[ok, 5:8]
    assert e_mean.max() <= 1e-5 and e_sq.max() <= 1e-5, (e_mean.max(), e_sq.max())
    assert np.abs(x_before).max() > 0
