"""GPU tests of the storage compaction (ltpc_compact) through the C ABI.

Compaction is data movement only.  Bars: after it the storage is grouped by
cell, each cell's particles in its grouping order (for the bijection mode:
ascending old id, which is numpy's stable sort by cell of the old storage),
the velocities bit-identical to the old ones they came from, removed
particles dropped; the next steps on the compacted storage match the oracle
run on the read-back arrays (FP64 within 1e-12 per particle).
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


def _vel_err(v_gpu, v_ref):
    d = np.sqrt(sum((a - b) ** 2 for a, b in zip(v_gpu, v_ref)))
    nrm = np.sqrt(sum(b * b for b in v_ref))
    floor = 1e-3 * np.sqrt(np.mean(nrm * nrm)) if nrm.size else 1.0
    return d / np.maximum(nrm, floor)


def cells_workload(counts, seed=3, T_eV=14.0, dt=3e-11, pairing_mode=1):
    counts = np.asarray(counts, np.int64)
    M = counts.size
    rng = np.random.default_rng([seed, 17])
    n = int(counts.sum())
    vt = math.sqrt(T_eV * W.E_CHARGE / W.M_E)
    cell = np.repeat(np.arange(M, dtype=np.int32), counts)
    wl = W._base(M, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt, vz=rng.standard_normal(n) * vt,
                 cell=cell, inv_vol=np.full(M, 1e15), dt_cell=np.full(M, dt), lnlam_cell=np.full(M, 10.0), seed=seed,
                 capacity=2 * n, pairing_mode=pairing_mode)
    return wl


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_compact_order_values_and_next_steps(L, orc, prec):
    wl = cells_workload([4097, 6000, 300, 9001, 5, 4500], seed=5)
    if prec == "f32":
        for k in ("vx", "vy", "vz"):
            wl[k] = wl[k].astype(np.float32).astype(np.float64)
    col = L.Collider.from_workload(wl, precision=L.F64 if prec == "f64" else L.F32, correction=0)
    col.load_workload(wl)
    for s in range(3):                                   # ionization appends outside the cells' runs
        col.step(col.dt, s)
    col.sync()
    px, py, pz, pc, _ = col.read()
    assert px.size > wl["vx"].size                        # there are appended particles
    assert not np.all(np.diff(pc) >= 0)
    col.compact()
    col.sync()
    gx, gy, gz, gc, _ = col.read()
    order = np.argsort(pc, kind="stable")
    assert gx.size == px.size
    assert np.array_equal(gc, pc[order])
    for a, b in zip((gx, gy, gz), (px, py, pz)):
        assert np.array_equal(a, b[order])
    mom, _ = col.moments()
    col.sync()
    assert np.array_equal(mom[:, 0], np.bincount(gc, minlength=wl["M"]).astype(np.float64))
    if prec == "f32":
        return
    # the next steps on the compacted storage against the oracle from the read-back arrays
    wl2 = dict(wl, vx=gx.copy(), vy=gy.copy(), vz=gz.copy(), cell=gc.copy(), capacity=wl["capacity"])
    st = orc.State(wl2)
    P = orc.make_params(wl2)
    for s in range(3, 5):
        col.step(col.dt, s)
        orc.step(st, P, s)
        col.sync()
        hx, hy, hz, hc, _ = col.read()
        assert hx.size == st.n and np.array_equal(hc, st.cell[:st.n]), s
        err = _vel_err((hx, hy, hz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        assert err.max() <= 1e-12, (s, err.max())


def test_compact_drops_removed_particles(L):
    """Key sort with absorbing walls: the particles that left are dropped, the rest keep
    their values, per cell."""
    M, ppc, dx = 8, 500, 1e-4
    rng = np.random.default_rng(9)
    n = M * ppc
    vt = math.sqrt(200.0 * W.E_CHARGE / W.M_E)
    cell = np.repeat(np.arange(M, dtype=np.int32), ppc)
    wl = W._base(M, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt, vz=rng.standard_normal(n) * vt,
                 cell=cell, x=(cell + rng.random(n)) * dx, inv_vol=np.full(M, 1e15), dt_cell=np.full(M, 1e-10),
                 lnlam_cell=np.full(M, 10.0), seed=9, capacity=2 * n, neutral=False)
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.set_field(dx, np.zeros(M), L.WALL_ABSORB)
    col.load_workload(wl)
    col.push(col.dt, 0)
    col.sync()
    px, py, pz, pc, pxx = col.read()
    gone = int((pc < 0).sum())
    assert gone > 0
    col.compact()
    col.sync()
    gx, gy, gz, gc, gxx = col.read()
    assert gx.size == px.size - gone and np.all(gc >= 0) and np.all(np.diff(gc) >= 0)
    for j in range(M):
        a = np.sort(np.stack([px[pc == j], py[pc == j], pz[pc == j], pxx[pc == j]], 1), axis=0)
        b = np.sort(np.stack([gx[gc == j], gy[gc == j], gz[gc == j], gxx[gc == j]], 1), axis=0)
        assert np.array_equal(a, b), j
