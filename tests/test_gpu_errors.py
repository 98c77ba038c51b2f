"""GPU error paths through the C ABI, checked against the oracle where a result exists.

* Out-of-range cell ids in a load large enough that every thread of the
  load-time histogram and of the scatter runs many loop iterations: the
  grouping of the valid particles equals the oracle's, and the deferred error
  is EINVAL.
* A cell larger than the largest compiled class: the load and the next pass
  report EUNSUPPORTED, and every other cell still collides exactly as the
  oracle's run of those cells alone.
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


def _cells_workload(counts, seed, shuffled, T_eV=2.0, dens=1e18):
    counts = np.asarray(counts, np.int64)
    M = counts.size
    rng = np.random.default_rng([seed, 5150])
    n = int(counts.sum())
    vt = math.sqrt(T_eV * W.E_CHARGE / W.M_E)
    cell = np.repeat(np.arange(M, dtype=np.int32), counts)
    vx, vy, vz = (rng.standard_normal(n) * vt for _ in range(3))
    if shuffled:
        p = rng.permutation(n)
        vx, vy, vz, cell = vx[p], vy[p], vz[p], cell[p]
    dt = 0.1 / W.nrl_nu_e(dens, T_eV, 10.0)
    return W._base(M, vx=vx, vy=vy, vz=vz, cell=cell.astype(np.int32), inv_vol=np.full(M, dens / 1000.0),
                   dt_cell=np.full(M, dt), lnlam_cell=np.full(M, 10.0), seed=seed, capacity=2 * n, steps=1,
                   coulomb=True, neutral=False, precision="f64", dt=dt)


def test_async_load_bad_ids_many_loop_iterations(L, orc):
    """3.2 M particles (about ten histogram and scatter loop iterations per thread) with a
    handful of out-of-range ids, negative and too large, spread over the array."""
    import torch
    wl = _cells_workload(np.full(320, 10000), seed=41, shuffled=True)
    n = wl["vx"].size
    bad_at = np.array([0, 31, 32, 777_777, 1_500_001, 2_999_999, n - 1])
    cell = wl["cell"].copy()
    cell[bad_at] = np.array([-1, wl["M"], -7, wl["M"] + 100, 2 ** 31 - 1, -2 ** 31, wl["M"]], dtype=np.int64)
    host = [torch.from_numpy(np.ascontiguousarray(wl[k])).pin_memory() for k in ("vx", "vy", "vz")]
    hcell = torch.from_numpy(np.ascontiguousarray(cell, dtype=np.int32)).pin_memory()
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_host(*(h.numpy() for h in host), hcell.numpy(), asynchronous=True)
    assert col.sync_code() == L.EINVAL
    cs, perm, cnt = col.grouping()
    valid = np.ones(n, bool)
    valid[bad_at] = False
    vidx = np.nonzero(valid)[0]
    ocounts, ocs, operm = orc.group(cell[valid], wl["M"])
    assert np.array_equal(cnt, ocounts)
    assert np.array_equal(cs.astype(np.uint64), ocs)
    total = int(ocs[-1])
    assert total == n - bad_at.size
    for j in range(wl["M"]):
        a, b = int(ocs[j]), int(ocs[j + 1])
        assert np.array_equal(np.sort(perm[a:b]), vidx[operm[a:b]]), j
    col.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_cell_above_largest_class_unsupported(L, orc, prec):
    """One cell one particle above the largest class (65536 in FP32, 49152 in FP64): the load
    and the pass report EUNSUPPORTED; the other cells collide as the oracle's run of them alone."""
    big = 65537 if prec == "f32" else 49153
    wl = _cells_workload([700, big, 301, 2], seed=43, shuffled=False)
    col = L.Collider.from_workload(wl, precision=L.F32 if prec == "f32" else L.F64, correction=0)
    with pytest.raises(L.LtpcError) as ei:
        col.load_workload(wl)
    assert ei.value.code == L.EUNSUPPORTED
    vx0, vy0, vz0, cell0, _ = col.read()
    col.collide_coulomb(wl["dt"], 0)
    assert col.sync_code() == L.EUNSUPPORTED
    gx, gy, gz, gc, _ = col.read()
    assert np.array_equal(gc, cell0)
    big_mask = gc == 1
    # the oversized cell is left as it was
    assert np.array_equal(gx[big_mask], vx0[big_mask]) and np.array_equal(gz[big_mask], vz0[big_mask])
    keep = ~big_mask
    sub = W.subset_cells(wl, np.array([0, 2, 3]))
    st = orc.State(sub)
    if prec == "f32":      # the oracle starts from the same binary32 values
        st.vx[:st.n], st.vy[:st.n], st.vz[:st.n] = vx0[keep], vy0[keep], vz0[keep]
    P = orc.make_params(sub)
    orc.coulomb(st, P, 0)
    ref = np.stack([st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]])
    got = np.stack([gx[keep], gy[keep], gz[keep]]).astype(np.float64)
    d = np.linalg.norm(got - ref, axis=0)
    if prec == "f64":      # per particle, relative to its own speed
        err = d / np.linalg.norm(ref, axis=0)
        assert err.max() <= 1e-12, err.max()
    else:                  # binary32 arithmetic: per particle, relative to the rms speed
        err = d / np.sqrt(np.mean(np.sum(ref * ref, axis=0)))
        assert err.max() <= 1e-5, err.max()
    col.close()
