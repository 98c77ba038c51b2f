"""GPU parity of recombination C5 (RS0-RS5 of Table 4) through the C ABI.

The oracle runs S1, S2a (C1/C2 with appends, then C5 over the particles of the
step's pairing order) and S3 in the same order as the fused pass.  Bars: FP64
velocities within 1e-12, cell ids (removed primaries -1), counts and moments'
particle numbers exact, over several steps and in every cluster class; FP32
moments within 1e-5; the bijection mode refuses C5.
"""
import numpy as np
import pytest

from paper_2508_06771_gb300 import workloads as W

pytestmark = pytest.mark.gpu

K_REC, DE_REC = 2e-33, 4.21


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


def _workload(counts, seed=5, T_eV=14.0, shuffled=False):
    counts = np.asarray(counts, np.int64)
    rng = np.random.default_rng([seed, 6262])
    n = int(counts.sum())
    vt = np.sqrt(T_eV * W.E_CHARGE / W.M_E)
    cell = np.repeat(np.arange(counts.size, dtype=np.int32), counts)
    v = [rng.standard_normal(n) * vt for _ in range(3)]
    if shuffled:
        p = rng.permutation(n)
        v = [c[p] for c in v]
        cell = cell[p]
    M = counts.size
    return W._base(M, vx=v[0], vy=v[1], vz=v[2], cell=cell, inv_vol=np.full(M, 1e20 / 1000.0),
                   dt_cell=np.full(M, 2e-11), lnlam_cell=np.full(M, 10.0), seed=seed, capacity=2 * n, steps=3,
                   coulomb=True, neutral=True, precision="f64", dt=2e-11)


@pytest.mark.parametrize("shuffled", [False, True])
def test_fp64_steps_with_recombination(L, orc, shuffled):
    counts = [1, 2, 3, 700, 2049, 4097, 9000, 13000, 30001]       # every class of the key-sort tables
    wl = _workload(counts, shuffled=shuffled)
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.set_recombination(K_REC, DE_REC)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    removed = 0
    for s in range(3):
        col.step(col.dt, s)
        n0 = st.n
        orc.coulomb(st, P, s)
        orc.neutral(st, P, s)
        removed += orc.recombine(st, P, s, K_REC, DE_REC, n_start=n0)
        omom, ohist = orc.moments(st, P)
        mom, hist = col.moments()
        col.sync()
        gx, gy, gz, gc, _ = col.read()
        assert gx.size == st.n, s
        assert np.array_equal(gc, st.cell[:st.n]), s
        assert np.array_equal(mom[:, 0], omom[:, 0]) and np.array_equal(hist, ohist), s
        live = gc >= 0
        err = _vel_err((gx[live], gy[live], gz[live]), (st.vx[:st.n][live], st.vy[:st.n][live], st.vz[:st.n][live]))
        assert err.max() <= 1e-12, (s, err.max())
    assert removed > 100
    # the grouping after removals holds exactly the live particles
    cs, perm, cnt = col.grouping()
    ocounts, ocs, operm = orc.group(gc, wl["M"])
    assert np.array_equal(cnt, ocounts) and np.array_equal(cs.astype(np.uint64), ocs)
    for j in range(wl["M"]):
        a, b = int(ocs[j]), int(ocs[j + 1])
        assert np.array_equal(np.sort(perm[a:b]), operm[a:b]), j


def test_fp32_moments_with_recombination(L, orc):
    wl = _workload([5000] * 12, seed=8, T_eV=6.0)
    wl["n_neutral"] = 0.0                                    # C5 alone besides Coulomb
    for k in ("vx", "vy", "vz"):
        wl[k] = wl[k].astype(np.float32).astype(np.float64)
    col = L.Collider.from_workload(wl, precision=L.F32)
    col.set_recombination(K_REC, DE_REC)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl, correction=True)
    col.step(col.dt, 0)
    n0 = st.n
    orc.coulomb(st, P, 0)
    gone = orc.recombine(st, P, 0, K_REC, DE_REC, n_start=n0)
    omom, _ = orc.moments(st, P)
    mom, _ = col.moments()
    col.sync()
    assert gone > 0
    assert np.array_equal(mom[:, 0], omom[:, 0])
    N = omom[:, 0]
    vrms = np.sqrt(omom[:, 5:8].sum(1) / N)
    e1 = np.abs(mom[:, 2:5] - omom[:, 2:5]) / (N * vrms)[:, None]
    e2 = np.abs(mom[:, 5:8] - omom[:, 5:8]) / omom[:, 5:8]
    assert e1.max() <= 1e-5 and e2.max() <= 1e-5, (e1.max(), e2.max())


def test_bijection_mode_refuses_recombination(L):
    wl = _workload([5000], seed=2)
    wl["pairing_mode"] = 1
    col = L.Collider.from_workload(wl, precision=L.F32)
    with pytest.raises(L.LtpcError) as ei:
        col.set_recombination(K_REC, DE_REC)
    assert ei.value.code == L.EINVAL
