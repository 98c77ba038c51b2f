"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: grouping and pairing order bit-exact; FP64 velocities within 1e-12
relative per particle; FP32 per-cell moments within 1e-5 (see _fp32_bar).
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


def big_cells_workload(counts, seed=3, T_eV=2.0, shuffled=True, dens=1e18):
    """Cells with the given counts (spanning every cluster class), optionally shuffled storage."""
    counts = np.asarray(counts, np.int64)
    M = counts.size
    rng = np.random.default_rng([seed, 77])
    n = int(counts.sum())
    vt = math.sqrt(T_eV * W.E_CHARGE / W.M_E)
    cell = np.repeat(np.arange(M, dtype=np.int32), counts)
    vx, vy, vz = (rng.standard_normal(n) * vt for _ in range(3))
    if shuffled:
        p = rng.permutation(n)
        vx, vy, vz, cell = vx[p], vy[p], vz[p], cell[p]
    dt = 0.1 / W.nrl_nu_e(dens, T_eV, 10.0)
    return W._base(M, vx=vx, vy=vy, vz=vz, cell=cell.astype(np.int32), inv_vol=np.full(M, dens / 1000.0),
                   dt_cell=np.full(M, dt), lnlam_cell=np.full(M, 10.0), seed=seed, capacity=2 * n, steps=3,
                   coulomb=True, neutral=True, precision="f64", dt=dt)


CLASS_EDGES = [1, 2, 3, 5, 100, 2047, 2048, 2049, 4095, 4096, 4097, 9999, 12288, 12289, 30001, 32768, 32769,
               49152]


def _vel_err(v_gpu, v_ref):
    """Per-particle |dv| / max(|v_ref|, 1e-3 v_rms)."""
    d = np.sqrt(sum((a - b) ** 2 for a, b in zip(v_gpu, v_ref)))
    nrm = np.sqrt(sum(b * b for b in v_ref))
    floor = 1e-3 * np.sqrt(np.mean(nrm * nrm)) if nrm.size else 1.0
    return d / np.maximum(nrm, floor)


# ----------------------------------------------------------------------------- grouping, pairing
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_grouping_and_pair_order_bit_exact(L, orc, prec):
    counts = CLASS_EDGES + ([65536] if prec == "f32" else [])
    wl = big_cells_workload(counts, seed=4)
    col = L.Collider.from_workload(wl, precision=L.F32 if prec == "f32" else L.F64)
    col.load_workload(wl)
    cs, perm, cnt = col.grouping()
    ocounts, ocs, operm = orc.group(wl["cell"], wl["M"])
    assert np.array_equal(cnt, ocounts)
    assert np.array_equal(cs.astype(np.uint64), ocs)
    for j in range(wl["M"]):
        a, b = int(ocs[j]), int(ocs[j + 1])
        assert np.array_equal(np.sort(perm[a:b]), operm[a:b]), j
    for step in (0, 1, 12345):
        gcs, gorder = col.pair_order(step)
        ocs2, oorder = orc.pair_order(wl["cell"], wl["M"], wl["seed"], step)
        assert np.array_equal(gcs.astype(np.uint64), ocs2)
        bad = np.nonzero(gorder != oorder)[0]
        assert bad.size == 0, f"step {step}: {bad.size} positions differ, first {bad[:5]}"
    col.sync()


@pytest.mark.parametrize("shuffled", [False, True])
def test_grouping_after_appends(L, orc, shuffled):
    """CCS1-CCS3 after ionization appends: for storage loaded in cell order the loaded particles
    are placed from their cell's run and the appended ones from the cell's cursor; for shuffled
    storage all take the cursor.  Either way each cell's segment holds exactly its particles, and
    the pairing order matches the oracle's."""
    wl = W.ragged(M=24, mean_ppc=400, seed=9, T_eV=30.0, shuffled=shuffled)
    wl["dt_cell"] = np.full(wl["M"], 5e-11)
    col = L.Collider.from_workload(wl, precision=L.F64)
    col.load_workload(wl)
    n0 = col.count()
    for s in range(3):
        col.step(col.dt, s)
    col.sync()
    assert col.count() > n0, "no secondaries appended"
    _, _, _, cell, _ = col.read()
    cs, perm, cnt = col.grouping()
    ocounts, ocs, operm = orc.group(cell, wl["M"])
    assert np.array_equal(cnt, ocounts)
    assert np.array_equal(cs.astype(np.uint64), ocs)
    for j in range(wl["M"]):
        a, b = int(ocs[j]), int(ocs[j + 1])
        assert np.array_equal(np.sort(perm[a:b]), operm[a:b]), j
    if not shuffled:   # cell-ordered load: loaded ids in index order, then the appended ones at their slots
        assert np.array_equal(perm, operm)
    gcs, gorder = col.pair_order(3)
    ocs2, oorder = orc.pair_order(cell, wl["M"], wl["seed"], 3)
    assert np.array_equal(gorder, oorder)
    col.sync()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_every_class_table_pairs_bit_exact(L, orc, prec):
    """Every class table (every compiled block/cluster shape in use) gives the
    oracle's pairing order bit for bit, and the same FP32 moments within 1e-5."""
    counts = [3, 2049, 4097, 12289, 20000, 24577, 32769, 49153, 65536] if prec == "f32" else \
        [3, 2049, 4097, 6145, 12289, 20000, 32768]
    wl = big_cells_workload(counts, seed=8)
    col = L.Collider.from_workload(wl, precision=L.F32 if prec == "f32" else L.F64)
    col.load_workload(wl)
    ocs, oorder = orc.pair_order(wl["cell"], wl["M"], wl["seed"], 7)
    ref = None
    tables = 0
    for t in range(8):
        try:
            col.set_class_table(t)
        except L.LtpcError as e:
            assert e.code == L.EINVAL
            break
        tables += 1
        gcs, gorder = col.pair_order(7)
        assert np.array_equal(gcs.astype(np.uint64), ocs)
        assert np.array_equal(gorder, oorder), t
        col.load_workload(wl)
        col.set_class_table(t)
        col.collide_coulomb(wl["dt"], 0)        # Coulomb only: no discrete decisions to flip
        mom, _ = col.moments()
        if ref is None:
            ref = mom
        else:
            np.testing.assert_array_equal(mom[:, 0], ref[:, 0])
            s2 = ref[:, 5:8]                                          # sums of v_i^2
            s1 = np.sqrt(ref[:, 0:1] * s2)                            # N v_rms per component
            assert (np.abs(mom[:, 2:5] - ref[:, 2:5]) / s1).max() <= 1e-5, t
            assert (np.abs(mom[:, 5:8] - s2) / s2).max() <= 1e-5, t
    assert tables >= 2
    col.sync()


def test_pair_order_ragged_shuffled(L, orc):
    wl = W.ragged(M=41, mean_ppc=400, seed=9, shuffled=True)
    col = L.Collider.from_workload(wl, precision=L.F64)
    col.load_workload(wl)
    gcs, gorder = col.pair_order(7)
    ocs, oorder = orc.pair_order(wl["cell"], wl["M"], wl["seed"], 7)
    assert np.array_equal(gorder, oorder)


# ----------------------------------------------------------------------------- FP64 parity
def _fp64_coulomb_case(L, orc, wl, steps=(0,)):
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    worst = 0.0
    for s in steps:
        # single-step parity from an identical state
        vx, vy, vz, cell, _ = col.read()
        st.vx[:st.n], st.vy[:st.n], st.vz[:st.n] = vx, vy, vz
        col.collide_coulomb(col.dt, s)
        orc.coulomb(st, P, s)
        gx, gy, gz, gc, _ = col.read()
        col.sync()
        err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        worst = max(worst, float(err.max()))
        assert err.max() <= FP64_TOL, (s, err.max(), int(err.argmax()))
    return worst


def test_fp64_coulomb_relax_reduced(L, orc):
    wl = W.relax_64x1000(M=16, ppc=1000)
    _fp64_coulomb_case(L, orc, wl, steps=(0, 1, 2))


def test_fp64_coulomb_all_classes(L, orc):
    wl = big_cells_workload(CLASS_EDGES, seed=5)
    _fp64_coulomb_case(L, orc, wl, steps=(3,))


def test_fp64_neutral_step_and_append(L, orc):
    wl = W.ragged(M=29, mean_ppc=300, seed=11, shuffled=True, T_eV=15.0)
    wl["dt_cell"] = np.full(wl["M"], 4e-11)       # many e-n collisions, some ionizations
    wl["x"] = np.arange(wl["vx"].size, dtype=np.float64) * 1e-3
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    col.collide_neutral(col.dt, 5)
    info = orc.neutral(st, P, 5)
    gx, gy, gz, gc, gpos = col.read()
    col.sync()
    assert info["ionization"] > 0 and info["elastic"] > 0
    assert gx.size == st.n, (gx.size, st.n)
    assert np.array_equal(gc, st.cell[:st.n])
    assert np.array_equal(gpos, st.x[:st.n])
    err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
    assert err.max() <= FP64_TOL, (err.max(), int(err.argmax()))


def test_fp64_fused_step_moments(L, orc):
    wl = W.ragged(M=33, mean_ppc=350, seed=13, shuffled=False, T_eV=12.0)
    wl["dt_cell"] = np.full(wl["M"], 1e-11)
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    for s in range(3):
        vx, vy, vz, cell, _ = col.read()
        st.n = vx.size
        st.vx[:st.n], st.vy[:st.n], st.vz[:st.n], st.cell[:st.n] = vx, vy, vz, cell
        col.step(col.dt, s)
        omom, ohist, _ = orc.step(st, P, s)
        mom, hist = col.moments()
        col.sync()
        assert np.array_equal(mom[:, 0], omom[:, 0])
        scale = np.maximum(np.abs(omom), 1e-300)
        vscale = np.sqrt(omom[:, 5:8].sum(1, keepdims=True) / np.maximum(omom[:, :1], 1))
        d = np.abs(mom - omom)
        d[:, 2:5] /= np.maximum(vscale * np.maximum(omom[:, :1], 1), 1e-300)
        d[:, [1, 5, 6, 7, 8, 9]] /= scale[:, [1, 5, 6, 7, 8, 9]]
        d[:, 0] = 0
        assert d.max() <= 1e-12, (s, d.max(), np.unravel_index(d.argmax(), d.shape))
        assert np.array_equal(hist, ohist)
        gx, gy, gz, _, _ = col.read()
        err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        assert err.max() <= FP64_TOL


# ----------------------------------------------------------------------------- FP32 parity
def _moment_errors(mom, omom, vth):
    """Per-cell errors: N exact, sums of v over N v_th, sums of v^2 and speed sums relative."""
    N = np.maximum(omom[:, 0], 1)
    e = np.zeros_like(omom)
    e[:, 0] = np.abs(mom[:, 0] - omom[:, 0])
    e[:, 2:5] = np.abs(mom[:, 2:5] - omom[:, 2:5]) / (N[:, None] * vth)
    for k in (5, 6, 7, 8, 9):
        e[:, k] = np.abs(mom[:, k] - omom[:, k]) / np.maximum(np.abs(omom[:, k]), 1e-300)
    e[omom[:, 9] == 0, 9] = np.abs(mom[omom[:, 9] == 0, 9]) > 0
    return e


def test_fp32_coulomb_moments(L, orc):
    wl = W.tail_4096x10000(M=48, ppc=2000, steps=3)
    wl["neutral"] = False
    v32 = [wl[k].astype(np.float32) for k in ("vx", "vy", "vz")]
    for k, v in zip(("vx", "vy", "vz"), v32):
        wl[k] = v.astype(np.float64)       # the oracle starts from the same binary32 values
    col = L.Collider.from_workload(wl, precision=L.F32)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl, correction=True)
    vth = math.sqrt(2.0 * W.E_CHARGE / W.M_E)
    for s in range(3):
        col.collide_coulomb(wl["dt"], s)
        orc.coulomb(st, P, s)
        omom, _ = orc.moments(st, P)
        mom, _ = col.moments()
        col.sync()
        e = _moment_errors(mom, omom, vth)
        assert e[:, 0].max() == 0
        assert e[:, 2:9].max() <= FP32_TOL, (s, e[:, 2:9].max(axis=0))


def test_fp32_restoration_with_drift(L, orc):
    """Cells drifting at several times their thermal speed: the restoration's state before S1
    must not lose digits to the drift (the stored moments are not centred).  Each cell's thermal
    energy, sum |v - mean|^2 of the read-back velocities, stays within 1e-6 of the FP64
    oracle's, and the moments within the FP32 bar."""
    wl = W.tail_4096x10000(M=16, ppc=2000, steps=2)
    wl["neutral"] = False
    vth = math.sqrt(2.0 * W.E_CHARGE / W.M_E)
    wl["vz"] = wl["vz"] + 10.0 * vth
    wl["vx"] = wl["vx"] - 4.0 * vth
    for k in ("vx", "vy", "vz"):
        wl[k] = wl[k].astype(np.float32).astype(np.float64)   # the oracle starts from the same values
    col = L.Collider.from_workload(wl, precision=L.F32)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl, correction=True)
    for s in range(2):
        col.collide_coulomb(wl["dt"], s)
        orc.coulomb(st, P, s)
    gx, gy, gz, cell, _ = col.read()
    mom, _ = col.moments()
    col.sync()

    def thermal(vx, vy, vz):
        out = np.zeros(wl["M"])
        for j in range(wl["M"]):
            sel = cell == j
            v = np.stack([vx[sel], vy[sel], vz[sel]], 1).astype(np.float64)
            out[j] = ((v - v.mean(0)) ** 2).sum()
        return out

    Kg = thermal(gx, gy, gz)
    Ko = thermal(st.vx[:st.n], st.vy[:st.n], st.vz[:st.n])
    assert (np.abs(Kg - Ko) / Ko).max() <= 1e-6, (np.abs(Kg - Ko) / Ko).max()
    omom, _ = orc.moments(st, P)
    e = _moment_errors(mom, omom, vth)
    assert e[:, 0].max() == 0
    assert e[:, 2:9].max() <= FP32_TOL, e[:, 2:9].max(axis=0)


def test_fp32_full_step_with_flip_accounting(L, orc):
    wl = W.tail_4096x10000(M=32, ppc=2000, steps=1)
    for k in ("vx", "vy", "vz"):
        wl[k] = wl[k].astype(np.float32).astype(np.float64)
    col = L.Collider.from_workload(wl, precision=L.F32)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl, correction=True)
    vth = math.sqrt(2.0 * W.E_CHARGE / W.M_E)
    orc.coulomb(st, P, 0)
    probe = orc.State(wl)
    probe.vx[:], probe.vy[:], probe.vz[:] = st.vx, st.vy, st.vz
    dec = orc.neutral(probe, P, 0, with_decisions=True)
    near = np.zeros(wl["M"], bool)
    near[st.cell[:st.n][dec["margin"] < 1e-6]] = True
    orc.neutral(st, P, 0)
    omom, _ = orc.moments(st, P)
    col.step(wl["dt"], 0)
    mom, _ = col.moments()
    col.sync()
    e = _moment_errors(mom, omom, vth)
    ok = ~near
    assert near.sum() <= 2, near.sum()
    assert e[ok, 0].max() == 0
    assert e[ok][:, 2:9].max() <= FP32_TOL, e[ok][:, 2:9].max(axis=0)


# ----------------------------------------------------------------------------- determinism, errors
def test_determinism_graph_and_repeat(L):
    wl = W.tail_4096x10000(M=16, ppc=3000, steps=1)
    outs = []
    for use_graph in (True, True, False):
        col = L.Collider.from_workload(wl, precision=L.F32, use_graph=use_graph)
        col.load_workload(wl)
        col.run(wl["dt"], 0, 4)
        outs.append(col.read())
        col.sync()
    for o in outs[1:]:
        for a, b in zip(outs[0][:4], o[:4]):
            assert np.array_equal(a, b)


def test_capacity_overflow_reported(L):
    wl = W.ragged(M=4, mean_ppc=500, seed=2, T_eV=60.0, with_empty=False)
    wl["dt_cell"] = np.full(4, 2e-10)
    col = L.Collider.from_workload(wl, precision=L.F64, capacity=wl["vx"].size)
    col.load_workload(wl)
    col.collide_neutral(col.dt, 0)
    assert col.sync_code() == L.ECAPACITY


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_restoration_after_rolled_back_append(L, orc, prec):
    """After a capacity error the stored moments count secondaries that were never appended, so
    the next Coulomb pass cannot take the restoration's state before S1 from them: it sums the
    velocities itself.  That pass, with the restoration on, against the oracle from the same
    state: FP64 velocities within 1e-12, FP32 moments within 1e-5."""
    wl = W.ragged(M=4, mean_ppc=500, seed=2, T_eV=60.0, with_empty=False)
    wl["dt_cell"] = np.full(4, 2e-10)
    if prec == "f32":
        for k in ("vx", "vy", "vz"):
            wl[k] = wl[k].astype(np.float32).astype(np.float64)
    col = L.Collider.from_workload(wl, precision=L.F64 if prec == "f64" else L.F32, capacity=wl["vx"].size,
                                   correction=1)
    col.load_workload(wl)
    col.collide_neutral(col.dt, 0)
    assert col.sync_code() == L.ECAPACITY
    vx, vy, vz, cell, _ = col.read()
    counts = np.bincount(cell, minlength=wl["M"])
    stored, _ = col.moments()
    assert (stored[:, 0] != counts).any(), "the stored counts should include the dropped secondaries"
    st = orc.State(dict(wl, vx=vx.astype(np.float64), vy=vy.astype(np.float64), vz=vz.astype(np.float64),
                        cell=cell))
    P = orc.make_params(wl, correction=True)
    col.collide_coulomb(col.dt, 1)
    orc.coulomb(st, P, 1)
    assert col.sync_code() == 0
    if prec == "f64":
        gx, gy, gz, _, _ = col.read()
        err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        assert err.max() <= FP64_TOL, (err.max(), int(err.argmax()))
    else:
        omom, _ = orc.moments(st, P)
        mom, _ = col.moments()
        vth = math.sqrt(2.0 * 60.0 * W.E_CHARGE / W.M_E)
        e = _moment_errors(mom, omom, vth)
        assert e[:, 0].max() == 0
        assert e[:, 2:9].max() <= FP32_TOL, e[:, 2:9].max(axis=0)


def test_bad_cell_and_nonfinite_rejected(L):
    wl = W.ragged(M=5, mean_ppc=20, seed=1, with_empty=False)
    col = L.Collider.from_workload(wl, precision=L.F64)
    bad = wl["cell"].copy()
    bad[3] = 5
    with pytest.raises(L.LtpcError) as ei:
        col.load(wl["vx"], wl["vy"], wl["vz"], bad)
    assert ei.value.code == L.EINVAL
    vx = wl["vx"].copy()
    vx[7] = np.nan
    with pytest.raises(L.LtpcError) as ei:
        col.load(vx, wl["vy"], wl["vz"], wl["cell"])
    assert ei.value.code == L.ENONFINITE


def test_async_load_matches_sync_and_defers_errors(L):
    """LTPC_LOAD_ASYNC: the same state as a synchronous load; a bad cell id is
    reported by the next sync, and the particles with valid ids are stepped."""
    import torch
    wl = W.ragged(M=16, mean_ppc=300, seed=6, with_empty=True)
    host = [torch.from_numpy(np.ascontiguousarray(wl[k])).pin_memory() for k in ("vx", "vy", "vz")]
    hcell = torch.from_numpy(np.ascontiguousarray(wl["cell"], dtype=np.int32)).pin_memory()
    res = []
    for asynchronous in (False, True):
        col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
        col.load_host(*(h.numpy() for h in host), hcell.numpy(), asynchronous=asynchronous)
        col.step(wl["dt"], 0)
        assert col.sync_code() == L.OK
        res.append(col.moments())
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])

    bad = hcell.clone()
    bad[5] = wl["M"] + 3
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_host(*(h.numpy() for h in host), bad.numpy(), asynchronous=True)   # no error yet
    col.collide_coulomb(wl["dt"], 0)
    assert col.sync_code() == L.EINVAL
    mom, _ = col.moments()
    assert int(round(mom[:, 0].sum())) == len(wl["vx"]) - 1


@pytest.mark.parametrize("neutral", [False, True])
def test_cached_grouping_identical(L, orc, neutral):
    """cache_grouping skips CCS3 while nothing was loaded or appended; the results are
    bit-identical to grouping every step (with appends the grouping is redone)."""
    wl = W.ragged(M=21, mean_ppc=400, seed=17, shuffled=True, T_eV=14.0)
    wl["dt_cell"] = np.full(wl["M"], 3e-11)
    wl["neutral"] = neutral
    out = []
    for cache in (False, True):
        col = L.Collider.from_workload(wl, precision=L.F64, correction=0, cache_grouping=cache)
        col.load_workload(wl)
        col.run(col.dt, 0, 4)
        mom, hist = col.moments()
        out.append((mom, hist, col.read()))
        assert col.sync_code() == L.OK
    (m0, h0, r0), (m1, h1, r1) = out
    np.testing.assert_array_equal(m0, m1)
    np.testing.assert_array_equal(h0, h1)
    for a, b in zip(r0[:4], r1[:4]):
        np.testing.assert_array_equal(a, b)
