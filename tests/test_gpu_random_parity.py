"""Randomized GPU parity against the oracle (FP64, through the C ABI).

Each seed draws a batch of cells whose sizes mix the edge cases (empty, 1, 2,
3 particles) with every size class (single CTAs up to clusters), stores the
particles in shuffled order, and runs two fused steps (Coulomb, null-collision
e-n with ionization appends, moments).  Per step, from the same state:
pairing order bit-exact, particle count and cells exact, velocities within
1e-12 relative, per-cell moments within 1e-12 and the energy histogram exact.
"""
import numpy as np
import pytest

from test_gpu_parity import FP64_TOL, L, _vel_err, big_cells_workload   # noqa: F401 (L: fixture)

pytestmark = pytest.mark.gpu


def _random_counts(rng):
    M = int(rng.integers(4, 28))
    kind = rng.random(M)
    counts = np.where(kind < 0.08, 0,
             np.where(kind < 0.16, 1,
             np.where(kind < 0.26, rng.integers(2, 4, M),
             np.where(kind < 0.70, rng.integers(4, 3000, M),
             np.where(kind < 0.90, rng.integers(3000, 12289, M), rng.integers(12289, 26000, M))))))
    counts[0] = max(counts[0], 2)
    return [int(c) for c in counts]


@pytest.mark.parametrize("seed", [101, 202, 303])
def test_random_batches_fp64(L, orc, seed):
    rng = np.random.default_rng(seed)
    counts = _random_counts(rng)
    wl = big_cells_workload(counts, seed=seed, T_eV=float(rng.uniform(5.0, 15.0)), shuffled=True)
    wl["dt_cell"] = np.full(wl["M"], float(rng.uniform(1e-11, 4e-11)))   # candidates and a few ionizations
    col = L.Collider.from_workload(wl, precision=L.F64, correction=0)
    col.load_workload(wl)
    st = orc.State(wl)
    P = orc.make_params(wl)
    for s in range(2):
        vx, vy, vz, cell, _ = col.read()
        st.n = vx.size
        st.vx[:st.n], st.vy[:st.n], st.vz[:st.n], st.cell[:st.n] = vx, vy, vz, cell
        gcs, gorder = col.pair_order(s)
        ocs, oorder = orc.pair_order(cell, wl["M"], wl["seed"], s)
        assert np.array_equal(gcs.astype(np.uint64), ocs)
        assert np.array_equal(gorder, oorder), (seed, s)
        col.step(col.dt, s)
        omom, ohist, _ = orc.step(st, P, s)
        mom, hist = col.moments()
        col.sync()
        gx, gy, gz, gc, _ = col.read()
        assert gx.size == st.n, (seed, s, gx.size, st.n)
        assert np.array_equal(gc, st.cell[:st.n])
        err = _vel_err((gx, gy, gz), (st.vx[:st.n], st.vy[:st.n], st.vz[:st.n]))
        assert err.max() <= FP64_TOL, (seed, s, err.max())
        assert np.array_equal(mom[:, 0], omom[:, 0])
        vscale = np.sqrt(omom[:, 5:8].sum(1) / np.maximum(omom[:, 0], 1))
        d = np.abs(mom[:, 2:5] - omom[:, 2:5]) / np.maximum(vscale * np.maximum(omom[:, 0], 1), 1e-300)[:, None]
        assert d.max() <= 1e-12, (seed, s, d.max())
        rel = np.abs(mom[:, 5:10] - omom[:, 5:10]) / np.maximum(np.abs(omom[:, 5:10]), 1e-300)
        assert rel.max() <= 1e-12, (seed, s, rel.max())
        assert np.array_equal(hist, ohist)
