"""Pin of the oracle's id-addressed random streams: a subset of cells run with
the particles' original ids reproduces exactly what the full run does to those
cells (cells are independent in S1 and S2a)."""
import numpy as np

from paper_2508_06771_gb300 import workloads as W


def test_subset_with_ids_equals_full_run(orc):
    wl = W.ragged(M=30, mean_ppc=200, seed=31, shuffled=True, T_eV=20.0)
    wl["dt_cell"] = np.full(wl["M"], 2e-11)
    P = orc.make_params(wl, correction=True)
    full = orc.State(wl)
    orc.coulomb(full, P, 4)
    orc.neutral(full, P, 4)
    fm, fh = orc.moments(full, P)
    cells = np.array([1, 5, 7, 12, 29])
    sub_wl = W.subset_cells(wl, cells)
    sub = orc.State(sub_wl)
    orc.coulomb(sub, P, 4)
    orc.neutral(sub, P, 4)
    sm, sh = orc.moments(sub, P)
    np.testing.assert_array_equal(sm, fm[cells])
    np.testing.assert_array_equal(sh, fh[cells])


def test_subset_keeps_per_cell_arrays_aligned():
    """A subset of an instance batch carries each kept cell's instance label and count."""
    full = W.instances_64(seed=0, instances=[0, 1])
    cells = np.array([0, 7, full["M"] - 1])
    sub = W.subset_cells(full, cells)
    assert np.array_equal(sub["instance_of_cell"], np.asarray(full["instance_of_cell"])[cells])
    assert sub["instance_of_cell"].size == sub["M"] == cells.size
    assert np.array_equal(np.bincount(sub["cell"], minlength=sub["M"]),
                          np.bincount(full["cell"], minlength=full["M"])[cells])
