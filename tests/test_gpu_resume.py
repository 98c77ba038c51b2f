"""GPU: checkpoint and resume.

A pass takes each cell's state before the Coulomb step (for the momentum and
energy restoration) from the moments the previous pass left, and every random
number is a function of (seed, particle id, step, use).  So a checkpoint is the
particles, the moments and the next step number.  A run resumed from one, on a
fresh context, must reproduce the uninterrupted run bit for bit, including the
ionization secondaries appended on the way.
"""
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


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_resume_is_bit_exact(L, prec):
    wl = W.ragged(M=24, mean_ppc=400, seed=12, T_eV=30.0)
    wl["dt_cell"] = np.full(wl["M"], 5e-11)          # frequent e-n collisions: secondaries appended
    kw = dict(precision=L.F32 if prec == "f32" else L.F64, correction=1)

    whole = L.Collider.from_workload(wl, **kw)
    whole.load_workload(wl)
    for s in range(6):
        whole.step(whole.dt, s)
    ref_v = whole.read()
    ref_mom, ref_hist = whole.moments()
    whole.sync()

    first = L.Collider.from_workload(wl, **kw)
    first.load_workload(wl)
    for s in range(3):
        first.step(first.dt, s)
    vx, vy, vz, cell, _ = first.read()
    mom, hist = first.moments()
    first.sync()
    assert vx.size > wl["vx"].size, "no secondaries appended before the checkpoint"

    resumed = L.Collider.from_workload(wl, **kw)
    resumed.load(vx, vy, vz, cell)
    resumed.set_moments(mom, hist)
    for s in range(3, 6):
        resumed.step(resumed.dt, s)
    got_v = resumed.read()
    got_mom, got_hist = resumed.moments()
    resumed.sync()

    for a, b in zip(got_v[:4], ref_v[:4]):
        assert a.shape == b.shape and np.array_equal(a, b)
    assert np.array_equal(got_mom, ref_mom)
    assert np.array_equal(got_hist, ref_hist)
