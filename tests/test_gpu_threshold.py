"""GPU: electrons at the ionization threshold stay finite.

The electron-neutral step decides an ionization from the particle's energy and
then shares the excess E - E_ion between primary and secondary (Table 3, CS5).
When the energy lies within rounding of E_ion, the excess recomputed in binary32
can come out one unit below zero; the kernel must clamp it instead of taking the
square root of a negative number.  Every particle here sits within a few units
in the last place of the threshold, with a collision probability near one.
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


def threshold_workload(M=64, ppc=2000, seed=11):
    rng = np.random.default_rng([seed, 1576])
    n = M * ppc
    v_thr = math.sqrt(2.0 * W.E_ION * W.E_CHARGE / W.M_E)
    # speeds within +-4 units of 2^-24 of the threshold speed, isotropic directions
    speed = v_thr * (1.0 + rng.integers(-4, 5, n) * 2.0 ** -24)
    c = 1.0 - 2.0 * rng.random(n)
    s = np.sqrt(1.0 - c * c)
    ph = 2.0 * np.pi * rng.random(n)
    vx, vy, vz = speed * s * np.cos(ph), speed * s * np.sin(ph), speed * c
    cell = np.repeat(np.arange(M, dtype=np.int32), ppc)
    dt = 1e-9                       # nu_max dt ~ 9: almost every particle is a candidate
    return W._base(M, vx=vx, vy=vy, vz=vz, cell=cell, inv_vol=np.full(M, 1e18 / ppc), dt_cell=np.full(M, dt),
                   lnlam_cell=np.full(M, 10.0), seed=seed, capacity=2 * n, steps=1, coulomb=False, neutral=True,
                   precision="f32", dt=dt)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ionization_at_threshold_stays_finite(L, prec):
    wl = threshold_workload()
    col = L.Collider.from_workload(wl, precision=L.F32 if prec == "f32" else L.F64)
    col.load_workload(wl)
    n0 = col.count()
    for step in range(3):
        col.collide_neutral(wl["dt"], step)
    col.sync()
    assert col.count() > n0, "no ionization happened"
    vx, vy, vz, _, _ = col.read()
    assert np.isfinite(vx).all() and np.isfinite(vy).all() and np.isfinite(vz).all()
    mom, _ = col.moments()
    assert np.isfinite(mom).all()
