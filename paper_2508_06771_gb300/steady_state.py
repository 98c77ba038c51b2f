"""0-D steady state of electrons in a constant field (Sec. 6, the EEDF with and without Coulomb).

The paper's test problem keeps only the collision (DSMC) part of the solver:
a constant electric field E heats the electrons, elastic and ionization
collisions with a fixed neutral background cool them, Coulomb collisions
among the electrons act at the electron density n_e, and all densities are
held fixed while the run steps to a state whose observables (electron
temperature, rate coefficients, mobility) no longer change.

Here every cell is one independent 0-D replica: cell j spans [j dx, (j+1) dx)
with dx so wide that no electron leaves its cell during a run, so the push of
S2b/S2c only accelerates (v_z += dt a, a = -e E / m).  The electron density
that the Coulomb step sees is n_e = w N_j / V_j; n_e / n_n = 0 is taken as a
vanishing density (1e-9 n_n: the Coulomb frequency scales with n_e).  Fixed
densities with ionization: every `resample_every` steps each cell is brought
back to its initial count by keeping a uniformly random subset of its
particles (independent of velocity, so the distribution is unchanged in
expectation); between resamplings N_j grows by the ionization count.

Observables, per cell then averaged: T_e = (2/3) <eps>, the rate coefficients
k_el = sum sigma_el |v| / N and k_ion = sum sigma_ion |v| / N, the drift
velocity <v_z> and the reduced mobility mu n_n = |<v_z>| n_n / E.

Closed forms for the checks (two-term theory, constant elastic cross section,
cold neutrals, isotropic scattering, no ionization): with lambda = 1 / (n_n
sigma_el), the Druyvesteyn distribution f(eps) ~ sqrt(eps) exp(-(eps/eps0)^2),
eps0 = e E lambda sqrt(M / 3m), has <eps> = eps0 Gamma(5/4) / Gamma(3/4) and
<eps^2> / <eps>^2 = Gamma(7/4) Gamma(3/4) / Gamma(5/4)^2 = 1.3708.  When
electron-electron collisions are much more frequent than electron-neutral
ones, f is a Maxwellian drifting with velocity W: the field force m a balances
the momentum loss (m^2 W / 3kT) <nu v^2>, so W = 3 a lambda / (4 <v>), and the
heating m a W balances the elastic loss (m^2 / (M lambda)) <v^3>, which gives
k T = e E lambda sqrt(3 pi M / (128 m)) and <eps^2> / <eps>^2 = 5/3.  (With the
anisotropy set by electron-neutral collisions alone, the Lorentz limit, the
same balance gives k T = e E lambda sqrt(M / 12 m), 6 % higher.)
"""
from __future__ import annotations

import math

import numpy as np

from . import ltpc
from . import workloads as W

DX_0D = 1.0e4          # m: cell width of a replica (no electron crosses it in a run)


def druyvesteyn_mean(E_field: float, n_neutral: float, sigma_el: float, mass_ratio: float) -> float:
    """<eps> [eV] of the Druyvesteyn distribution (constant sigma_el, M/m = mass_ratio)."""
    lam = 1.0 / (n_neutral * sigma_el)
    eps0 = E_field * lam * math.sqrt(mass_ratio / 3.0)          # eV: e E lambda / e
    return eps0 * math.gamma(1.25) / math.gamma(0.75)


def drifting_maxwellian_mean(E_field: float, n_neutral: float, sigma_el: float, mass_ratio: float) -> float:
    """<eps> = 3/2 k T [eV] of the drifting Maxwellian whose heating balances the elastic loss
    (electron-electron collisions dominant)."""
    lam = 1.0 / (n_neutral * sigma_el)
    return 1.5 * E_field * lam * math.sqrt(3.0 * math.pi * mass_ratio / 128.0)


def lorentz_maxwellian_mean(E_field: float, n_neutral: float, sigma_el: float, mass_ratio: float) -> float:
    """<eps> [eV] of a Maxwellian whose anisotropy is set by electron-neutral collisions alone."""
    lam = 1.0 / (n_neutral * sigma_el)
    return 1.5 * E_field * lam * math.sqrt(mass_ratio / 12.0)


DRUYVESTEYN_RATIO = math.gamma(1.75) * math.gamma(0.75) / math.gamma(1.25) ** 2
MAXWELL_RATIO = 5.0 / 3.0


def zero_d(M: int = 64, ppc: int = 2000, *, E_field: float, ion_frac: float = 0.0,
           n_neutral: float = W.N_NEUTRAL, mass_neutral: float = W.M_AR, T0_eV: float = 1.0,
           sigma_el: float = W.SIGMA_EL, sigma_ion: float = 0.0, e_ion: float = 1e30, xs=None,
           dt: float = 1e-11, seed: int = 0, capacity_factor: float = 1.5) -> dict:
    """A workload of M independent 0-D replicas of ppc electrons (Maxwellian at T0_eV).

    E_field [V/m] along z; ion_frac = n_e / n_n; xs = (elastic table, ionization table,
    sigma_max) for tabulated cross sections (the constants are used otherwise)."""
    rng = np.random.default_rng([seed, 606])
    n = M * ppc
    vt = math.sqrt(T0_eV * W.E_CHARGE / W.M_E)
    cell = np.repeat(np.arange(M, dtype=np.int32), ppc)
    n_e = ion_frac * n_neutral if ion_frac > 0 else 1e-9 * n_neutral
    wl = W._base(M, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt,
                 vz=rng.standard_normal(n) * vt, cell=cell, x=(cell + 0.5) * DX_0D,
                 inv_vol=np.full(M, n_e / ppc), dt_cell=np.full(M, dt), lnlam_cell=np.full(M, 10.0),
                 seed=seed, capacity=int(capacity_factor * n), n_neutral=n_neutral, mass_neutral=mass_neutral,
                 sigma_el=sigma_el, sigma_ion=sigma_ion, e_ion=e_ion, lnlam_mode=ltpc.LNL_NRL, dt=dt)
    wl["accel"] = np.full(M, -W.E_CHARGE * E_field / W.M_E)
    wl["E_field"] = float(E_field)
    wl["ion_frac"] = float(ion_frac)
    wl["ppc"] = int(ppc)
    if xs is not None:
        wl["xs"] = xs
    return wl


HALF_M_OVER_E = 0.5 * W.M_E / W.E_CHARGE


def observables(mom: np.ndarray, E_field: float, n_neutral: float) -> dict:
    """The paper's observables of one moments snapshot, over all replicas."""
    N = float(mom[:, 0].sum())
    if N <= 0:
        return dict(N=0.0)
    eps = HALF_M_OVER_E * float(mom[:, 5:8].sum()) / N
    vz = float(mom[:, 4].sum()) / N
    return dict(N=N, mean_eps=eps, T_e=2.0 * eps / 3.0, k_el=float(mom[:, 8].sum()) / N,
                k_ion=float(mom[:, 9].sum()) / N, drift=vz, mu_n=abs(vz) * n_neutral / E_field)


def _resample(col, ppc: int, rng) -> int:
    """Bring every cell back to ppc particles by a uniformly random subset (fixed density)."""
    vx, vy, vz, cell, x = col.read()
    keep = []
    order = np.argsort(cell, kind="stable")
    bounds = np.searchsorted(cell[order], np.arange(col.M + 1))
    for j in range(col.M):
        idx = order[bounds[j]:bounds[j + 1]]
        if idx.size > ppc:
            idx = rng.choice(idx, ppc, replace=False)
        keep.append(np.sort(idx))
    keep = np.concatenate(keep)
    col.load(vx[keep], vy[keep], vz[keep], cell[keep], x[keep])
    return int(cell.size - keep.size)


def run(wl: dict, steps: int, *, precision: int = ltpc.F32, sample_every: int = 500, average_last: float = 0.4,
        resample_every: int = 0, seed: int = 1, autotune: bool = True) -> dict:
    """Step a zero_d workload `steps` times through the library (ltpc_run: Coulomb, e-n
    collisions, push, moments every step) and average the observables over the last
    `average_last` fraction of the samples.  Also the shape of the EEDF from the particles
    read back at each sample of that window: <eps^2> / <eps>^2 (Druyvesteyn 1.3708,
    Maxwellian 5/3) and the summed energy histogram."""
    import time

    col = ltpc.Collider.from_workload(wl, precision=precision)
    col.set_field(DX_0D, wl["accel"], ltpc.WALL_PERIODIC)
    col.load_workload(wl)
    dt = float(wl["dt"])
    if autotune:
        col.autotune(dt)
    rng = np.random.default_rng([seed, 707])
    series, shape, vmax2, hist_sum, removed = [], [], [], None, 0
    s = 0
    n_samples = (steps + sample_every - 1) // sample_every
    first_avg = int(math.floor((1.0 - average_last) * n_samples))
    t0 = time.perf_counter()
    for k in range(n_samples):
        n = min(sample_every, steps - s)
        col.run(dt, s, n)
        s += n
        mom, hist = col.moments()
        col.sync()
        series.append(dict(step=s, **observables(mom, wl["E_field"], wl["n_neutral"])))
        if k >= first_avg:
            vx, vy, vz, cell, _ = col.read()
            v2 = vx.astype(np.float64) ** 2 + vy.astype(np.float64) ** 2 + vz.astype(np.float64) ** 2
            e = HALF_M_OVER_E * v2
            shape.append((float(np.mean(e)), float(np.mean(e * e))))
            vm = np.zeros(col.M)
            np.maximum.at(vm, cell[cell >= 0], v2[cell >= 0])
            vmax2.append(vm)
            h = hist.sum(0).astype(np.float64)
            hist_sum = h if hist_sum is None else hist_sum + h
        if resample_every and s % resample_every == 0 and s < steps:
            removed += _resample(col, wl["ppc"], rng)
    wall = time.perf_counter() - t0
    win = series[first_avg:]
    out = {key: float(np.mean([d[key] for d in win])) for key in ("mean_eps", "T_e", "k_el", "k_ion", "drift", "mu_n")}
    out["eps_std_err"] = float(np.std([d["mean_eps"] for d in win]) / math.sqrt(max(1, len(win) - 1)))
    m1 = np.mean([a for a, _ in shape])
    m2 = np.mean([b for _, b in shape])
    out.update(ratio=float(m2 / (m1 * m1)), vmax2_cell=np.mean(vmax2, axis=0), steps=steps, dt=dt, wall_s=wall, removed_by_resampling=removed,
               series=series, hist=hist_sum / max(1, len(shape)), particles=int(series[-1]["N"]))
    col.close()
    return out
