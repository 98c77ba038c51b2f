"""Seeded synthetic workloads shaped like the paper's collision benchmarks.

This module only draws inputs: particle velocities, cell ids and per-cell
parameters.  It holds none of the collision arithmetic and imports neither the
CUDA library nor the oracle, so both sides can take identical inputs from it.

Every workload is a dict with
  M                 number of cells (all instances together)
  vx, vy, vz        float64 velocities [m/s], cell-contiguous storage
  cell              int32 cell id per particle
  inv_vol           float64 [M]; cell density is n_j = weight * N_j * inv_vol[j]
  dt_cell           float64 [M]; time step of each cell [s]
  lnlam_cell        float64 [M]; Coulomb logarithm (constant mode)
  lnlam_mode        0 = constant per cell, 1 = NRL from the cell's moments
  weight, mass, charge, eps0                     species / constants (SI)
  n_neutral, mass_neutral, sigma_el, sigma_ion, e_ion   neutral background
  seed, capacity, steps, coulomb, neutral, precision     run settings

Velocities are generated per block of cells from numpy ``default_rng`` seeded
with (seed, block), so any subset of cells can be regenerated on its own.
"""
from __future__ import annotations

import math

import numpy as np

E_CHARGE = 1.602176634e-19       # C
M_E = 9.1093837015e-31           # kg
EPS0 = 8.8541878128e-12          # F/m
AMU = 1.66053906660e-27          # kg
M_AR = 39.948 * AMU

# Neutral argon background and analytic cross sections (LXCat tables are not
# available; constant elastic and step ionization cross sections stand in).
N_NEUTRAL = 3.22e22              # m^-3  (3.22e16 cm^-3, the paper's 0-D case)
SIGMA_EL = 1e-19                 # m^2
SIGMA_ION = 2e-20                # m^2 above threshold
E_ION = 15.76                    # eV

BLOCK = 64                       # cells per generator block


def nrl_nu_e(n_m3: float, T_eV: float, lnlam: float) -> float:
    """NRL-formulary electron collision rate 2.91e-6 n[cm^-3] lnL T^-3/2 [1/s] (time-step recipe)."""
    return 2.91e-6 * (n_m3 * 1e-6) * lnlam * T_eV ** -1.5


def _vth(T_eV: float) -> float:
    return math.sqrt(T_eV * E_CHARGE / M_E)


def _base(M: int, **kw) -> dict:
    d = dict(M=M, mass=M_E, charge=E_CHARGE, eps0=EPS0, weight=1.0,
             n_neutral=N_NEUTRAL, mass_neutral=M_AR, sigma_el=SIGMA_EL, sigma_ion=SIGMA_ION,
             e_ion=E_ION, seed=0, lnlam_mode=0, odd_mode=0, x=None)
    d.update(kw)
    return d


def _assemble(M, counts, gen_block, seed, blocks=None, dtype=np.float64):
    """Concatenate per-block velocity draws; `gen_block(rng, cells)` returns (vx, vy, vz)."""
    counts = np.asarray(counts, dtype=np.int64)
    nb = (M + BLOCK - 1) // BLOCK
    sel = range(nb) if blocks is None else blocks
    vxs, vys, vzs, cells = [], [], [], []
    for b in sel:
        cs = np.arange(b * BLOCK, min(M, (b + 1) * BLOCK))
        rng = np.random.default_rng([seed, b])
        vx, vy, vz = gen_block(rng, cs)
        vxs.append(vx.astype(dtype, copy=False)); vys.append(vy.astype(dtype, copy=False))
        vzs.append(vz.astype(dtype, copy=False))
        cells.append(np.repeat(cs.astype(np.int32), counts[cs]))
    return (np.concatenate(vxs), np.concatenate(vys), np.concatenate(vzs),
            np.concatenate(cells).astype(np.int32))


def relax_64x1000(M: int = 64, ppc: int = 1000, seed: int = 0, steps: int = 100) -> dict:
    """Plain FP64 e-e Coulomb: anisotropic Maxwellian T_par = 2 eV (z), T_perp = 1 eV, n = 1e18,
    lnL = 10, dt = 0.1 / nu_e at T = (T_par + 2 T_perp)/3.  Each cell's sample is centred and
    rescaled so that its temperatures are exactly T_par and T_perp."""
    T_par, T_perp, n = 2.0, 1.0, 1e18
    counts = np.full(M, ppc, np.int64)

    def gen(rng, cs):
        out = []
        for T in (T_perp, T_perp, T_par):
            v = rng.standard_normal((cs.size, ppc)) * _vth(T)
            v -= v.mean(axis=1, keepdims=True)
            v *= _vth(T) / np.sqrt((v * v).mean(axis=1, keepdims=True))
            out.append(v.reshape(-1))
        return out

    vx, vy, vz, cell = _assemble(M, counts, gen, seed)
    dt = 0.1 / nrl_nu_e(n, (T_par + 2 * T_perp) / 3.0, 10.0)
    return _base(M, vx=vx, vy=vy, vz=vz, cell=cell, inv_vol=np.full(M, n / ppc),
                 dt_cell=np.full(M, dt), lnlam_cell=np.full(M, 10.0), seed=seed,
                 capacity=int(vx.size), steps=steps, coulomb=True, neutral=False, precision="f64",
                 T_par=T_par, T_perp=T_perp, density=n, dt=dt)


def tail_4096x10000(M: int = 4096, ppc: int = 10000, hot: int | None = None, seed: int = 0, steps: int = 1000,
         blocks=None) -> dict:
    """FP32 Coulomb + e-n: 95 % at 2 eV and 5 % (exactly `hot` per cell) at 20 eV, isotropic, zero
    drift; n_e = 3.22e21 (ionization fraction 0.1 of n_n); lnL = 10; dt fixed so that the
    null-collision probability at step 0 is 0.02 for the largest speed of the initial state."""
    hot = ppc // 20 if hot is None else hot
    n_e = 3.22e21
    counts = np.full(M, ppc, np.int64)

    def gen(rng, cs):
        out = []
        for _ in range(3):
            v = rng.standard_normal((cs.size, ppc))
            v[:, : ppc - hot] *= _vth(2.0)
            v[:, ppc - hot:] *= _vth(20.0)
            out.append(v.reshape(-1))
        return out

    vx, vy, vz, cell = _assemble(M, counts, gen, seed, blocks)
    vmax = float(np.sqrt((vx * vx + vy * vy + vz * vz).max()))
    dt = -math.log1p(-0.02) / (N_NEUTRAL * (SIGMA_EL + SIGMA_ION) * vmax)
    return _base(M, vx=vx, vy=vy, vz=vz, cell=cell, inv_vol=np.full(M, n_e / ppc),
                 dt_cell=np.full(M, dt), lnlam_cell=np.full(M, 10.0), seed=seed,
                 capacity=2 * int(vx.size), steps=steps, coulomb=True, neutral=True, precision="f32",
                 density=n_e, dt=dt, vmax0=vmax)


def loguniform_counts(nx: int = 256, ny: int = 256, seed: int = 0) -> np.ndarray:
    """Per-cell counts floor(exp(U(ln 16, ln 65537))) on an nx x ny grid (cell id = ix + nx iy)."""
    rng = np.random.default_rng([seed, 999_999])
    return np.floor(np.exp(rng.uniform(math.log(16.0), math.log(65537.0), nx * ny))).astype(np.int64)


def loguniform_256x256(nx: int = 256, ny: int = 256, seed: int = 0, steps: int = 200, blocks=None,
         dtype=np.float64) -> dict:
    """Uneven-cell batch: log-uniform counts in [16, 65536], isotropic 2 eV Maxwellian, density
    proportional to the count (1e18 m^-3 at 1024 particles), NRL lnL per cell, dt = 0.1/max nu_e."""
    M = nx * ny
    counts = loguniform_counts(nx, ny, seed)
    T = 2.0

    def gen(rng, cs):
        n = int(counts[cs].sum())
        return [rng.standard_normal(n) * _vth(T) for _ in range(3)]

    vx, vy, vz, cell = _assemble(M, counts, gen, seed, blocks, dtype)
    inv = 1e18 / 1024.0
    n_max = inv * float(counts.max())
    ln_max = 23.5 - math.log(math.sqrt(n_max * 1e-6) * T ** -1.25) - math.sqrt(1e-5 + (math.log(T) - 2) ** 2 / 16)
    dt = 0.1 / nrl_nu_e(n_max, T, ln_max)
    return _base(M, vx=vx, vy=vy, vz=vz, cell=cell, inv_vol=np.full(M, inv), dt_cell=np.full(M, dt),
                 lnlam_cell=np.full(M, 10.0), lnlam_mode=1, seed=seed, capacity=int(counts.sum()),
                 steps=steps, coulomb=True, neutral=False, precision="f32", counts=counts, dt=dt,
                 nx=nx, ny=ny)


def instances_layout(n_inst: int = 64, seed: int = 0):
    """Instance sizes: cells U{64..4096}, particles per cell U{100..20000}, T U(0.5, 5) eV."""
    rng = np.random.default_rng([seed, 888_888])
    Mi = rng.integers(64, 4097, n_inst)
    ppc = rng.integers(100, 20001, n_inst)
    T = rng.uniform(0.5, 5.0, n_inst)
    return Mi, ppc, T


def instances_64(n_inst: int = 64, seed: int = 0, steps: int = 100, instances=None, dtype=np.float64,
         scale_ppc: float = 1.0) -> dict:
    """Batch of independent plasma instances (disjoint cell ranges): n = 1e18, lnL = 10,
    dt_i = 0.1 / nu_e(T_i).  `instances` selects a subset (cells renumbered densely)."""
    Mi, ppc, T = instances_layout(n_inst, seed)
    ppc = np.maximum(2, (ppc * scale_ppc).astype(np.int64))
    sel = list(range(n_inst)) if instances is None else list(instances)
    n = 1e18
    vxs, vys, vzs, cells, inv, dts, inst_of_cell = [], [], [], [], [], [], []
    base = 0
    for i in sel:
        rng = np.random.default_rng([seed, 10_000 + i])
        cnt = int(Mi[i] * ppc[i])
        vt = _vth(float(T[i]))
        vxs.append((rng.standard_normal(cnt) * vt).astype(dtype))
        vys.append((rng.standard_normal(cnt) * vt).astype(dtype))
        vzs.append((rng.standard_normal(cnt) * vt).astype(dtype))
        cells.append((base + np.repeat(np.arange(Mi[i]), ppc[i])).astype(np.int32))
        inv.append(np.full(Mi[i], n / ppc[i]))
        dts.append(np.full(Mi[i], 0.1 / nrl_nu_e(n, float(T[i]), 10.0)))
        inst_of_cell.append(np.full(Mi[i], i, np.int32))
        base += int(Mi[i])
    vx = np.concatenate(vxs); vy = np.concatenate(vys); vz = np.concatenate(vzs)
    M = base
    return _base(M, vx=vx, vy=vy, vz=vz, cell=np.concatenate(cells), inv_vol=np.concatenate(inv),
                 dt_cell=np.concatenate(dts), lnlam_cell=np.full(M, 10.0), seed=seed,
                 capacity=int(vx.size), steps=steps, coulomb=True, neutral=False, precision="f32",
                 instance_of_cell=np.concatenate(inst_of_cell), instances=sel,
                 Mi=Mi[sel], ppc=ppc[sel], T_inst=T[sel])


def ragged(M: int = 37, mean_ppc: int = 300, seed: int = 7, T_eV: float = 3.0, shuffled: bool = False,
           dt: float | None = None, with_empty: bool = True) -> dict:
    """Small test workload with ragged counts (odd, even, 0, 1, 2, 3 per cell) and optional
    shuffled storage (particles not cell-contiguous)."""
    rng = np.random.default_rng([seed, 4242])
    counts = rng.integers(0, 2 * mean_ppc, M)
    if with_empty and M >= 6:
        counts[:6] = [0, 1, 2, 3, 4, 5]
    n = int(counts.sum())
    vt = _vth(T_eV)
    vx = rng.standard_normal(n) * vt
    vy = rng.standard_normal(n) * vt
    vz = rng.standard_normal(n) * vt * 1.3
    cell = np.repeat(np.arange(M, dtype=np.int32), counts)
    if shuffled:
        p = rng.permutation(n)
        vx, vy, vz, cell = vx[p], vy[p], vz[p], cell[p]
    dens = 1e19
    dt = dt if dt is not None else 0.1 / nrl_nu_e(dens, T_eV, 10.0)
    return _base(M, vx=vx, vy=vy, vz=vz, cell=cell.astype(np.int32),
                 inv_vol=np.full(M, dens / max(1, mean_ppc)), dt_cell=np.full(M, dt),
                 lnlam_cell=np.full(M, 10.0), seed=seed, capacity=2 * max(n, 1), steps=10,
                 coulomb=True, neutral=True, precision="f64", counts=counts, dt=dt)


def subset_cells(wl: dict, cells) -> dict:
    """Restrict a workload to the given cells (renumbered 0..len-1, order kept)."""
    cells = np.asarray(cells, dtype=np.int64)
    remap = np.full(wl["M"], -1, np.int64)
    remap[cells] = np.arange(cells.size)
    keep = remap[wl["cell"]] >= 0
    out = dict(wl)
    out["ids"] = np.nonzero(keep)[0].astype(np.uint32)    # original indices: the random-stream ids
    base_ids = wl.get("cell_ids")
    out["cell_ids"] = (cells if base_ids is None else np.asarray(base_ids)[cells]).astype(np.uint32)
    out.update(M=int(cells.size), vx=wl["vx"][keep], vy=wl["vy"][keep], vz=wl["vz"][keep],
               cell=remap[wl["cell"][keep]].astype(np.int32), inv_vol=wl["inv_vol"][cells],
               dt_cell=wl["dt_cell"][cells], lnlam_cell=wl["lnlam_cell"][cells])
    out["capacity"] = max(int(keep.sum()) * 2, 1)
    if wl.get("x") is not None:
        out["x"] = wl["x"][keep]
    for key in ("instance_of_cell", "counts"):            # other per-cell arrays
        if wl.get(key) is not None:
            out[key] = np.asarray(wl[key])[cells]
    return out


# ----------------------------------------------------------------------------- cross-section tables
# Sec. 4.2 replaces the LXCat lookup with a piecewise polynomial of each cross
# section (error under 2 %).  The LXCat argon data are not available, so smooth
# argon-like stand-ins are tabulated instead: an elastic cross section with a
# low-energy minimum and a peak near 12 eV, and an ionization cross section of
# the ln(E/I)/(E/I) form above I = 15.76 eV peaking near 2.9e-20 m^2.  A table is
# a cubic per interval of a uniform grid in ln E (Hermite: values and slopes at
# the knots), the layout both the library and the oracle evaluate.

def sigma_el_argon_like(E):
    """Elastic stand-in [m^2] for E [eV]."""
    E = np.asarray(E, np.float64)
    return 1.2e-20 + 1.45e-19 * (E / 12.0) ** 2 / (1.0 + (E / 12.0) ** 2.6) + 4e-21 / (1.0 + E / 0.05)


def sigma_ion_argon_like(E):
    """Ionization stand-in [m^2] for E [eV]: 2.9e-20 e ln(E/I) / (E/I) above I = 15.76 eV."""
    E = np.asarray(E, np.float64)
    x = np.maximum(E / E_ION, 1.0)
    return np.where(E >= E_ION, 2.9e-20 * math.e * np.log(x) / x, 0.0)


def xsec_table(f, e_lo, e_hi, pieces, zero_below):
    """Piecewise cubic Hermite table of f on a uniform ln E grid [e_lo, e_hi]: a dict with
    lnE0, h, pieces, zero_below and coef [pieces, 4] (sigma = c0 + c1 t + c2 t^2 + c3 t^3,
    t = (ln E - lnE0)/h - i in interval i)."""
    lnE = np.linspace(math.log(e_lo), math.log(e_hi), pieces + 1)
    h = lnE[1] - lnE[0]
    E = np.exp(lnE)
    y = f(E)
    # slopes d sigma / d lnE by a centred difference of the function itself
    eps = 1e-5
    d = (f(E * math.exp(eps)) - f(E * math.exp(-eps))) / (2 * eps)
    if zero_below:
        d[0] = (f(E[0] * math.exp(eps)) - y[0]) / eps     # one-sided at the threshold
    coef = np.zeros((pieces, 4))
    for i in range(pieces):
        y0, y1, m0, m1 = y[i], y[i + 1], d[i] * h, d[i + 1] * h
        coef[i] = [y0, m0, 3 * (y1 - y0) - 2 * m0 - m1, 2 * (y0 - y1) + m0 + m1]
    return {"lnE0": float(lnE[0]), "h": float(h), "pieces": int(pieces), "zero_below": int(zero_below),
            "coef": coef}


def argon_like_tables(pieces_el=64, pieces_ion=48):
    """The elastic table on [0.01, 1000] eV, the ionization one on [I, 1000] eV, and a bound
    on sigma_el + sigma_ion over all energies (2 % over the largest of a dense sampling; the
    null-collision bound uses it)."""
    el = xsec_table(sigma_el_argon_like, 1e-2, 1e3, pieces_el, zero_below=False)
    ion = xsec_table(sigma_ion_argon_like, E_ION, 1e3, pieces_ion, zero_below=True)
    E = np.exp(np.linspace(math.log(1e-3), math.log(1e4), 200001))
    smax = 1.02 * float(np.max(sigma_el_argon_like(E) + sigma_ion_argon_like(E)))
    return el, ion, smax
