"""Pins of the oracle's tabulated cross sections and per-particle collision selection (Sec. 4.2).

* The piecewise-cubic tables stay within 2 % of the smooth cross sections they
  stand for (the paper's bound for its polynomial fits) over 0.01-1000 eV, hit
  the knot values exactly, vanish below the ionization threshold and hold the
  last value above the table.
* Per-particle selection: elastic and ionization counts over many particles
  equal the sums of pi_el and min(1, pi_el + pi_ion) - pi_el, pi_c = 1 -
  exp(-dt v sigma_c n_n) (binomial, within 4 sigma) -- the analytic collision
  frequency of each particle.
* Null-collision and per-particle selection give the same mean number of real
  collisions to first order in dt (within 4 sigma), the comparison the paper
  makes between the two methods.
* The moments' rate sums use the tables: sum sigma_el v / N of a Maxwellian
  sample matches <sigma_el v> integrated over the Maxwellian.
"""
import math

import numpy as np
from scipy import integrate

from paper_2508_06771_gb300 import workloads as W


def test_tables_within_two_percent(orc):
    el, ion, smax = W.argon_like_tables()
    E = np.exp(np.linspace(math.log(0.011), math.log(990.0), 3001))
    g_el = np.array([orc.xs_eval(el, e) for e in E])
    assert np.max(np.abs(g_el / W.sigma_el_argon_like(E) - 1)) < 0.02
    Ei = E[E > W.E_ION * 1.0001]
    g_ion = np.array([orc.xs_eval(ion, e) for e in Ei])
    assert np.max(np.abs(g_ion / W.sigma_ion_argon_like(Ei) - 1)) < 0.02
    knots = np.exp(el["lnE0"] + el["h"] * np.arange(el["pieces"]))
    assert np.allclose([orc.xs_eval(el, e) for e in knots], el["coef"][:, 0], rtol=1e-12, atol=0)
    assert orc.xs_eval(ion, W.E_ION * 0.999) == 0.0 and orc.xs_eval(ion, 0.5) == 0.0
    last = el["coef"][-1].sum()
    assert math.isclose(orc.xs_eval(el, 5e3), last, rel_tol=1e-12)
    assert smax >= np.max(g_el[:, None].ravel()) and smax > 1e-19


def _hot_wl(n_cells, ppc, T, seed, dt, selection, xs=True):
    rng = np.random.default_rng(seed)
    n = n_cells * ppc
    vt = math.sqrt(T * W.E_CHARGE / W.M_E)
    wl = W._base(n_cells, vx=rng.standard_normal(n) * vt, vy=rng.standard_normal(n) * vt,
                 vz=rng.standard_normal(n) * vt, cell=np.repeat(np.arange(n_cells, dtype=np.int32), ppc),
                 inv_vol=np.full(n_cells, 1e17), dt_cell=np.full(n_cells, dt), lnlam_cell=np.full(n_cells, 10.0),
                 seed=seed, capacity=3 * n, selection=selection)
    if xs:
        wl["xs"] = W.argon_like_tables()
    return wl


def test_per_particle_counts_match_probabilities(orc):
    wl = _hot_wl(8, 4000, 15.0, 3, 3e-11, selection=1)
    el, ion, _ = wl["xs"]
    P = orc.make_params(wl)
    tot_el = tot_ion = exp_el = exp_ion = var_el = var_ion = 0.0
    for s in range(6):
        st = orc.State(wl)
        vx, vy, vz, _ = st.views()
        v2 = vx * vx + vy * vy + vz * vz
        v = np.sqrt(v2)
        E = 0.5 * W.M_E * v2 / W.E_CHARGE
        sel = W.sigma_el_argon_like(E)
        sio = W.sigma_ion_argon_like(E)
        p_el = -np.expm1(-wl["dt_cell"][0] * v * sel * wl["n_neutral"])
        p_io = -np.expm1(-wl["dt_cell"][0] * v * sio * wl["n_neutral"])
        p_io = np.minimum(1.0, p_el + p_io) - p_el      # one uniform against pi_el, pi_el + pi_ion
        info = orc.neutral(st, P, s)
        tot_el += info["elastic"]; tot_ion += info["ionization"]
        exp_el += p_el.sum(); exp_ion += p_io.sum()
        var_el += (p_el * (1 - p_el)).sum(); var_ion += (p_io * (1 - p_io)).sum()
    # the table differs from the smooth stand-in by < 1e-4, far inside 4 sigma
    assert abs(tot_el - exp_el) < 4 * math.sqrt(var_el) + 1e-3 * exp_el, (tot_el, exp_el)
    assert abs(tot_ion - exp_ion) < 4 * math.sqrt(var_ion) + 1e-3 * exp_ion, (tot_ion, exp_ion)
    assert tot_ion > 100 and tot_el > 1000


def test_null_and_per_particle_agree_in_expectation(orc):
    res = {}
    for selection in (0, 1):
        wl = _hot_wl(8, 4000, 12.0, 5, 1e-13, selection=selection)     # nu dt ~ 1e-3: first order
        P = orc.make_params(wl)
        hits = 0
        for s in range(40):
            st = orc.State(wl)
            info = orc.neutral(st, P, s)
            hits += info["elastic"] + info["ionization"]
        res[selection] = hits
    a, b = res[0], res[1]
    assert a > 400 and abs(a - b) < 4 * math.sqrt(a + b) + 0.005 * (a + b), res


def test_rate_sums_use_the_tables(orc):
    T = 5.0
    wl = _hot_wl(4, 50000, T, 9, 1e-12, selection=0)
    P = orc.make_params(wl)
    st = orc.State(wl)
    mom, _ = orc.moments(st, P)
    k_el = mom[:, 8].sum() / mom[:, 0].sum()
    kT = T * W.E_CHARGE

    def f(E):                                           # Maxwellian energy density times sigma v
        v = math.sqrt(2 * E * W.E_CHARGE / W.M_E)
        return 2 * math.sqrt(E * W.E_CHARGE / math.pi) * (kT) ** -1.5 * math.exp(-E * W.E_CHARGE / kT) * \
            W.E_CHARGE * float(W.sigma_el_argon_like(E)) * v
    ref, _ = integrate.quad(f, 0, 60 * T, limit=400, points=[0.05, 1, 12])
    assert abs(k_el / ref - 1) < 0.01, (k_el, ref)
