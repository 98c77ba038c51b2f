"""Benchmark of the collision step on GB300: particle-updates/s and HBM roofline.

Default workload (N=1): 4096 cells x 10000 electrons, FP32 velocities,
Takizuka-Abe Coulomb + null-collision electron-neutral step + moments, fused
per cell, replayed as a CUDA graph.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload tail_4096x10000|relax_64x1000|loguniform_256x256|instances_64]

With N > 1 (torchrun), every rank runs an independent replica of the workload
(its own seed): the method shards by cell and instance with no exchange, so
there is no data-path collective (weak scaling).  `--impl reference` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "collision particle-updates/s (FP32 batched vs FP64 plain) and % of HBM roofline"
W_E_OVER_M = 1.602176634e-19 / 9.1093837015e-31     # electron charge-to-mass ratio (field leg)
UNIT = "particle-updates/s"


# ----------------------------------------------------------------------------- helpers
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    return 6800.0, "fallback (6.8 TB/s)"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2508_06771_gb300", "csrc", "*"))):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload):
    """Per-launch DRAM bytes of the cell kernel from the committed ncu summary, if it was
    taken on the current kernel sources; else None."""
    f = os.path.join(ROOT, "profiles", f"cells_{workload}_ncu.md")
    if not os.path.exists(f):
        return None
    vals = {}
    for line in open(f):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while a region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0, period_ms=50):
        self.gpu, self.period = gpu_index, period_ms
        self.proc = None

    def __enter__(self):
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", f"-lms={self.period}"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.out.close()

    def summary(self):
        rows = []
        try:
            for line in open(self.out.name):
                f = [t.strip() for t in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        finally:
            os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload(name, seed, rank=0, cells=None):
    from paper_2508_06771_gb300 import workloads as W
    if name == "tail_4096x10000":
        wl = W.tail_4096x10000(seed=seed, M=cells or 4096)
        desc = f"tail_4096x10000: 1D grid of {wl['M']} cells x 10000 electrons (N0={wl['vx'].size:,}), FP32 SoA velocities, " \
               "95% at 2 eV + 500/cell at 20 eV, Takizuka-Abe Coulomb + null-collision e-n (elastic, " \
               "ionization >15.76 eV), fused per-cell moments"
    elif name == "relax_64x1000":
        wl = W.relax_64x1000(seed=seed)
        desc = "relax_64x1000: 64 cells x 1000 electrons, FP64, anisotropic Maxwellian, Coulomb only"
    elif name == "loguniform_256x256":
        if cells:       # profiling cases: the first `cells` cells (whole 64-cell blocks) only
            wl = W.loguniform_256x256(seed=seed, dtype=np.float32, blocks=list(range((cells + W.BLOCK - 1) // W.BLOCK)))
            wl["capacity"] = max(1, wl["vx"].size)
            sub = f" (cells 0..{min(cells, wl['M']) - 1} populated only)"
        else:
            wl = W.loguniform_256x256(seed=seed, dtype=np.float32)
            sub = ""
        desc = f"loguniform_256x256: 256x256 cells, log-uniform 16..65536 per cell{sub} (N0={wl['vx'].size:,}), FP32, NRL lnL, Coulomb"
    elif name == "instances_64":
        wl = W.instances_64(seed=seed, dtype=np.float32)
        desc = f"instances_64: 64 instances, {wl['M']} cells, N0={wl['vx'].size:,}, FP32, per-instance dt, Coulomb"
    else:
        raise SystemExit(f"unknown workload {name}")
    return wl, desc


def algorithmic_bytes_per_particle(prec):
    """Cell kernel: read the id list (4 B), gather the velocities, write them back."""
    es = 4 if prec == "f32" else 8
    return 4 + 6 * es


# ----------------------------------------------------------------------------- reference arm
def oracle_sample(workload, cells=16, pairing_mode=0):
    """A few of the workload's cells, generated on their own (the oracle's inputs), and
    whether the workload has the electron-neutral step."""
    from paper_2508_06771_gb300 import workloads as W
    blocks = list(range(max(1, (cells + W.BLOCK - 1) // W.BLOCK)))
    if workload == "tail_4096x10000":
        full = W.tail_4096x10000(seed=0, blocks=blocks)
    elif workload == "relax_64x1000":
        full = W.relax_64x1000(seed=0)
    elif workload == "loguniform_256x256":
        full = W.loguniform_256x256(seed=0, blocks=blocks)
    else:
        full = W.instances_64(seed=0, instances=[0])
    wl = W.subset_cells(full, np.arange(min(cells, full["M"])))
    wl["capacity"] = 2 * wl["vx"].size
    wl["pairing_mode"] = pairing_mode
    return wl, bool(full.get("neutral", False))


def _oracle_run(wl, neutral, warmup, steps, budget_s):
    """The oracle as it stands on `wl` -- `steps` steps after `warmup`, or as many as fit
    in `budget_s`.  Returns (particle-updates, seconds, steps)."""
    import oracle as orc
    st = orc.State(wl, capacity=wl["capacity"])
    P = orc.make_params(wl, correction=True)
    for k in range(warmup):
        orc.step(st, P, k, True, neutral)
    upd, done = 0, 0
    t0 = time.perf_counter()
    while (done < steps) if steps else (time.perf_counter() - t0 < budget_s):
        upd += st.n
        orc.step(st, P, warmup + done, True, neutral)
        done += 1
    return upd, time.perf_counter() - t0, done


def oracle_rate(wl, neutral, warmup=0, steps=0, budget_s=8.0, processes=1):
    """Particle-updates/s of the oracle on `wl`: in this process, or in `processes` worker
    processes (this script with --oracle-worker; they load only numpy and the oracle), summed
    over processes and divided by the slowest one's time."""
    if processes <= 1:
        res = [_oracle_run(wl, neutral, warmup, steps, budget_s)]
    else:
        import pickle
        with tempfile.TemporaryDirectory() as td:
            f = os.path.join(td, "sample.pkl")
            with open(f, "wb") as fh:
                pickle.dump({"wl": wl, "neutral": neutral, "warmup": warmup, "steps": steps,
                             "budget_s": budget_s}, fh)
            procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker", f],
                                      stdout=subprocess.PIPE, text=True) for _ in range(processes)]
            res = []
            for pr in procs:
                out, _ = pr.communicate()
                if pr.returncode != 0:
                    raise RuntimeError(f"oracle worker failed ({pr.returncode})")
                r = json.loads(out.strip().splitlines()[-1])
                res.append((r["upd"], r["seconds"], r["steps"]))
    upd = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return upd / el, el, min(r[2] for r in res)


def oracle_worker(path):
    import pickle
    with open(path, "rb") as fh:
        job = pickle.load(fh)
    upd, el, done = _oracle_run(job["wl"], job["neutral"], job["warmup"], job["steps"], job["budget_s"])
    print(json.dumps({"upd": upd, "seconds": el, "steps": done}), flush=True)


def reduce_over_ranks(elapsed, units, world, device="cpu"):
    """Whole-job timing of a weak-scaling run: the slowest rank's time and the units all
    ranks processed (every rank runs its own replica; the timed region ends in a barrier)."""
    if world <= 1:
        return float(elapsed), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    cores = host_cores()
    # size the sample so that every process's warm-up + timed steps take ~2 minutes in all
    pm = 1 if args.pairing == "bijection" else 0
    wl1, neutral = oracle_sample(args.workload, cells=16, pairing_mode=pm)
    v1, _, _ = oracle_rate(wl1, neutral, steps=1)
    per_particle = 1.0 / v1
    nsteps = args.steps + args.warmup
    target = 120.0 / nsteps / per_particle
    ppc = wl1["vx"].size / wl1["M"]
    cells = int(max(1, min(512, target // ppc)))   # at most ~5M particles per process
    wl, neutral = oracle_sample(args.workload, cells=cells, pairing_mode=pm)
    v, el, _ = oracle_rate(wl, neutral, warmup=args.warmup, steps=args.steps, processes=cores)
    sample = (f"{wl['M']} of the workload's cells ({wl['vx'].size:,} particles) per process, {args.steps} steps "
              f"after {args.warmup} warm-up, FP64 oracle, {cores} processes (one per host core)")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": make_workload_desc(args.workload)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_workload_desc(name):
    return {"tail_4096x10000": "tail_4096x10000: 4096 cells x 10000 electrons, FP32 Coulomb + e-n null collision",
            "relax_64x1000": "relax_64x1000: 64 cells x 1000 electrons, FP64 Coulomb",
            "loguniform_256x256": "loguniform_256x256: 256x256 log-uniform cells, FP32 Coulomb",
            "instances_64": "instances_64: 64 instances, FP32 Coulomb"}[name]


def sample_cells(wl, k=40, seed=1):
    """Cells the accuracy probe compares: the 4 smallest, the 4 largest, k random ones, and
    for a batch of instances two cells of every instance."""
    counts = np.bincount(wl["cell"], minlength=wl["M"])
    order = np.argsort(counts, kind="stable")
    rng = np.random.default_rng(seed)
    pick = set(order[:4].tolist()) | set(order[-4:].tolist())
    pick |= set(rng.choice(wl["M"], size=min(k, wl["M"]), replace=False).tolist())
    inst = wl.get("instance_of_cell")
    if inst is not None:
        for i in np.unique(inst):
            cs = np.nonzero(inst == i)[0]
            pick |= set(rng.choice(cs, size=min(2, cs.size), replace=False).tolist())
    return np.array(sorted(c for c in pick if counts[c] > 0))


def moment_errors(mom, omom):
    """Per-cell errors: N exact, sums of v over N v_rms, sums of v^2 and of sigma v relative."""
    N = np.maximum(omom[:, 0], 1)
    vth = np.sqrt(omom[:, 5:8].sum(1) / N)
    e = np.zeros_like(omom)
    e[:, 0] = np.abs(mom[:, 0] - omom[:, 0])
    e[:, 2:5] = np.abs(mom[:, 2:5] - omom[:, 2:5]) / (N * vth)[:, None]
    for k in (5, 6, 7, 8, 9):
        e[:, k] = np.abs(mom[:, k] - omom[:, k]) / np.maximum(np.abs(omom[:, k]), 1e-300)
    z = omom[:, 9] == 0
    e[z, 9] = (np.abs(mom[z, 9]) > 0).astype(float)
    return e


def accuracy_vs_oracle(probe):
    """The GPU's first step against the FP64 oracle on the probe's sampled cells, from the same
    (binary32-rounded, in FP32) inputs, with the particles' original ids.  Errors per result;
    cells where a null-collision decision sits within the oracle's margin are counted apart.
    Runs in the CPU-baseline leg: the only place the benchmark executes the oracle."""
    import oracle as orc
    from paper_2508_06771_gb300 import workloads as W
    wl, cells, gmom, step = probe["wl"], probe["cells"], probe["mom"], probe["step"]
    f32 = probe["prec"] == "f32"
    sub = W.subset_cells(wl, cells)
    if f32:
        for k in ("vx", "vy", "vz"):
            sub[k] = np.asarray(sub[k], np.float32).astype(np.float64)
    P = orc.make_params(sub, correction=f32, pairing_mode=probe["pairing_mode"])
    st = orc.State(sub)
    lnlam = None
    if sub.get("lnlam_mode", 0) == 1:
        m0, _ = orc.moments(st, P)
        lnlam = orc.lnlambda_from_moments(m0, sub["inv_vol"], sub["weight"], sub["mass"], sub["charge"])
    orc.coulomb(st, P, step, lnlam)
    near = np.zeros(sub["M"], bool)
    margin = 1e-5 if probe["pairing_mode"] == 1 else 1e-6
    if probe["neutral"]:
        pr = orc.State(sub)
        pr.vx[:], pr.vy[:], pr.vz[:] = st.vx, st.vy, st.vz
        dec = orc.neutral(pr, P, step, with_decisions=True)
        near[st.cell[:st.n][dec["margin"] < margin]] = True
        orc.neutral(st, P, step)
    omom, _ = orc.moments(st, P)
    e = moment_errors(gmom, omom)
    ok = ~near
    names = {2: "sum_v", 5: "sum_v2", 8: "sum_sigma_el_v", 9: "sum_sigma_ion_v"}
    out = {"against": "FP64 oracle, same inputs and ids, one fused step",
           "cells_compared": int(ok.sum()), "cells_with_decision_in_margin": int(near.sum()),
           "bar": 1e-5 if f32 else 1e-12, "count_exact": bool(e[ok, 0].max() == 0 if ok.any() else True),
           "max_rel_err": float(e[ok][:, 2:10].max()) if ok.any() else None,
           "per_result_max_rel_err": {nm: float(e[ok][:, k:k + (3 if k in (2, 5) else 1)].max())
                                      for k, nm in names.items()} if ok.any() else {}}
    inst = sub.get("instance_of_cell")
    if inst is not None:
        # per-instance conservation: momentum over N m v_rms, energy relative, worst sampled cell
        dP, dE = {}, {}
        m = sub["mass"]
        for i in np.unique(inst):
            sel = (inst == i) & ok
            if not sel.any():
                continue
            N = np.maximum(omom[sel, 0], 1)
            vrms = np.sqrt(omom[sel, 5:8].sum(1) / N)
            dp = np.linalg.norm(m * (gmom[sel, 2:5] - omom[sel, 2:5]), axis=1) / (N * m * vrms)
            de = np.abs(gmom[sel, 5:8].sum(1) - omom[sel, 5:8].sum(1)) / omom[sel, 5:8].sum(1)
            dP[int(i)], dE[int(i)] = float(dp.max()), float(de.max())
        out["per_instance"] = {"instances": len(dP), "dP_over_NmV_max": max(dP.values()),
                               "dP_over_NmV_median": float(np.median(list(dP.values()))),
                               "dE_over_E_max": max(dE.values()),
                               "dE_over_E_median": float(np.median(list(dE.values())))}
    return out


def relaxation_check(ltpc, steps=100):
    """relax_64x1000 on the GPU (FP64, the bench's context settings): T_par(t), T_perp(t) from
    the moments of every step against the NRL isotropization ODE.  Takizuka-Abe at this step
    (0.1 of the e-e collision time) relaxes at about 0.74 of the NRL rate (the deficit scales
    like dt^(1/3)); reported are the fitted rate ratio and the largest temperature deviation."""
    from scipy import integrate
    from paper_2508_06771_gb300 import workloads as W
    wl = W.relax_64x1000()
    col = ltpc.Collider.from_workload(wl, precision=ltpc.F64)
    col.load_workload(wl)
    Tpar, Tperp = [], []

    def temps():
        mom, _ = col.moments()
        N = mom[:, 0].sum()
        mean = mom[:, 2:5].sum(0) / N
        sq = mom[:, 5:8].sum(0) / N
        T = W.M_E * (sq - mean * mean) / W.E_CHARGE
        Tpar.append(T[2]); Tperp.append(0.5 * (T[0] + T[1]))

    temps()
    for k in range(steps):
        col.collide_coulomb(wl["dt"], k)
        temps()
    col.sync()
    col.close()
    t = np.arange(steps + 1) * wl["dt"]
    e2 = W.E_CHARGE ** 2 / (4 * math.pi * W.EPS0)

    def nu_T(tpar, tperp):
        A = tperp / tpar - 1.0
        pref = 2 * math.sqrt(math.pi) * e2 ** 2 * wl["density"] * 10.0 / (math.sqrt(W.M_E) * (tpar * W.E_CHARGE) ** 1.5)
        if abs(A) < 1e-3:
            f = 4.0 / 15.0 - 8.0 * A / 35.0 + 4.0 * A * A / 21.0
        elif A < 0:
            r = math.sqrt(-A); f = (-3 + (A + 3) * math.atanh(r) / r) / A ** 2
        else:
            r = math.sqrt(A); f = (-3 + (A + 3) * math.atan(r) / r) / A ** 2
        return pref * f

    sol = integrate.solve_ivp(lambda _, y: [2 * nu_T(*y) * (y[1] - y[0]), -nu_T(*y) * (y[1] - y[0])],
                              (0, t[-1]), [wl["T_par"], wl["T_perp"]], t_eval=t, rtol=1e-10, atol=1e-14,
                              method="DOP853", max_step=t[1] - t[0])
    rp, rq = sol.y
    dT = np.array(Tpar) - np.array(Tperp)
    # e-folding rates fitted over the first 53 ns (ten steps), the window of the oracle's pin
    # (later the NRL curve reaches its floor and the sample's difference the sampling noise)
    win = t <= 53e-9 * (1 + 1e-9)
    k = -np.polyfit(t[win], np.log(dT[win]), 1)[0]
    kr = -np.polyfit(t[win], np.log((rp - rq)[win]), 1)[0]
    Tm = (np.array(Tpar) + 2 * np.array(Tperp)) / 3
    return {"workload": "relax_64x1000, FP64, 100 Coulomb steps", "rate_ratio_to_nrl": float(k / kr),
            "expected_ratio_at_this_dt": "about 0.74 over the first 53 ns (deficit ~ dt^(1/3); the oracle's pin "
                                         "extrapolates to 1)",
            "max_dev_T_par_over_T": float(np.max(np.abs(np.array(Tpar) - rp) / Tm)),
            "max_dev_T_perp_over_T": float(np.max(np.abs(np.array(Tperp) - rq) / Tm)),
            "mean_temperature_drift": float(abs(Tm[-1] - Tm[0]) / Tm[0])}


def cpu_baseline(workload, budget_s=8.0, pairing_mode=0, probe=None):
    """The oracle as it stands on a bounded sample of the workload (rank 0, N=1), on one core
    and on every host core (one process per core); and the GPU's accuracy probe against it."""
    import oracle as orc
    orc.build()
    accuracy = accuracy_vs_oracle(probe) if probe is not None else None
    wl, neutral = oracle_sample(workload, cells=16, pairing_mode=pairing_mode)
    v1, el1, s1 = oracle_rate(wl, neutral, budget_s=budget_s)
    cores = host_cores()
    vn, eln, sn = oracle_rate(wl, neutral, budget_s=budget_s, processes=cores) if cores > 1 else (v1, el1, s1)
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle", "single_core": v1,
            "sample": f"{wl['M']} cells ({wl['vx'].size:,} particles) of the workload per process, full steps "
                      f"(Coulomb{' + e-n' if neutral else ''} + moments), FP64; {cores} processes x {sn} steps "
                      f"in {eln:.1f} s, and 1 process x {s1} steps in {el1:.1f} s"}, accuracy


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2508_06771_gb300 import build as B
    from paper_2508_06771_gb300 import ltpc

    torch.cuda.set_device(local_rank)
    B.build()
    wl, desc = make_workload(args.workload, seed=rank, cells=args.cells)
    prec = "f32" if wl["precision"] == "f32" else "f64"
    pmode = ltpc.PAIR_BIJECTION if args.pairing == "bijection" else ltpc.PAIR_KEY
    wl["pairing_mode"] = pmode
    col = ltpc.Collider.from_workload(wl, precision=ltpc.F32 if prec == "f32" else ltpc.F64)
    dt = col.dt
    col.load_workload(wl)
    n0 = col.count()
    table = 0
    if not args.no_autotune:              # class table (block/cluster shapes) chosen by measurement
        table = col.autotune(dt)
    classes = col.classes()
    stream = torch.cuda.current_stream()

    # ---- the learned part: trained briefly on this workload's own particle data (another seed),
    # then served in-loop every step and checked against the exact per-cell reduction
    from paper_2508_06771_gb300 import surrogate as SG
    net = ltpc.Surrogate(batch_max=4096, n_cells_max=wl["M"], seed=rank)
    sur = {"trained": False}
    if not args.no_train:
        t0 = time.perf_counter()
        SG.identity_norm(net)
        wl_tr, _ = make_workload(args.workload, seed=1000 + rank, cells=args.cells)
        wl_tr["pairing_mode"] = pmode
        col_tr = ltpc.Collider.from_workload(wl_tr)
        col_tr.load_workload(wl_tr)
        X, T, _ = SG.collect(col_tr, net, dt, 0, args.train_steps, every=args.train_every,
                             per_cells=(100, 300, 1000, 0))
        col_tr.close()
        del col_tr
        Xn, Tn = SG.fit_norm(net, X, T)
        losses = SG.train(net, Xn, Tn, epochs=args.train_epochs, batch=4096, lr=1e-3)
        del X, T, Xn, Tn
        torch.cuda.empty_cache()
        sur = {"trained": True, "samples": int(wl["M"] * (args.train_steps // args.train_every) * 4),
               "snapshot_every": args.train_every, "epochs": args.train_epochs,
               "final_loss": losses[-1] if losses else None, "train_seconds": time.perf_counter() - t0}
    rates = torch.empty((wl["M"], 2), dtype=torch.float32, device="cuda")

    def full_step(k):
        col.step(dt, k)
        net.infer(col, rates)

    # storage compaction inside the timed region when the workload appends particles
    appends = bool(wl.get("neutral", False) and wl.get("n_neutral", 0.0) > 0)
    compact_every = args.compact_every if appends else 0

    step = 0
    # ---- accuracy probe: the first step's moments of sampled cells (compared with the oracle
    # in the CPU-baseline leg, the only place the benchmark runs it)
    probe = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cells = sample_cells(wl)
        col.step(dt, step)
        mom0, _ = col.moments()
        col.sync()
        probe = {"wl": wl, "cells": cells, "mom": mom0[cells], "step": step, "prec": prec,
                 "neutral": bool(wl.get("neutral", False) and wl.get("n_neutral", 0.0) > 0), "pairing_mode": pmode}
        step += 1
    # warm-up (also captures the graph)
    for _ in range(args.warmup):
        full_step(step)
        step += 1
    col.sync()
    n_start = col.count()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- timed region: K graph replays, device-resident inputs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(args.steps):
            full_step(step + k)
            if compact_every and (k + 1) % compact_every == 0:
                col.compact()                    # appended particles back into their cells' runs
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    step += args.steps
    ms = e0.elapsed_time(e1)
    col.sync()
    n_end = col.count()
    updates = args.steps * (n_start + n_end) / 2.0      # particle count grows ~linearly through the run
    ms_max, upd_all = reduce_over_ranks(ms, updates, world, "cuda")
    value = upd_all / (ms_max / 1e3)
    launches_per_step = 3 + len(classes) + 3      # scatter, cells per class, regroup, append; surrogate x3
    # a compaction: scatter, cursors, gather; the load's state, histogram, finite check, two run
    # kernels, regroup; the moments pass (scatter, cells per class, regroup, append)
    launches_per_compaction = 3 + 6 + 3 + len(classes) + 1   # and the step state before the next replay
    n_compactions = args.steps // compact_every if compact_every else 0
    # in-loop check: surrogate rates of the last step against the exact particle reduction
    _, exact = net.features(col, normalize=False)
    pred = net.infer(col)
    mi = exact[:, 0] > 0
    if sur["trained"] and bool(mi.any()):
        sur["k_ion_rel_err_median"], sur["k_ion_rel_err_mean"] = SG.relative_errors(pred[:, 0], exact[:, 0], mi)
        sur["k_el_rel_err_median"], sur["k_el_rel_err_mean"] = SG.relative_errors(pred[:, 1], exact[:, 1])
    else:
        sur["errors"] = None
        sur["why"] = "not trained in this run" if not sur["trained"] else "no electron-neutral collisions in this workload"
    sur["served"] = "every step, all cells (features from the fused moments, BF16 MLP, rates)"

    # ---- per-kernel device times (CUDA events on the launching stream) for the roofline
    nprof = min(max(args.steps, 5), 30)
    per = []
    for _ in range(nprof):
        per.append(col.profile_step(dt, step))
        step += 1
    per = np.array(per)
    avg = per.mean(0)
    names = ["scatter"] + [f"cells_C{c['cluster']}x{c['threads']}" for c in classes] + ["regroup", "append"]
    dom = int(np.argmax(avg))
    n_now = col.count()
    # count the particles the dominant class processes
    counts = col.grouping()[2].astype(np.int64) if dom not in (0, len(names) - 2, len(names) - 1) else None
    if counts is not None:
        k = dom - 1
        lo = classes[k - 1]["max_n"] if k > 0 else 0
        hi = classes[k]["max_n"]
        units = int(counts[(counts > lo) & (counts <= hi)].sum())
        bpp = algorithmic_bytes_per_particle(prec)
    else:
        units, bpp = n_now, 8
    alg_bytes = units * bpp
    achieved = alg_bytes / (avg[dom] * 1e-3) / 1e9
    peak, peak_src = peaks()
    traffic = recorded_traffic(args.workload) if dom not in (0,) else None

    # ---- FP64 plain form on the same workload (no graph), for the FP32-vs-FP64 comparison
    fp64 = None
    colD = None
    if prec == "f32" and not args.no_fp64:
        colD = ltpc.Collider.from_workload(wl, precision=ltpc.F64, use_graph=False)
        try:
            colD.load_workload(wl)
        except ltpc.LtpcError as e:       # e.g. cells above the binary64 shapes' capacity
            fp64 = {"unavailable": str(e)}
            colD.close()
            colD = None
    if colD is not None:
        colD.run(dt, 0, 2)
        colD.sync()
        ns = max(3, min(10, args.steps // 10))
        nA = colD.count()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        colD.run(dt, 2, ns)
        f1.record(stream)
        torch.cuda.synchronize()
        colD.sync()
        nB = colD.count()
        fms = f0.elapsed_time(f1)
        fp64 = {"value": ns * (nA + nB) / 2.0 / (fms / 1e3), "unit": UNIT, "ms_per_step": fms / ns,
                "steps": ns, "form": "same kernels in binary64, one launch per class, no graph, no correction"}
        fp64["fp32_speedup"] = value / world / fp64["value"]
        colD.close()
        colD = None
        torch.cuda.empty_cache()

    # ---- cached grouping (the per-step CCS3 scatter skipped while no particle was loaded or
    # appended), reported beside the default, which groups every step
    cached = None
    if not args.no_cached:
        if wl.get("neutral", False) and wl.get("n_neutral", 0.0) > 0:
            cached = {"applicable": False,
                      "why": "ionization appends particles nearly every step, so the grouping is redone"}
        else:
            colC = ltpc.Collider.from_workload(wl, precision=col.precision, cache_grouping=True)
            colC.set_class_table(table)
            colC.load_workload(wl)
            colC.run(dt, 0, 3)
            colC.sync()
            nc = max(3, min(50, args.steps))
            nCa = colC.count()
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            colC.run(dt, 3, nc)
            c1.record(stream)
            torch.cuda.synchronize()
            colC.sync()
            cms = c0.elapsed_time(c1)
            cached = {"applicable": True, "value": nc * (nCa + colC.count()) / 2.0 / (cms / 1e3), "unit": UNIT,
                      "ms_per_step": cms / nc, "steps": nc}
            colC.close()
            colC = None
            torch.cuda.empty_cache()

    # ---- end to end through the C ABI: host buffers in, moments out, every step.
    # Two contexts on two streams alternate steps, so the host-to-device copy of
    # step s+1's inputs (the link is the bound) overlaps the kernels of step s.
    e2e = None
    if not args.no_e2e:
        ne = max(20, min(60, args.steps // 10))
        host = [torch.from_numpy(np.ascontiguousarray(wl[k], dtype=np.float32 if prec == "f32" else np.float64))
                .pin_memory() for k in ("vx", "vy", "vz")]
        hcell = torch.from_numpy(np.ascontiguousarray(wl["cell"], dtype=np.int32)).pin_memory()
        hn = [h.numpy() for h in host]
        s2 = torch.cuda.Stream()
        col2 = ltpc.Collider.from_workload(wl, precision=col.precision, stream=s2)
        col2.set_class_table(table)
        net2 = ltpc.Surrogate(batch_max=4096, n_cells_max=wl["M"], seed=rank)
        net2.set_params(net.get_params())
        net2.set_norm(*net.norm)
        rates2 = torch.empty_like(rates)
        lanes = []
        for c_, n_, r_ in ((col, net, rates), (col2, net2, rates2)):
            lanes.append((c_, n_, r_, torch.empty((wl["M"], 10), dtype=torch.float64).pin_memory(),
                          torch.empty((wl["M"], 64), dtype=torch.int32).pin_memory()))

        def issue(k):
            c_, n_, r_, _, _ = lanes[k % 2]
            c_.load_host(hn[0], hn[1], hn[2], hcell.numpy(), asynchronous=True)
            c_.step(dt, k)
            n_.infer(c_, r_)

        for k in range(2):                      # warm both lanes (graph capture)
            issue(k)
            lanes[k % 2][0].moments_host(lanes[k % 2][3].numpy(), lanes[k % 2][4].numpy())
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        issue(0)
        for k in range(ne):
            if k + 1 < ne:
                issue(k + 1)
            c_, _, _, hm, hh = lanes[k % 2]
            c_.moments_host(hm.numpy(), hh.numpy())      # this step's result on the host
        torch.cuda.synchronize()
        barrier()
        el = time.perf_counter() - t0
        for c_ in (col, col2):
            c_.sync()                             # deferred load errors, if any
        el_max, upd_e = reduce_over_ranks(el, ne * n0, world, "cuda")
        es = 4 if prec == "f32" else 8
        e2e = {"value": upd_e / el_max, "unit": UNIT,
               "h2d_bytes_per_step": int(n0 * (3 * es + 4)),
               "d2h_bytes_per_step": int(wl["M"] * (10 * 8 + 64 * 4)), "steps": ne,
               "ms_per_step": el / ne * 1e3,
               "path": "ltpc_load_particles(pinned host, LTPC_LOAD_ASYNC) + ltpc_step + ltpc_mlp_infer + "
                       "ltpc_moments(host), two contexts on two streams alternating steps"}
        col2.close()
        net2.close()
        del col2, net2
        torch.cuda.empty_cache()

    # ---- the key-sort pairing on the same workload (the bijection mode is the default)
    key_leg = None
    if pmode == ltpc.PAIR_BIJECTION and not args.no_key_leg and int(np.bincount(wl["cell"]).max()) > 4096:
        wlk = dict(wl)
        wlk["pairing_mode"] = ltpc.PAIR_KEY
        colK = ltpc.Collider.from_workload(wlk, precision=col.precision)
        colK.load_workload(wlk)
        tk = colK.autotune(dt) if not args.no_autotune else 0
        colK.run(dt, 0, 3)
        colK.sync()
        nk = max(5, min(50, args.steps // 4))
        nKa = colK.count()
        torch.cuda.synchronize()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        colK.run(dt, 3, nk)
        k1.record(stream)
        torch.cuda.synchronize()
        colK.sync()
        kms = k0.elapsed_time(k1)
        perk = np.array([colK.profile_step(dt, 3 + nk + q) for q in range(5)]).mean(0)
        ck = colK.classes()
        cnt = colK.grouping()[2].astype(np.int64)
        dk = int(np.argmax(perk[1:1 + len(ck)]))
        lo = ck[dk - 1]["max_n"] if dk > 0 else 0
        uk = int(cnt[(cnt > lo) & (cnt <= ck[dk]["max_n"])].sum())
        ach = uk * algorithmic_bytes_per_particle(prec) / (perk[1 + dk] * 1e-3) / 1e9
        key_leg = {"pairing": "key sort (every particle's Philox key, per-cell bucket sort)",
                   "value": nk * (nKa + colK.count()) / 2.0 / (kms / 1e3), "unit": UNIT, "ms_per_step": kms / nk,
                   "steps": nk, "class_table_index": tk, "dominant_kernel_ms": float(perk[1 + dk]),
                   "roofline_frac": ach / peaks()[0]}
        colK.close()
        del colK
        torch.cuda.empty_cache()

    # ---- particles changing cells every step: the push in a field (S2b/S2c) and the grouping of
    # the new cells (CCS1-CCS3) every step, on the same electrons with positions
    push_leg = None
    if args.workload == "tail_4096x10000" and not args.no_push_leg:
        wlp = dict(wl)
        wlp["pairing_mode"] = ltpc.PAIR_KEY
        dxp = 2e-6
        rngp = np.random.default_rng([rank, 777])
        wlp["x"] = ((wl["cell"] + rngp.random(wl["cell"].size)) * dxp).astype(np.float32)
        colP = ltpc.Collider.from_workload(wlp, precision=col.precision)
        accel = np.full(wl["M"], -W_E_OVER_M * 3220.0)       # E = 32.2 V/cm along z (the paper's 0-D field)
        colP.set_field(dxp, accel, ltpc.WALL_PERIODIC)
        colP.load_workload(wlp)
        colP.run(dt, 0, 3)
        colP.sync()
        npu = max(5, min(50, args.steps // 4))
        nPa = colP.count()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        colP.run(dt, 3, npu)
        p1.record(stream)
        torch.cuda.synchronize()
        colP.sync()
        pms = p0.elapsed_time(p1)
        _, _, _, cellP, _ = colP.read()
        n0p = wlp["x"].size
        moved = float(np.mean(cellP[:n0p] != wl["cell"][:n0p]))
        push_leg = {"what": "Coulomb + e-n + push in E = 32.2 V/cm (periodic), regrouped every step, key-sort pairing",
                    "value": npu * (nPa + colP.count()) / 2.0 / (pms / 1e3), "unit": UNIT, "ms_per_step": pms / npu,
                    "steps": npu, "cell_width_m": dxp, "fraction_changed_cell_since_load": moved}
        colP.close()
        del colP
        torch.cuda.empty_cache()

    relaxation = relaxation_check(ltpc) if args.workload == "relax_64x1000" else None

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, accuracy = cpu_baseline(args.workload, pairing_mode=pmode, probe=probe)

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded numpy generator, one replica per rank)",
            "config": {"workload": desc, "cells": wl["M"], "particles_start": int(n0),
                       "particles_end_of_timed": int(n_end), "precision": f"{prec} velocities, collision "
                       "arithmetic and sums within a CTA; f64 across a cluster's CTAs and in the "
                       "moments", "graph": True,
                       "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (
                           n0 * (16 if prec == 'f32' else 28) / 1e6),
                       "class_table": [f"C={c['cluster']} x {c['threads']} thr, cells<={c['max_n']}" for c in classes],
                       "class_table_index": table, "autotuned": not args.no_autotune,
                       "pairing": ("keyed bijection of id ranks for cells > 4096 (candidates by pairing position), "
                                   "key sort below" if args.pairing == "bijection" else "key sort"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "compact_every": compact_every or None},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": names[dom],
                         "kernel_ms": float(avg[dom]), "algorithmic_bytes": int(alg_bytes),
                         "bytes_per_particle": bpp, "peak_source": peak_src,
                         "kernel_share": {n: float(a / avg.sum()) for n, a in zip(names, avg)}},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "cached_grouping": cached,
            "gpu_launches": int(launches_per_step * args.steps + launches_per_compaction * n_compactions),
            "clocks": clocks,
            "fp64_plain": fp64,
            "accuracy": accuracy,
            "relaxation": relaxation,
            "key_sort": key_leg,
            "push_every_step": push_leg,
            "surrogate": sur,
            "ns_per_particle_step": ms_max * 1e6 / (upd_all / world),
        }
        print(json.dumps(line), flush=True)
    col.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tail_4096x10000", choices=["relax_64x1000", "tail_4096x10000", "loguniform_256x256", "instances_64"])
    ap.add_argument("--no-autotune", action="store_true", help="keep the default class table")
    ap.add_argument("--no-key-leg", action="store_true", help="skip the key-sort comparison leg")
    ap.add_argument("--no-push-leg", action="store_true", help="skip the push (re-grouping every step) leg")
    ap.add_argument("--pairing", default="bijection", choices=["key", "bijection"],
                    help="in-cell pairing: key sort, or the keyed bijection for cells above 4096")
    ap.add_argument("--cells", type=int, default=None,
                    help="tail_4096x10000 and loguniform_256x256 only: number of cells (profiling cases)")
    ap.add_argument("--compact-every", type=int, default=200,
                    help="steps between storage compactions in the timed region (0: never; workloads with appends)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cached", action="store_true", help="skip the cached-grouping leg")
    ap.add_argument("--no-train", action="store_true", help="serve the surrogate with its initial weights")
    ap.add_argument("--train-steps", type=int, default=1024)
    ap.add_argument("--train-every", type=int, default=16)
    ap.add_argument("--train-epochs", type=int, default=8)
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_worker:
        oracle_worker(args.oracle_worker)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
