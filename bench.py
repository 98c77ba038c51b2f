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
        wl = W.loguniform_256x256(seed=seed, dtype=np.float32)
        desc = f"loguniform_256x256: 256x256 cells, log-uniform 16..65536 per cell (N0={wl['vx'].size:,}), FP32, NRL lnL, Coulomb"
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
def oracle_sample(workload, cells=16):
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
    wl1, neutral = oracle_sample(args.workload, cells=16)
    v1, _, _ = oracle_rate(wl1, neutral, steps=1)
    per_particle = 1.0 / v1
    nsteps = args.steps + args.warmup
    target = 120.0 / nsteps / per_particle
    ppc = wl1["vx"].size / wl1["M"]
    cells = int(max(1, min(512, target // ppc)))   # at most ~5M particles per process
    wl, neutral = oracle_sample(args.workload, cells=cells)
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


def cpu_baseline(workload, budget_s=8.0):
    """The oracle as it stands on a bounded sample of the workload (rank 0, N=1), on one core
    and on every host core (one process per core)."""
    import oracle as orc
    orc.build()
    wl, neutral = oracle_sample(workload, cells=16)
    v1, el1, s1 = oracle_rate(wl, neutral, budget_s=budget_s)
    cores = host_cores()
    vn, eln, sn = oracle_rate(wl, neutral, budget_s=budget_s, processes=cores) if cores > 1 else (v1, el1, s1)
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle", "single_core": v1,
            "sample": f"{wl['M']} cells ({wl['vx'].size:,} particles) of the workload per process, full steps "
                      f"(Coulomb{' + e-n' if neutral else ''} + moments), FP64; {cores} processes x {sn} steps "
                      f"in {eln:.1f} s, and 1 process x {s1} steps in {el1:.1f} s"}


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

    step = 0
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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded numpy generator, one replica per rank)",
            "config": {"workload": desc, "cells": wl["M"], "particles_start": int(n0),
                       "particles_end_of_timed": int(n_end), "precision": f"{prec} velocities and collision "
                       "arithmetic, f64 per-cell sums", "graph": True,
                       "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (
                           n0 * (16 if prec == 'f32' else 28) / 1e6),
                       "class_table": [f"C={c['cluster']} x {c['threads']} thr, cells<={c['max_n']}" for c in classes],
                       "class_table_index": table, "autotuned": not args.no_autotune,
                       "pairing": args.pairing,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": names[dom],
                         "kernel_ms": float(avg[dom]), "algorithmic_bytes": int(alg_bytes),
                         "bytes_per_particle": bpp, "peak_source": peak_src,
                         "kernel_share": {n: float(a / avg.sum()) for n, a in zip(names, avg)}},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "cached_grouping": cached,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
            "fp64_plain": fp64,
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
    ap.add_argument("--pairing", default="key", choices=["key", "bijection"],
                    help="in-cell pairing: key sort, or the keyed bijection for cells above 4096")
    ap.add_argument("--cells", type=int, default=None, help="tail_4096x10000 only: number of cells (profiling cases)")
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
