#!/usr/bin/env python
"""Benchmark: star-updates/s of the Henon Monte Carlo timestep on GB300.

Default workload: Plummer sphere, N = 10^7 equal-mass stars (Henon units),
mixed-precision orbits, one cluster per GPU.  A "step" is one full timestep
(Eq. 7 bins, relaxation, new orbits, sort, potential, energy correction)
through the library's graph-captured cmc_step.  Inputs (0.6 GB of state)
are larger than the L2 cache; no flush is needed between steps.

Prints one JSON line on rank 0.  --impl reference times the FP64 oracle on
the host cores instead (a bounded sample of the same workload per step).
Multi-GPU (torchrun): independent replicas, one cluster per rank (weak
scaling); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "star-updates/s per timestep at N=1e7 (1 GB300) + HBM roofline %, mixed vs FP64"
UNIT = "star-updates/s"
# the step profiles (ncu launch lists at N = 1e7) the roofline's traffic comes from
PROFILES = [os.path.join(ROOT, "profiles", "step_kernels_N1e7_%s.md" % p)
            for p in ("mixed", "fp64")]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return None
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f if l.strip()]
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ peaks, roofline
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of every CUDA source of the library (as the profile summaries
    record it): a summary's DRAM figures count only for the same kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1206_5878_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".hpp")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic_per_star(kernel: str, precision: str):
    """DRAM bytes per star of one kernel launch from the committed ncu
    summary, or None when a kernel source changed since it was taken."""
    for path in PROFILES:
        if not os.path.exists(path):
            continue
        src, val = None, None
        with open(path) as f:
            for line in f:
                if line.startswith("source_hash:"):
                    src = line.split(":", 1)[1].strip()
                if line.startswith("dram_bytes_per_star_%s_%s:" % (kernel, precision)):
                    val = float(line.split(":", 1)[1])
        if val is not None:
            return val if src == kernel_source_hash() else None
    return None


def profiled_fp64_pipe(kernel: str):
    """The FP64 pipe's active fraction in one kernel from the committed ncu
    counter summary (N = 4e6, mixed), or None when a kernel source changed
    since it was taken."""
    path = os.path.join(ROOT, "profiles", "kernels_counters_N4e6_mixed.md")
    if not os.path.exists(path):
        return None
    src, val = None, None
    with open(path) as f:
        for line in f:
            if line.startswith("source_hash:"):
                src = line.split(":", 1)[1].strip()
            if line.startswith("fp64_pipe_pct_%s:" % kernel):
                val = float(line.split(":", 1)[1]) / 100.0
    return val if val is not None and src == kernel_source_hash() else None


# Compulsory HBM bytes per star of each stage's kernels (table probes and
# scratch between the kernels of one stage not counted), and the kernel
# that carries the stage (mixed mode).
#   timestep:   r, v_r, v_t, m read (32 B)
#   relax:      v_r, v_t, m (8 B each), id (4 B) read; v_r, v_t written
#   turning:    r, v_r, v_t, Phi read; r_min, r_max written
#   orbit:      r, v_r, v_t, Phi, m, id read; sort key and 48-B payload written
#   sort:       5 passes of key + value read and written
#   gather:     key, value and payload read; r, 1/r, v_r, v_t, m, id, r_old, c written
#               (with the potential's per-tile sums of m and m/r)
#   potential:  1/r, m read; Phi, M, the float table written
#   correction: r, 1/r, Phi, v_r, v_t, r_old, c read; v_r, v_t written
STAGE_BYTES = {"timestep": 32, "relax": 44, "turning": 48, "orbit": 5 * 8 + 4 + 8 + 48,
               "sort": 5 * 24, "gather": 12 + 48 + 60, "potential": 16 + 24,
               "correction": 56 + 16}
STAGE_KERNEL = {"timestep": "k_bins", "relax": "k_relax", "turning": "k_turning_mixed",
                "orbit": "k_orbit", "sort": "k_pass", "gather": "k_gather",
                "potential": "k_potential", "correction": "k_correction_mixed"}



# FP64 peak derived from the unit counts and clock (nominal 1.25 TFLOP/s)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# FP64 operations per star of the formulas of the kernels that can dominate
# a step (each +, -, x, /, sqrt counted once):
#   k_relax (98 per pair of stars): two random azimuths (9 each: u^2, v^2,
#     their sum, its reciprocal, two products for cos, three for sin), the
#     second star's velocity (2), w and |w|^2 (8), |w| (1), the deflection
#     numerator pi m^2 n lnL dt (5) and sin^2(beta/2) (2), cos beta, sin beta
#     (6), the frame e1, u (12), w' (17), the mass ratios (3), the new
#     velocities (12) and the two new tangential speeds (8)
#   k_turning_mixed (28 per bound star): E (5), J (1), the r_max root in its
#     shell (13), the r_min root (9, sharing J^2)
KERNEL_FLOPS = {"relax": ("k_relax", 98 / 2), "turning": ("k_turning_mixed", 28)}
# ------------------------------------------------------------ oracle sample
def oracle_sample_step(state, n_orbit: int, seed: int, step: int):
    """One oracle timestep measured on a bounded sample of the workload:
    Eq. 7 bins, relaxation, sort, potential and energy correction on all N
    stars, the orbit step on n_orbit random stars scaled to N.  Returns the
    seconds of one timestep of N stars."""
    import numpy as np

    import oracle
    r, vr, vt, m, ids, phi = state
    n = r.shape[0]
    lnL = oracle.coulomb_log(n)
    t0 = time.perf_counter()
    dt, nbin = oracle.timestep(r, vr, vt, m, lnL)
    vr2, vt2, _ = oracle.relax(vr, vt, m, ids, nbin, dt, lnL, seed, step)
    t1 = time.perf_counter()
    rng = np.random.default_rng(step)
    ks = rng.choice(n, size=min(n_orbit, n), replace=False)
    rn = r.copy()
    tt = time.perf_counter()
    rn[ks] = oracle.orbit_sample(r, phi, vr2, vt2, ids, ks, seed, step)
    t2 = time.perf_counter()
    perm = oracle.sort_perm(rn, ids)
    t3 = time.perf_counter()
    phin = oracle.potential(r, m, "recursion")
    oracle.energy_correction(r, phin, vr2, vt2, r, np.zeros(n))
    t4 = time.perf_counter()
    per_star_sample = (t2 - tt) / len(ks)
    whole = (t1 - t0) + (t4 - t2)
    del perm
    return whole + per_star_sample * n


def host_cpu():
    """CPU model and core count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model or "unknown", "nproc": os.cpu_count()}


def oracle_full_steps(n: int, steps: int, seed: int = 1):
    """The oracle's complete timestep (every stage, every star, one core) on
    a Plummer cluster of n stars, measured over `steps` steps."""
    import initial_conditions as ic
    import oracle
    oracle.build()
    d = ic.plummer(n, seed=seed)
    o = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=seed)
    t0 = time.perf_counter()
    o.step(steps)
    sec = time.perf_counter() - t0
    return {"n_stars": n, "steps": steps, "value": n * steps / sec, "unit": UNIT,
            "ms_per_step": 1e3 * sec / steps, "cores": 1, "kind": "oracle",
            "sample": "complete oracle timesteps of a Plummer N=%d cluster, measured" % n}


def _ensemble_worker(args):
    """One process: one complete oracle timestep of each cluster assigned to
    it (the clusters of the 64-cluster ensemble)."""
    rank, nproc = args
    import initial_conditions as ic
    import oracle
    oracle.build()
    sizes = ic.ensemble_sizes(64, 1)
    done = 0
    sec = 0.0
    for c in range(rank, len(sizes), nproc):
        d = ic.plummer(int(sizes[c]), 1000 + c)
        o = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=1000 + c)
        t0 = time.perf_counter()
        o.step(1)
        sec += time.perf_counter() - t0
        done += int(sizes[c])
    return done, sec


def oracle_ensemble_per_core():
    """The 64-cluster ensemble on the host: one oracle process per core
    (spawned), each taking every nproc-th cluster through one complete
    timestep.  Rate = all clusters' stars / the slowest process's stepping
    time."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc) as pool:
        res = pool.map(_ensemble_worker, [(r, nproc) for r in range(nproc)])
    stars = sum(r[0] for r in res)
    sec = max(r[1] for r in res)
    return {"value": stars / sec, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": "one complete oracle timestep of each of the 64 ensemble clusters "
                      "(%d stars), one process per core, measured" % stars}


def build_oracle_state(n: int, seed: int):
    import numpy as np

    import initial_conditions as ic
    import oracle
    d = ic.plummer(n, seed=seed)
    perm = oracle.sort_perm(d["r"], d["id"])
    r, vr, vt, m, ids = (np.ascontiguousarray(d[k][perm]) for k in ("r", "vr", "vt", "m", "id"))
    phi = oracle.potential(r, m, "recursion")
    return r, vr, vt, m, ids, phi


def cpu_baseline(n: int, seed: int, n_orbit: int = 50_000):
    import oracle
    oracle.build()
    st = build_oracle_state(n, seed)
    sec = oracle_sample_step(st, n_orbit, seed, 0)
    return {"value": n / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "estimated_from_sample": True, "orbit_sample_stars": n_orbit,
            "sample": ("one oracle timestep of the N=%d Plummer cluster: Eq. 7 bins, "
                       "relaxation, sort, potential and energy correction measured on all "
                       "stars, the orbit step measured on %d random stars and its time "
                       "scaled to N (FP64, one core)" % (n, n_orbit)),
            "host": host_cpu()}


# ------------------------------------------------------------------ suite
# cmc_config.precision of the bench's names
PRECISIONS = {"fp64": 0, "mixed": 1, "fp64-bisection": 2}

SUITE = [
    # name, N, masses, precisions, steps (the measured-workload list)
    ("plummer_1e4_fp64", 10_000, "equal", ("fp64",), 10),
    ("plummer_1e5", 100_000, "equal", ("fp64", "mixed"), 200),
    ("salpeter_1e6_mixed", 1_000_000, "salpeter", ("mixed",), 100),
    ("ensemble_64", None, "equal", ("fp64", "mixed"), 50),
    ("plummer_1e7", 10_000_000, "equal", ("mixed", "fp64"), 20),
]


def run_suite(args):
    """Every measured workload: star-updates/s over the timed steps (CUDA
    events around the graph launches), total-energy drift from the start,
    the 10/50/90% Lagrangian radii at the end, the sort and potential stages
    against HBM (their compulsory bytes), and the oracle's star-updates/s on
    one core (whole steps up to N = 1e5, sampled orbit steps above).  One
    JSON line per workload and precision."""
    import numpy as np
    import torch

    import initial_conditions as ic
    import paper_1206_5878_gb300 as g
    g.load()
    hbm, _ = measured_peaks()
    for name, n, masses, precs, steps in SUITE:
        if name == "ensemble_64":
            cat, sizes, seeds = ic.ensemble(64, seed=1)
            state, sizes, seeds = cat, [int(x) for x in sizes], [int(x) for x in seeds]
            n = sum(sizes)
        else:
            d = ic.plummer(n, seed=1, masses=masses)
            state = {k: d[k] for k in ("r", "vr", "vt", "m", "id")}
            sizes, seeds = None, [1]
        dev = {k: torch.from_numpy(np.ascontiguousarray(
            v if k != "id" else v.view(np.int32))).cuda() for k, v in state.items()}
        cpu = None
        if args.cpu and name != "ensemble_64":
            cpu = cpu_baseline_full(n, masses) if n <= 100_000 else \
                cpu_baseline(n, 1, n_orbit=20_000)["value"]
        for prec in precs:
            c = g.Cluster(dev, seeds, sizes=sizes, precision=PRECISIONS[prec])
            E0 = c.total_energy()
            c.step(2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            c.step(steps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            drift = float(np.max(np.abs(c.total_energy() / E0 - 1)))
            stg = c.step_profiled(2)
            lag = c.lagrange_radii([0.1, 0.5, 0.9])[0].tolist() if sizes is None else None
            st = c.stats()
            esc = sum(x["escaped"] for x in st)
            out = {"workload": name, "precision": prec, "n_stars": n, "clusters": len(seeds),
                   "steps": steps + 2, "ms_per_step": ms,
                   "star_updates_per_s": n / (ms / 1e3),
                   "energy_drift": drift, "escaped": esc, "lagrange_10_50_90": lag,
                   "sort_hbm_frac": STAGE_BYTES["sort"] * n / (stg["sort"] / 2 / 1e3) / 1e9 / hbm,
                   "potential_hbm_frac": STAGE_BYTES["potential"] * n /
                   (stg["potential"] / 2 / 1e3) / 1e9 / hbm,
                   "stages_ms": {k: v / 2 for k, v in stg.items()},
                   "oracle_star_updates_per_s": cpu}
            print(json.dumps(out), flush=True)
            c.close()


def cpu_baseline_full(n: int, masses: str) -> float:
    """The oracle's whole timestep (every stage on every star) on one core."""
    import initial_conditions as ic
    import oracle
    oracle.build()
    d = ic.plummer(n, seed=1, masses=masses)
    o = oracle.Cluster(d["r"], d["vr"], d["vt"], d["m"], d["id"], seed=1)
    t0 = time.perf_counter()
    o.step(1)
    return n / (time.perf_counter() - t0)


# ------------------------------------------------------------------- arms
def run_reference(args, rank, world):
    """The oracle on the host cores, on the GPU arm's workload (Plummer N
    stars, seed), each step a bounded sample of it: the O(N) stages (Eq. 7
    bins, relaxation, sort, potential, energy correction) on all N stars and
    the orbit step on a random sample of stars against the full table.
    The rate is the oracle's per-star-update cost measured on that sample,
    1 / (t_all_stages / N + t_orbit / n_sample): an estimate of a whole
    N-star step, never a timed one (a whole step of 10^7 stars takes the
    oracle minutes); ms_per_step is the sampled step's measured wall time."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    log("reference arm: oracle on the host, N=%d" % args.n)
    st = build_oracle_state(args.n, args.seed)
    n_orbit = args.ref_orbit_sample
    for w in range(args.warmup):
        oracle_sample_step(st, n_orbit, args.seed, w)
    est, wall = 0.0, 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        est += oracle_sample_step(st, n_orbit, args.seed, args.warmup + k)
        wall += time.perf_counter() - t0
    value = args.n * args.steps / est
    sample = ("per step: Eq. 7 bins, relaxation, sort, potential and energy correction "
              "measured on all %d stars, the orbit step measured on %d random stars; the "
              "rate is N / (t_stages + t_orbit N / %d) (FP64, one core)"
              % (args.n, n_orbit, n_orbit))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "Plummer N=%d equal-mass, fp64 orbits (oracle; orbit "
                                   "step sampled on %d stars per step)" % (args.n, n_orbit),
                       "n_stars": args.n, "precision": "fp64 (the oracle on the host)",
                       "seed": args.seed, "parallelism": "single"},
            "estimated_from_sample": True,
            "estimated_ms_per_full_step": 1e3 * est / args.steps,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "estimated_from_sample": True, "orbit_sample_stars": n_orbit,
                             "sample": sample, "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    if args.ref_full:
        line["measured_full_step"] = oracle_full_steps(100_000, 2, args.seed)
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ranks
class Ranks:
    """The launch's ranks as the timing sees them: a barrier on both sides
    of the timed region and the maximum time over ranks.  device: "cuda"
    with NCCL on a GPU box, "cpu" with gloo (the multi-process tests)."""

    def __init__(self, rank: int, world: int, device: str = "cuda"):
        self.rank, self.world, self.device = rank, world, device

    def _sync(self):
        if self.device == "cuda":
            import torch
            torch.cuda.synchronize()

    def barrier(self):
        self._sync()
        if self.world > 1:
            import torch
            torch.distributed.barrier()
        self._sync()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())


def replica_seed(base: int, rank: int) -> int:
    """One independent cluster per rank (weak scaling): seed base + rank."""
    return base + rank


def whole_job_rate(n_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Star-updates/s of all ranks together over the slowest rank's time."""
    return n_per_rank * steps * world / (ms_max / 1e3)


def run_cmc(args, rank, world, local_rank):
    import numpy as np
    import torch

    import initial_conditions as ic
    import paper_1206_5878_gb300 as g

    torch.cuda.set_device(local_rank)
    ranks = Ranks(rank, world, "cuda")
    seed = replica_seed(args.seed, rank)
    n = args.n
    prec = PRECISIONS[args.precision]
    log("rank %d: building Plummer N=%d seed=%d" % (rank, n, seed))
    d = ic.plummer(n, seed=seed)
    dev = {k: torch.from_numpy(d[k].view(np.int32) if k == "id" else d[k]).cuda()
           for k in ("r", "vr", "vt", "m", "id")}
    c = g.Cluster(dev, [seed], precision=prec, rng=args.rng)
    stream = torch.cuda.current_stream()

    barrier, max_over_ranks = ranks.barrier, ranks.max
    dist = world > 1

    c.step(args.warmup)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        ev0.record(stream)
        c.step(args.steps)
        ev1.record(stream)
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    clocks = clk.summary()
    value = whole_job_rate(n, args.steps, world, ms)
    kernels = c.kernels_per_step() * args.steps

    # per-stage device times over the same number of steps (kernels launched
    # one by one with events between the stages)
    stages = c.step_profiled(args.steps)
    stages_avg = {k: v / args.steps for k, v in stages.items()}
    hbm, peak_kind = measured_peaks()
    # roofline of the dominant single kernel: the FP64-bound relaxation or
    # turning-point kernel (every other stage is shorter or several kernels)
    dom = max(KERNEL_FLOPS, key=lambda k: stages_avg.get(k, 0.0))
    dom_ms = stages_avg[dom]
    kname, flops_per_star = KERNEL_FLOPS[dom]
    nflops = flops_per_star * n
    achieved = nflops / (dom_ms / 1e3) / 1e9
    tun = c.tuning()
    traffic_ps = profiled_traffic_per_star(kname, args.precision)
    alg_bytes = STAGE_BYTES[dom] * n
    roof = {"kernel": kname, "stage": dom, "bound": "alu", "achieved": achieved,
            "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
            "peak_source": "derived (FP64): 152 SMs x 2 FMA lanes/clock x 2 flop x 2.07 GHz",
            "algorithmic_flops_per_launch": nflops,
            "traffic": None if traffic_ps is None else traffic_ps * n,
            "launch_ms": dom_ms,
            # the same kernel against HBM: its compulsory bytes, and the
            # DRAM bytes ncu measured (when the profile is current)
            "algorithmic_bytes_per_launch": alg_bytes,
            "hbm_frac_algorithmic": alg_bytes / (dom_ms / 1e3) / 1e9 / hbm,
            "hbm_frac_dram": None if traffic_ps is None
            else traffic_ps * n / (dom_ms / 1e3) / 1e9 / hbm,
            "hbm_peak_gbs": hbm, "hbm_peak_source": peak_kind,
            # what bounds it: the FP64 pipe's active fraction (ncu, N = 4e6)
            "fp64_pipe_active_ncu": profiled_fp64_pipe(kname),
            "note": "FP64 operations of the kernel's formulas (+, -, x, /, sqrt once each); "
                    "compiled without FMA contraction for bit-exact parity, so half the FMA "
                    "peak is the issue ceiling, and / and sqrt take several FP64 issues each"}
    # step-level compulsory traffic (248 B per star-update) against HBM
    step_frac = 248.0 * value / world / 1e9 / hbm

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64+f32" if prec == 1 else "f64", "data": "synthetic",
           "config": {"workload": "Plummer N=%d equal-mass, %s orbits" % (n, args.precision)
                      + ("" if args.rng == "philox" else ", Tausworthe streams"),
                      "rng": args.rng,
                      "n_stars": n, "precision": args.precision, "seed": args.seed,
                      "parallelism": "replicas" if dist else "single",
                      "l2": "inputs larger than L2 (state %.2f GB)" % (n * 60 / 1e9)},
           "gpu_launches": kernels, "stages_ms": stages_avg, "tuning": tun,
           "roofline": roof,
           "step_hbm_frac": step_frac, "clocks": clocks}

    if args.fp64 and prec == 1:
        c64 = g.Cluster(dev, [seed], precision=0)
        c64.step(1)
        barrier()
        k64 = max(1, min(args.steps, 3))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c64.step(k64)
        e1.record(stream)
        barrier()
        ms64 = max_over_ranks(e0.elapsed_time(e1))
        out["fp64"] = {"value": n * k64 * world / (ms64 / 1e3), "unit": UNIT,
                       "ms_per_step": ms64 / k64, "steps": k64,
                       "path": "FP32 screening with error bounds, every decision FP64's"}
        c64.close()
        # the same FP64 results by bisection on the FP64 table (one step)
        cb = g.Cluster(dev, [seed], precision=2)
        cb.step(1)
        barrier()
        e0.record(stream)
        cb.step(1)
        e1.record(stream)
        barrier()
        msb = max_over_ranks(e0.elapsed_time(e1))
        out["fp64_bisection"] = {"value": n * world / (msb / 1e3), "unit": UNIT,
                                 "ms_per_step": msb, "steps": 1}
        cb.close()

    if args.e2e:
        # the public API with host buffers: per step, the state goes in from
        # pinned host memory, one timestep runs, the state comes back
        pin = {k: torch.empty(n, dtype=torch.float64, pin_memory=True)
               for k in ("r", "vr", "vt", "m")}
        pin["id"] = torch.empty(n, dtype=torch.int32, pin_memory=True)
        hst = {k: v.numpy() for k, v in pin.items()}
        hst["id"] = hst["id"].view(np.uint32)
        st0 = c.get_state({k: hst[k] for k in ("r", "vr", "vt", "m", "id")})
        step0 = st0["step"]
        k_e2e = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for i in range(k_e2e):
            c.set_state(hst, step0 + i)
            c.step(1)
            c.get_state(hst)
        barrier()
        sec = max_over_ranks(time.perf_counter() - t0)
        out["e2e"] = {"value": n * k_e2e * world / sec, "unit": UNIT,
                      "h2d_bytes_per_step": n * (4 * 8 + 4),
                      "d2h_bytes_per_step": n * (4 * 8 + 4), "steps": k_e2e,
                      "api": "cmc_set_state(host) + cmc_step(1) + cmc_get_state(host)"}
    c.close()

    if rank == 0 and args.cpu and world == 1:
        log("cpu baseline: oracle on a sample of the workload")
        out["cpu_baseline"] = cpu_baseline(n, args.seed, args.cpu_orbit_sample)
        log("cpu baseline: complete oracle steps at N=1e5, and the ensemble on every core")
        out["cpu_baseline"]["measured_full_step"] = oracle_full_steps(100_000, 2, args.seed)
        out["cpu_baseline"]["ensemble_per_core"] = oracle_ensemble_per_core()
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cmc", choices=["cmc", "reference"])
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--precision", default="mixed", choices=sorted(PRECISIONS))
    ap.add_argument("--rng", default="philox", choices=["philox", "taus113"],
                    help="draws: counter-based Philox (default) or the paper's combined "
                         "Tausworthe streams")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-fp64", dest="fp64", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu", action="store_false")
    ap.add_argument("--cpu-orbit-sample", type=int, default=50_000)
    ap.add_argument("--ref-orbit-sample", type=int, default=20_000)
    ap.add_argument("--no-ref-full", dest="ref_full", action="store_false",
                    help="reference arm: skip the measured complete oracle steps at N=1e5")
    ap.add_argument("--suite", action="store_true",
                    help="run every measured workload (one JSON line each) instead of the "
                         "N=1e7 benchmark line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.suite:
        run_suite(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_cmc(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
