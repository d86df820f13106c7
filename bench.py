"""Benchmark of the APIC particle-in-cell step on GB300.

Metric: particle-steps/s of full steps (deposit, Poisson solve to the stated
tolerance, gather, push, absorption tallies, escape, injection) on the
precision form at scale: alpha = 0.225 (a = 0.45), B = 1, 1024 x 512 cells,
5e7 macro-particles per species, FP32 particles with the Poisson problem
solved in FP32 inside an FP64 residual refinement to 1e-10.  The line states
the FP32 path's error against the FP64 oracle (one step from the same states,
the same workload on 256 x 128 cells).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torch.distributed.run; every rank advances an independent
replica (the path has no data exchange between GPUs), rank 0 prints one JSON
line with the whole-job throughput.  The reference arm (--impl reference) is
the FP64 CPU oracle on a bounded sample of the same workload, one replica per
host core.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (full PIC step) FP32+refined vs FP64 at stated error; % HBM roofline"
UNIT = "particle-steps/s"
BYTES_PER_PARTICLE_STEP = 40  # FP32 state (x1, x2, vR, vZ, vTheta) read once and written once
# FP32 operations of one particle update as the equations state them (Eq. 3
# radius, cell and weights, bilinear gather of the two node gradients, the
# metric of Eq. 10, the Boris step of Eq. 9, the chord and rotation, the
# grain and escape tests, Eq. 2 and the new cell): 127, counted per
# operation (a multiply-add as two, a square root or division as one)
FLOPS_PER_PARTICLE_STEP = 127


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=30)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=None,
                    help="macro-particles per species (default: the workload's own count)")
    ap.add_argument("--workload", default="dipole1024",
                    choices=["dipole256", "dipole1024", "batched48", "sphere64", "window", "boltzmann256",
                             "floating256"],
                    help="window: the sensitivity window (forward-mode derivatives along alpha, phi_g, B) on the "
                         "256x128 dipole, 1e6 particles per species, K = 10 steps per window")
    ap.add_argument("--instances", type=int, default=None,
                    help="batched48 only: the first N instances (smaller runs, e.g. under a profiler)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--sort-interval", type=int, default=None,
                    help="override the workload's sort interval (steps between particle sorts)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the workload's sort interval and the default tiles (by default apic_autotune "
                         "chooses the sort interval and the push's tiles after the warm-up, untimed)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workloads(name="dipole256", n_per_species=None, n_instances=None):
    """List of instance configurations of the named workload (batched48:
    its first n_instances instances when given, e.g. for a profiler capture
    that must stay small)."""
    from paper_2307_11107_gb300 import workloads as W
    if name == "batched48":
        cs = W.batched_48()[:n_instances] if n_instances else W.batched_48()
        if n_per_species:
            for c in cs:
                c["species"] = [dict(sp, n_init=n_per_species) for sp in c["species"]]
        return cs
    if name == "dipole1024":
        c = W.dipole_1024("fp32")
    elif name == "boltzmann256":
        c = W.dipole_256_boltzmann("fp32")
    elif name == "floating256":
        c = W.dipole_256_floating("fp32")
    elif name == "sphere64":
        c = W.spherical_small("fp64")
    else:
        c = W.dipole_256("fp32")
    if n_per_species:
        c["species"] = [dict(sp, n_init=n_per_species) for sp in c["species"]]
    return [c]


def workload(n_per_species=None, name="dipole256"):
    return workloads(name, n_per_species)[0]


def replica_configs(name, n_per_species, rank, history_cap, n_instances=None):
    """Instance configurations of rank `rank`'s replica: the workload's own
    instances renumbered so that no two ranks share a random stream (the
    instance number is part of every Philox counter)."""
    cfgs = workloads(name, n_per_species, n_instances)
    for c in cfgs:
        c["instance"] = c.get("instance", 0) + rank * len(cfgs)
        c["history_cap"] = history_cap
    return cfgs


def replica_throughput(advanced, seconds, pg=None, device="cpu"):
    """Whole-job throughput of independent replicas: the particle-steps of all
    ranks summed, divided by the slowest rank's time.  Returns (value,
    particle-steps, seconds)."""
    if pg is None:
        return advanced / seconds, float(advanced), float(seconds)
    import torch
    adv = torch.tensor([float(advanced)], dtype=torch.float64, device=device)
    sec = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    pg.all_reduce(adv)
    pg.all_reduce(sec, op=pg.ReduceOp.MAX)
    a, t = float(adv.item()), float(sec.item())
    return a / t, a, t


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    architecture)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


# The CPU oracle's banded LU of a 1024 x 512 grid is 6.5 GB, takes about 95 s
# to factor on one core and about 1.1 s per solve (x86 host; factor ~ n1 n2^3,
# solve ~ n1 n2^2).  The CPU-baseline leg of the main line runs the same
# workload on 256 x 128 cells (the downsampled grid of the precision form's
# comparison); the reference arm runs the largest grid whose factorisation and
# solves fit its time budget (the full grid for short runs).
ORACLE_MAX_GRID = (256, 128)


def oracle_workload(cfg, grid=ORACLE_MAX_GRID):
    """The workload as the CPU oracle runs it: the same parameters, the grid
    reduced to at most `grid` cells."""
    c = dict(cfg)
    c["n1"], c["n2"] = min(cfg["n1"], grid[0]), min(cfg["n2"], grid[1])
    return c


def reference_grid(cfg, total_steps, budget_s=150.0):
    """Largest grid (the workload's, else halved in both directions) whose
    oracle set-up and total_steps Poisson solves take at most budget_s."""
    n1, n2 = cfg["n1"], cfg["n2"]
    while n1 > 64:
        a, b = n1 / 1024.0, n2 / 512.0
        if 95.0 * a * b ** 3 + total_steps * 1.1 * a * b * b <= budget_s:
            break
        n1, n2 = n1 // 2, n2 // 2
    return n1, n2


def _oracle_replica(job):
    """One oracle replica (a process of its own): warm-up steps untimed, then
    timed steps; returns (particle-steps advanced, seconds)."""
    cfg, n, warmup, steps, tag = job
    cfg = dict(cfg)
    sys.path.insert(0, ROOT)
    import oracle
    c = dict(cfg, instance=tag)
    c["species"] = [dict(s, n_init=n) for s in cfg["species"]]
    sim = oracle.Sim(c)
    for sp in range(len(c["species"])):
        sim.load_volume(sp, n)
    sim.step(warmup)
    adv = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        adv += sum(sim.count(sp) for sp in range(len(c["species"])))
        sim.step(1)
    return adv, time.perf_counter() - t0


def run_oracle(cfg, n_per_species, steps, warmup=0, cores=1, grid=ORACLE_MAX_GRID):
    """The FP64 CPU oracle as it stands on `steps` steps of the workload (grid
    per oracle_workload) with n_per_species macro-particles per species (the
    macro weight follows n_per_species), after `warmup` untimed steps.  With
    cores > 1, that many independent replicas (distinct random streams) run in
    spawned processes at once, one per core.  Returns (particle-steps/s of all
    replicas, seconds of the slowest)."""
    c = oracle_workload(cfg, grid)
    jobs = [(c, n_per_species, warmup, steps, 1000 + k) for k in range(cores)]
    if cores == 1:
        res = [_oracle_replica(jobs[0])]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_replica, jobs)
    adv = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    return adv / secs, secs


def profile_figure(key, workload_name):
    """A figure recorded under profiles/ (profiles/figures.txt lines
    "<key> <workload> <value>"), or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "figures.txt")) as f:
            for line in f:
                p = line.split()
                if len(p) >= 3 and p[0] == key and p[1] == workload_name:
                    return float(p[2])
    except Exception:
        pass
    return None


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cfg = workload(args.particles, args.workload if args.workload in ("dipole256", "dipole1024") else "dipole1024")
    steps, warm = max(1, args.steps), max(0, args.warmup)
    grid = reference_grid(cfg, steps + warm)
    oc = oracle_workload(cfg, grid)
    # one process: the banded LU's memory (6.5 GB on the full grid) is not
    # replicated per core; bounded particle sample, ~1.7e7 particle-steps/s
    cores = 1
    n = int(max(2000, min(cfg["species"][0]["n_init"], 5.0e8 / (2 * (steps + warm)))))
    val, secs = run_oracle(cfg, n, steps, warm, cores, grid)
    sample = ("%d untimed + %d timed full steps with %d macro-particles per species on %dx%d cells (FP64, banded LU "
              "factored once before the steps, 1 thread)" % (warm, steps, n, oc["n1"], oc["n2"]))
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
        "warmup": warm, "ms_per_step": 1e3 * secs / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "alpha": cfg["alpha"], "grid_cells": [cfg["n1"], cfg["n2"]],
                   "oracle_grid_cells": [oc["n1"], oc["n2"]], "particles_per_species": n, "sample": sample},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def precision_error(apic, cfg, n=200_000, seed=17):
    """The FP32 path's error against the FP64 oracle: one step of the same
    workload on the oracle's grid (oracle_workload) from the same FP32-rounded
    particle states (n per species, uniform in the logical box, Maxwellian
    velocities at each species' v_th).  Returns relative errors of rho and phi
    (max-norm), of the particles (largest scaled difference of matched
    states), of the grain charge and electric force, and of the absorbed
    counts."""
    import numpy as np
    import oracle
    c = oracle_workload(cfg)
    c = dict(c, no_inject=True, species=[dict(s, n_init=n) for s in cfg["species"]], poisson_max_iter=60)
    g, o = apic.Sim(c), oracle.Sim(c)
    rng = np.random.default_rng(seed)
    vth = [np.sqrt(s["T"] / s["m"]) for s in c["species"]]
    for sp in range(len(c["species"])):
        st = np.column_stack([rng.uniform(-0.999, c["x1_out"] - 1e-3, n), rng.uniform(-0.999, 0.999, n),
                              rng.standard_normal((n, 3)) * vth[sp]]).astype(np.float32).astype(np.float64)
        g.add_particles(sp, st)
        o.add_particles(sp, st)
    g.step(1)
    o.step(1)

    def rel(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    out = {"workload": "%s on %dx%d cells, one step, %d particles per species" % (cfg["name"], c["n1"], c["n2"], n),
           "rho": rel(g.field("rho"), o.grid("rho")), "phi": rel(g.field("phi"), o.grid("phi"))}
    from scipy.spatial import cKDTree
    worst, unmatched = 0.0, 0
    for sp in range(len(c["species"])):
        a, b = g.particles(sp), o.particles(sp)[0]
        scale = np.array([1.0, 1.0, vth[sp], vth[sp], vth[sp]])
        d, k = cKDTree(b / scale).query(a / scale)
        unmatched += abs(a.shape[0] - b.shape[0]) + int((np.unique(k, return_counts=True)[1] > 1).sum())
        worst = max(worst, float(np.sort(d)[-1 - min(unmatched, d.size - 1)]))
    t = g.tallies()
    sc = o.scalars()
    out.update(particles=worst, particles_unmatched=unmatched,
               grain_Q=abs(t["Q"] - sc["Q"]) / abs(sc["Q"]), grain_FZ=abs(t["FZ"] - sc["FZ"]) / max(abs(sc["FZ"]), 1e-300),
               absorbed=[t["counts"][sp]["absorbed"] - o.counts()[sp]["absorbed"] for sp in range(len(c["species"]))],
               tolerance={"fields": 2e-5, "particles": 2e-4})
    g.close()
    return out


def window_bench(args):
    """Sensitivity window (apic_sensitivity): the 256x128 dipole with 1e6
    macro-particles per species (or --particles), K = 10 steps per window,
    --steps windows timed with CUDA events after --warmup plain steps.  The
    value is the particle-steps advanced inside the windows per second."""
    import torch
    import paper_2307_11107_gb300 as apic
    from paper_2307_11107_gb300 import workloads as W
    apic.build()
    torch.cuda.set_device(0)
    K = 10
    cfg = W.dipole_256("fp32")
    n = args.particles or 1_000_000
    cfg["species"] = [dict(sp, n_init=n) for sp in cfg["species"]]
    cfg["history_cap"] = max(4096, (args.steps + 1) * K + args.warmup + 8)
    sim = apic.Sim(cfg)
    for sp in range(2):
        sim.load_volume(sp, n)
    sim.step(args.warmup)
    sim.sensitivity(2)  # tangent set-up outside the timed region
    stream = torch.cuda.current_stream()
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sim.sensitivity(K)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    hist = sim.tallies()["history"]
    steps = args.steps * K
    advanced = float((hist[-(steps + 1):-1, 7] + hist[-(steps + 1):-1, 8]).sum())
    line = {"metric": METRIC, "value": advanced / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sensitivity_window_256x128_2e6_K10", "window_steps": K, "windows": args.steps,
                       "particles_per_species": n, "parameters": ["alpha", "phi_g", "B"],
                       "outputs": ["drag F_Z", "electric F_Z", "current", "torque T_z", "grain charge Q"],
                       "precision": "FP32 particles and tangents; Poisson: " + sim.stats()["solver"]},
            "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "window":
        return window_bench(args)
    assert args.warmup >= 3, "at least 3 warm-up steps"
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    import paper_2307_11107_gb300 as apic
    apic.build()
    cfgs = replica_configs(args.workload, args.particles, rank, max(4096, args.steps + args.warmup + 8), args.instances)
    if args.sort_interval is not None:
        for c in cfgs:
            c["sort_interval"] = args.sort_interval
    cfg = cfgs[0]
    sim = apic.Sim(cfgs)
    for k, c in enumerate(cfgs):
        for sp in range(len(c["species"])):
            sim.load_volume(sp, c["species"][sp]["n_init"], instance=k)
    sim.step(args.warmup)
    tuned = None
    if not args.no_autotune and args.sort_interval is None:
        tuned = sim.autotune(max(8, args.warmup // 4))[0]
    tiles = sim.stats()

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    s0 = sim.stats()
    with ClockSampler(local) as clk:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    s1 = sim.stats()
    # particles advanced in timed step k = resident count after step k-1
    res = 0.0
    for k in range(len(cfgs)):
        hist = sim.tallies(k)["history"]
        res = res + hist[-(args.steps + 1):-1, 7] + hist[-(args.steps + 1):-1, 8]
    advanced = float(res.sum())
    value, total_adv, sec = replica_throughput(advanced, ms / 1e3, pg, "cuda")
    loop_iters = s1["poisson_loop_iters"] - s0["poisson_loop_iters"]
    launches = (args.steps * s1["kernels_per_step"] + loop_iters * s1["kernels_per_iter"] +
                (s1["sorts"] - s0["sorts"]) * s1["kernels_per_sort"])

    # roofline of the dominant kernel (push): CUDA events around its phase graph
    kt = min(args.steps, 100)
    sim.step_timed(kt)
    st = sim.stats()
    push_ms = st["phase_ms"]["push"] / kt
    n_avg = float(res.mean())
    peaks, src = measured_peaks()
    achieved = BYTES_PER_PARTICLE_STEP * n_avg / (push_ms / 1e3) / 1e9
    # the push kernel that ran: the FP32 vector push unless APIC_PUSH4=0
    vector = cfg.get("precision", "fp32") != "fp64" and os.environ.get("APIC_PUSH4", "1") != "0"
    kernel = "k_push4" if vector else "k_push"
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "k_push_traffic.txt")) as f:
            for line in f:
                if vector and line.startswith("dram_bytes_per_particle"):
                    traffic = float(line.split()[1]) * n_avg
    except Exception:
        pass
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "kernel": kernel,
            "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP, "peak_source": src,
            "push_ms": push_ms, "phase_ms_per_step": {k: v / kt for k, v in st["phase_ms"].items()},
            "sort_ms_per_sort": st["sort_ms"] / st["timed_sorts"] if st["timed_sorts"] else None}
    # the whole step against the same roofline: the particle state's bytes per
    # step over the step time (the solve, sort and injection add time, not bytes)
    full = BYTES_PER_PARTICLE_STEP * total_adv / args.steps / (ms / args.steps / 1e3) / 1e9
    roof["full_step"] = {"achieved": full, "frac": full / peaks["hbm_gbs"], "unit": "GB/s"}
    solve_ms = roof["phase_ms_per_step"].get("poisson", 0.0) + roof["phase_ms_per_step"].get("deposit_rho", 0.0)
    roof["poisson"] = {"ms_per_step": solve_ms, "dram_bytes_per_step": profile_figure("dram_bytes_per_solve_step",
                                                                                     cfg["name"])}
    # the ALU ceiling beside it: the push's FP32 arithmetic against the measured
    # FMA throughput of this GPU (the measured peaks hold no CUDA-core figure)
    try:
        fma_tflops = apic.probe_fp32_fma()
        alu = FLOPS_PER_PARTICLE_STEP * n_avg / (push_ms / 1e3) / 1e12
        roof["alu"] = {"flops_per_particle_step": FLOPS_PER_PARTICLE_STEP, "achieved": alu,
                       "peak": fma_tflops, "unit": "TFLOP/s", "frac": alu / fma_tflops,
                       "peak_source": "measured (apic_probe_fp32_fma)"}
    except Exception as e:  # the probe is a side figure: its failure leaves the line intact
        roof["alu"] = {"unavailable": str(e)}

    # end to end through the public API: initial state uploaded from pinned host
    # memory, then per step apic_step + apic_tallies (bins, counts, history row)
    e2e = None
    if not args.no_e2e and rank == 0 and len(cfgs) == 1:
        states = [sim.particles(sp) for sp in range(len(cfg["species"]))]
        pinned = []
        for stt in states:
            pt = torch.empty(stt.shape, dtype=torch.float64, pin_memory=True)
            pt.numpy()[:] = stt
            pinned.append(pt)
        cfg2 = dict(cfg, history_cap=64)
        sim.close()
        del sim
        torch.cuda.synchronize()
        sim2 = apic.Sim(cfg2)
        if tuned is not None:  # the schedule measured above, applied without measuring again
            sim2.set_schedule(tiles["sort_interval"], tiles["win_rows"], tiles["chunk_group"], tiles["chunk_items"])
        ke = min(args.steps, 1000)  # the timed run's steps (the upload amortised over as many)
        h2d = sum(p.numel() * 8 for p in pinned)
        barrier()
        t0 = time.perf_counter()
        for sp in range(len(pinned)):
            sim2.add_particles(sp, pinned[sp].numpy())
        adv2 = 0.0
        d2h = 0
        for k in range(ke):
            sim2.step(1)
            tt2 = sim2.tallies(history=True)
            adv2 += tt2["history"][-1, 7] + tt2["history"][-1, 8] if k < ke - 1 else 0.0
            d2h = tt2["bins"].nbytes + tt2["history"][-1:].nbytes + 12 * 8
        barrier()
        t1 = time.perf_counter()
        adv2 += float(sum(s.shape[0] for s in states))
        e2e = {"value": adv2 / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d // ke, "d2h_bytes_per_step": d2h,
               "steps": ke, "note": "initial state uploaded once from pinned host memory inside the timed region"}
        sim2.close()
    else:
        sim.close()

    cpu = None
    perr = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        oc = oracle_workload(cfg)
        n, k, kw = 1_000_000, 20, 2  # about 10-15 s of work per core
        val, secs = run_oracle(cfg, n, k, kw, 1)
        cores = host_cores()
        val_all, secs_all = run_oracle(cfg, n, k, kw, cores) if cores > 1 else (val, secs)
        cpu = {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(), "nproc": cores,
               "sample": "%d untimed + %d timed full steps of the same workload on %dx%d cells with %.0e "
                         "macro-particles per species (FP64, 1 thread)" % (kw, k, oc["n1"], oc["n2"], n),
               "seconds": secs,
               "all_cores": {"value": val_all, "unit": UNIT, "cores": cores, "seconds": secs_all,
                             "sample": "%d independent replicas of that sample in spawned processes, one per host "
                                       "core" % cores}}
        if len(cfgs) == 1:
            perr = precision_error(apic, cfg)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["name"] if len(cfgs) == 1 else "batched_48_instances" + (" (first %d)" % len(cfgs) if args.instances else ""),
                       "instances": len(cfgs), "alpha": cfg["alpha"], "a": 2 * cfg["alpha"], "B": cfg["B"],
                       "grid_cells": [cfg["n1"], cfg["n2"]],
                       "particles_per_species": [c["species"][0]["n_init"] for c in cfgs] if len(cfgs) > 1
                       else cfg["species"][0]["n_init"],
                       "poisson_tol": cfg["poisson_tol"],
                       "precision": "FP32 particles; Poisson: " + st["solver"],
                       "l2": "inputs larger than L2 (particle state %.0f MB)" % (
                           sum(len(c["species"]) * c["species"][0]["n_init"] for c in cfgs) * 20 / 1e6),
                       "electrons": "Boltzmann, n_e = exp(phi), Newton" if cfg.get("boltzmann") else "particles",
                       "grain": "isolated (floating potential)" if cfg.get("floating") else "fixed potential",
                       "dt": cfg["dt"],
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "sort_interval": tiles["sort_interval"], "autotuned": tuned is not None,
                       "push_window_rows": tiles["win_rows"], "push_chunk_group": tiles["chunk_group"],
                       "push_chunk_particles": 256 * tiles["chunk_items"]},
            "roofline": roof, "cpu_baseline": cpu, "error_vs_fp64_oracle": perr, "e2e": e2e,
            "gpu_launches": int(launches),
            "poisson_loop_iters": int(loop_iters), "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
