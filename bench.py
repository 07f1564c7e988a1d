"""Throughput of the 2D3V Weibel PIC step on GB300, one JSON line on stdout.

Workload (default): 1024 x 1024 cells, 64 particles per cell per species (134,217,728
particles), gamma = 3 beam (nb = 0.1) with T_perp = 0.1, background T = 0.001 with Krook
nu = 0.1, dx = 0.1, dt = 0.05; synthetic seeded load.  A step is the whole hot path: fused
gather/Boris/drag/move/Esirkepov deposit, Yee update, step finalisation, and the counting sort
every 8 steps.  Before the timed region the autotuner times every variant of the 2D particle
kernel on the run (config.tile reports its pick; --no-autotune or --tile/--ctas skip it).

  value     particle-steps/s with the particles resident in HBM (CUDA events on the engine
            stream, after warm-up; particle data >> L2, so no flush is needed)
  e2e       the same metric through the public API from HOST buffers: H2D load of the
            particles, the K steps, and the D2H read of the diagnostics, all timed
  roofline  push+deposit kernel: algorithmic bytes (48 B/particle + 64 B/cell per step) over
            its mean CUDA-event duration, against the measured HBM copy bandwidth
  cpu_baseline  the FP64 oracle on the host cores on a bounded sample (128 x 128 crop)

With --gpus N under torchrun each rank runs an independent replica (the single run does not
shard); value is the sum over ranks of particle-steps over the slowest rank's time.
--impl reference times the oracle on this machine's host cores instead.
Other workloads (--workload):
  hot3d  256 x 256 x 512 cells 3D3V, 8 particles per cell per species (536,870,912 particles),
         beam T_perp = 0.2, cold collisionless background; roofline basis 56 B/particle + 64 B/cell
  scan   the batched temperature / collision-rate scan: 256 independent 2D runs, nx and ny each
         from {128, 192, 256, 384, 512}, 32 particles per cell per species, beam T_perp ~ U[0,1],
         background Krook nu from {0, 0.01, 0.1, 1}; all runs stepped by one set of launches
         (one CUDA graph per sort interval).  The line also carries the same runs stepped as
         separate engines, one after the other ("per_run"), the unbatched baseline.
  closure  the learned-closure path: moment recorder on the 3D hot-beam state, network inference
         on 2^20 samples per call (value = samples/s, roofline on the tensor-core forward
         kernel) and a full-batch training step
  hybrid the quasi-neutral hybrid model: 1024 x 1024 nodes, 16 beam particles per cell
         (16,777,216), T_perp = 0.1, nu = 0.1; a step is the beam push/deposit, the variable-
         density field solve (CG in a CUDA graph while node) and the update, with a counting
         sort every 16 steps; roofline basis 44 B/particle + 24 B/node on the push
--j-filter 1 adds the binomial current filter before the E update (warm2d, hot3d).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
BYTES_PER_PARTICLE_2D = 48
BYTES_PER_PARTICLE_3D = 56
BYTES_PER_CELL = 64
# DRAM bytes per particle of the push kernels (dram__bytes_read.sum + dram__bytes_write.sum of
# one ncu capture of a small case, divided by its particles; the capture commands are in the
# profile summaries named here).  They describe the kernels as captured: re-capture after
# changing a kernel.
NCU_TRAFFIC_PER_PARTICLE = {
    2: (57.72, "profiles/push2d_warm_beam_krook_2d.md (256x256, 64 ppc per species)"),
    3: (59.06, "profiles/push3d_hot_beam_3d.md (128x128x64, 8 ppc per species)"),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _workers():
    return max(1, min(16, os.cpu_count() or 1))


def workload_name(args):
    if args.workload == "hybrid":
        return f"hybrid_beam_2d_{args.n}x{args.n}_ppc{args.ppc}"
    if args.workload == "closure":
        return f"closure_mlp_9x64x64x1_{args.samples}samples"
    if args.workload == "warm2d":
        return f"warm_beam_krook_2d_{args.n}x{args.n}_ppc{args.ppc}"
    if args.workload == "hot3d":
        nx, ny, nz = args.grid3
        return f"hot_beam_3d_{nx}x{ny}x{nz}_ppc{args.ppc}"
    return f"scan_{args.runs}runs_2d_ppc{args.ppc}"


def build_load(args, rank):
    """Particles of this rank's replica, drawn in parallel into shared memory."""
    import pic_inputs as pi
    if args.workload == "warm2d":
        return pi.weibel_load_parallel(ndim=2, nx=args.n, ny=args.n, ppc=args.ppc, T_perp_beam=0.1,
                                       T_bg=0.001, nu=0.1, seed=2 + 1000 * rank, workers=_workers(),
                                       name=workload_name(args))
    nx, ny, nz = args.grid3
    return pi.weibel_load_parallel(ndim=3, nx=nx, ny=ny, nz=nz, ppc=args.ppc, T_perp_beam=0.2,
                                   seed=3 + 1000 * rank, workers=_workers(), name=workload_name(args))


def _oracle_sample(args):
    """The bounded oracle sample of each workload: (workload, description)."""
    import pic_inputs as pi
    if args.workload == "warm2d":
        return pi.warm_beam_krook_2d(n=128, ppc=args.ppc, seed=2), "128x128 crop"
    if args.workload == "hot3d":
        return pi.hot_beam_3d(nx=32, ny=32, nz=64, ppc=args.ppc, seed=3), "32x32x64 crop"
    return (pi.weibel_load(ndim=2, nx=128, ny=128, ppc=args.ppc, T_perp_beam=0.5, T_bg=0.001,
                           nu=0.1, seed=1000), "one 128x128 run of the scan recipe")


def cpu_baseline_closure(args, seconds=15.0):
    """The FP64 oracle network (numpy) on 65536 samples, repeated for about `seconds`."""
    from oracle import mlp
    n = 65536
    rng = np.random.default_rng(5)
    x = rng.normal(size=(n, 9))
    p = mlp.init_params(1)
    mu, sd = np.zeros(9), np.ones(9)
    mlp.forward(p, x, mu, sd)
    t0 = time.perf_counter()
    reps = 0
    while True:
        mlp.forward(p, x, mu, sd)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": n * reps / el, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"{n} samples x {reps} forward passes in {el:.1f} s, FP64 numpy (BLAS threads)"}


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _time_oracle(wl, threads, seconds, steps=None, warmup=1):
    """Steps of the PIC oracle on wl: `warmup` untimed, then `steps` (or as many as fit in
    `seconds`); returns (particle-steps/s, steps, seconds)."""
    import oracle
    sim = oracle.Simulation.from_workload(wl, threads=threads)
    sim.step(warmup, record=False)
    t0 = time.perf_counter()
    n = 0
    while True:
        sim.step(1, record=True)
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= seconds):
            break
    return wl.nparticles * n / el, n, el


def cpu_baseline(args, seconds=15.0):
    """The oracle as it is on a bounded crop of the same physics: the all-core build (OpenMP over
    particles, per-thread current arrays) on every host core, and the single-threaded build."""
    if args.workload == "closure":
        return cpu_baseline_closure(args, seconds)
    if args.workload == "hybrid":
        return cpu_baseline_hybrid(args, seconds)
    cores = _host_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    wl, what = _oracle_sample(args)
    v1, n1, e1 = _time_oracle(wl, False, seconds / 2)
    va, na, ea = _time_oracle(wl, True, seconds / 2)
    return {"value": va, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{what}, {args.ppc} ppc/species ({wl.nparticles} particles), {na} steps in "
                      f"{ea:.1f} s, FP64 C, OpenMP on {cores} cores (-O3 -fopenmp)",
            "single_core": {"value": v1, "unit": METRIC, "cores": 1,
                            "sample": f"{n1} steps in {e1:.1f} s, FP64 C, one thread (-O2)"}}


def units_per_step(args):
    """Units of the metric one step of the workload processes (particles, or samples per call)."""
    if args.workload == "closure":
        return args.samples
    if args.workload == "hybrid":
        return args.n * args.n * args.ppc
    if args.workload == "warm2d":
        return 2 * args.n * args.n * args.ppc
    if args.workload == "hot3d":
        nx, ny, nz = args.grid3
        return 2 * nx * ny * nz * args.ppc
    import pic_inputs as pi
    return sum(2 * nx * ny * args.ppc for nx, ny, _, _ in pi.scan_table(args.runs))


def run_reference(args, rank, world):
    """The oracle on this machine's host cores, as it stands: W warm-up and K timed steps of its
    bounded sample of the workload (all cores; the closure and hybrid workloads time their
    numpy oracles for about 3 s per step)."""
    if rank != 0:
        return
    metric = "closure inference samples/s" if args.workload == "closure" else METRIC
    units = units_per_step(args)
    if args.workload in ("closure", "hybrid"):
        cb = cpu_baseline(args, seconds=max(5.0, 3.0 * args.steps))
        value, unit, cores, sample = cb["value"], cb["unit"], cb["cores"], cb["sample"]
        ms = None
    else:
        cores = _host_cores()
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        wl, what = _oracle_sample(args)
        value, n, el = _time_oracle(wl, True, 0.0, steps=args.steps, warmup=args.warmup)
        unit = METRIC
        ms = el / n * 1e3
        sample = (f"{what}, {args.ppc} ppc/species ({wl.nparticles} particles), {n} steps in {el:.1f} s "
                  f"after {args.warmup} warm-up, FP64 C, OpenMP on {cores} cores")
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # one step of the bounded sample, as timed (the full workload's step at the same
            # rate is given separately)
            "ms_per_step": ms if ms is not None else units / value * 1e3,
            "ms_per_full_step_extrapolated": units / value * 1e3, "units_per_step": units,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "oracle_sample": sample},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample,
                             "value": value, "unit": unit},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _init_dist(world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        return dist
    return None


def _max_over_ranks(dist, vals, device="cuda"):
    """Element-wise maximum over ranks (the slowest rank's times); identity without a group."""
    if dist is None:
        return vals
    import torch
    t = torch.tensor(vals, device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def _roofline(alg_bytes, push_n, push_ms, ndim=None, npart=None):
    peak, peak_kind = _peaks()
    push_avg_s = push_ms / max(1, push_n) / 1e3
    achieved = alg_bytes / push_avg_s / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": None, "kernel": "push_deposit",
           "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes,
           "mean_launch_ms": push_avg_s * 1e3}
    if ndim in NCU_TRAFFIC_PER_PARTICLE and npart:
        per, src = NCU_TRAFFIC_PER_PARTICLE[ndim]
        out["traffic"] = per * npart
        out["traffic_source"] = f"ncu DRAM bytes of a small case scaled by particles: {src}"
    return out


def _timed_steps(eng, steps, warmup, barrier, local_rank):
    """Warm up, then K steps between CUDA events on the engine stream, with clock sampling."""
    import torch
    eng.step(warmup)
    eng.sync()
    eng.kernel_times()            # drain warm-up timings
    base = eng.kernel_times()
    l0 = eng.launch_count()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    with Clocks(local_rank) as clk:
        start.record(eng.stream)
        eng.step(steps)
        stop.record(eng.stream)
        stop.synchronize()
    barrier()
    times = eng.kernel_times()
    delta = {k: (times[k][0] - base[k][0], times[k][1] - base[k][1]) for k in times}
    return start.elapsed_time(stop), eng.launch_count() - l0, delta, clk.summary()


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_0808_4078_gb300 as pic

    dist = _init_dist(world, local_rank)

    def barrier():
        if dist is not None:
            dist.barrier()

    L = build_load(args, rank)
    wl = L.workload
    npart = wl.nparticles
    ncell = wl.ncell
    cap = [s.n for s in wl.species]
    eng = pic.Engine(wl.ndim, wl.nx, wl.ny, wl.nz, dx=wl.dx, dt=wl.dt, capacity=cap,
                     sort_interval=args.sort, diag_interval=args.diag, diag_capacity=4096,
                     flags=pic.PIC_FLAG_PROFILE, device=f"cuda:{local_rank}", j_filter=args.j_filter,
                     tile=args.tile if wl.ndim == 2 else (0, 0), ctas_per_sm=args.ctas)
    # ---------------- end to end through the public API from (pinned) host buffers
    host = []
    for s in wl.species:
        host.append((torch.from_numpy(s.cell).pin_memory(), torch.from_numpy(s.offset).pin_memory(),
                     torch.from_numpy(s.u).pin_memory()))
    L.close()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for i, s in enumerate(wl.species):
        c, o, u = host[i]
        eng.load_species(i, s.q, s.m, s.w, s.nu, c.numpy(), o.numpy(), u.numpy())
    eng.step(args.steps)
    recs = eng.diag()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = sum(s.n * (4 + 4 * wl.ndim + 12) for s in wl.species)
    d2h = len(recs) * 128
    del host

    # ---------------- autotuner (its steps are steps of the run, outside the timed region)
    tune = None
    if wl.ndim == 2 and tuple(args.tile) == (0, 0) and args.ctas == 0 and not args.no_autotune:
        tune = eng.autotune(16)
    # ---------------- device-resident timing
    ms, launches, delta, clocks = _timed_steps(eng, args.steps, args.warmup, barrier, local_rank)
    phase = {k: v[1] / max(1, args.steps) for k, v in delta.items()}
    t_max, e2e_max = _max_over_ranks(dist, [ms, e2e_s])

    if rank == 0:
        bpp = BYTES_PER_PARTICLE_2D if wl.ndim == 2 else BYTES_PER_PARTICLE_3D
        alg_bytes = npart * bpp + ncell * BYTES_PER_CELL
        value = world * npart * args.steps / (t_max / 1e3)
        grid = [wl.nx, wl.ny] + ([wl.nz] if wl.ndim == 3 else [])
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "grid": grid, "ppc_per_species": args.ppc,
                       "particles_per_gpu": npart, "sort_interval": args.sort,
                       "diag_interval": args.diag, "parallelism": f"replicas{world}",
                       "j_filter": args.j_filter, "tile": list(eng.tile_config()),
                       "l2": f"inputs larger than L2 (particles {npart * (bpp // 2) / 1e9:.1f} GB/GPU), no flush"},
            "roofline": _roofline(alg_bytes, *delta["push_deposit"], ndim=wl.ndim, npart=npart),
            "phase_ms_per_step": phase,
            "e2e": {"value": world * npart * args.steps / e2e_max, "unit": METRIC,
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if tune is not None:
            line["autotune"] = [{"tile": [t[0], t[1]], "ctas_per_sm": t[2], "ms_per_step": t[3]} for t in tune]
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    eng.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched scan
def _scan_run(job):
    """Worker: the particles of run r of the scan table (spawned process)."""
    import pic_inputs as pi
    return pi.scan_run(job)


def _partition(table, world):
    """Greedy longest-first assignment of runs to ranks by cell count."""
    order = sorted(range(len(table)), key=lambda r: -table[r][0] * table[r][1])
    load = [0] * world
    out = [[] for _ in range(world)]
    for r in order:
        k = min(range(world), key=lambda i: load[i])
        out[k].append(r)
        load[k] += table[r][0] * table[r][1]
    return [sorted(o) for o in out]


def run_scan(args, rank, world, local_rank):
    import multiprocessing as mp
    import torch
    import pic_inputs as pi
    import paper_0808_4078_gb300 as pic

    dist = _init_dist(world, local_rank)

    def barrier():
        if dist is not None:
            dist.barrier()

    table = pi.scan_table(args.runs)
    mine = _partition(table, world)[rank]
    ppc = args.ppc
    cc = 2 * ppc                      # slots per cell: twice the mean (the smallest allowed)
    runs = [(table[r][0], table[r][1], 1, (table[r][0] * table[r][1] * ppc,) * 2) for r in mine]
    npart = sum(2 * nx * ny * ppc for nx, ny, _, _ in runs)
    ncell = sum(nx * ny for nx, ny, _, _ in runs)
    kw = dict(dx=0.1, dt=0.05, sort_interval=args.sort, diag_interval=args.diag,
              diag_capacity=1024, flags=pic.PIC_FLAG_PROFILE, cell_capacity=(cc, cc),
              device=f"cuda:{local_rank}")
    eng = pic.Engine(2, nspecies=2, runs=runs, **kw)
    jobs = [(r, table[r], ppc) for r in mine]
    idx = {r: k for k, r in enumerate(mine)}
    # end to end: the H2D loads (timed per call, generation excluded), K steps, the D2H reads
    load_s = 0.0
    with mp.get_context("spawn").Pool(_workers()) as pool:
        for r, wl in pool.imap_unordered(_scan_run, jobs):
            t0 = time.perf_counter()
            for i, s in enumerate(wl.species):
                eng.load_species(i, s.q, s.m, s.w, s.nu, s.cell, s.offset, s.u, run=idx[r])
            load_s += time.perf_counter() - t0
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    eng.step(args.steps)
    recs = [eng.diag(run=k) for k in range(len(mine))]
    torch.cuda.synchronize()
    e2e_s = load_s + time.perf_counter() - t0
    h2d = npart * 20
    d2h = sum(len(x) for x in recs) * 128

    ms, launches, delta, clocks = _timed_steps(eng, args.steps, args.warmup, barrier, local_rank)
    phase = {k: v[1] / max(1, args.steps) for k, v in delta.items()}
    eng.close()
    del eng
    torch.cuda.empty_cache()

    # theory line: Eq. (12) growth rate per run, c_s^2 = 3 T_perp / gamma_b^2 (transverse velocity
    # variance of the load), beta0 = sqrt(8) / 3, n_b = 0.1, the run's nu
    gb = 3.0
    params = [(3.0 * table[r][2] / gb ** 2, np.sqrt(gb * gb - 1) / gb, 0.1, table[r][3]) for r in mine]
    pic.dispersion_growth(params, 0.05, 10.0, 2000)              # load the module
    t0 = time.perf_counter()
    th_gamma, th_k = pic.dispersion_growth(params, 0.05, 10.0, 2000)
    theory_ms = (time.perf_counter() - t0) * 1e3

    # the same runs as separate engines, stepped one after the other
    per_run_ms = 0.0
    per_run_launches = 0
    if not args.no_per_run:
        with mp.get_context("spawn").Pool(_workers()) as pool:
            for r, wl in pool.imap_unordered(_scan_run, jobs):
                e1 = pic.Engine.from_workload(wl, **{k: v for k, v in kw.items() if k not in ("dx", "dt")})
                m1, l1, _, _ = _timed_steps(e1, args.steps, args.warmup, lambda: None, local_rank)
                per_run_ms += m1
                per_run_launches += l1
                e1.close()
    t_max, e2e_max, pr_max = _max_over_ranks(dist, [ms, e2e_s, per_run_ms])
    if dist is not None:
        import torch.distributed as tdist
        t = torch.tensor([float(npart)], device="cuda", dtype=torch.float64)
        tdist.all_reduce(t)
        tot_part = float(t[0])
    else:
        tot_part = float(npart)
    if rank == 0:
        alg_bytes = npart * BYTES_PER_PARTICLE_2D + ncell * BYTES_PER_CELL
        line = {
            "metric": METRIC, "value": tot_part * args.steps / (t_max / 1e3), "unit": METRIC,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args), "runs": args.runs, "ppc_per_species": ppc,
                       "particles": int(tot_part), "cells_rank0": ncell,
                       "cell_capacity": cc, "sort_interval": args.sort, "diag_interval": args.diag,
                       "parallelism": f"runs split over {world} GPU(s), greedy by cells",
                       "l2": "inputs larger than L2, no flush"},
            "roofline": _roofline(alg_bytes, *delta["push_deposit"]),
            "phase_ms_per_step": phase,
            "e2e": {"value": tot_part * args.steps / e2e_max, "unit": METRIC,
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        line["theory"] = {"what": "Eq. (12) max growth rate over k in [0.05, 10] (2000 points) per run",
                          "ms_with_copies": theory_ms, "runs": len(mine),
                          "gamma_range": [float(th_gamma.min()), float(th_gamma.max())],
                          "unstable_runs": int((th_gamma > 1e-6).sum())}
        if not args.no_per_run:
            line["per_run"] = {"value": tot_part * args.steps / (pr_max / 1e3), "unit": METRIC,
                               "ms_per_step": pr_max / args.steps, "gpu_launches": per_run_launches,
                               "what": "the same runs as separate engines, stepped one after the other"}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- closure (recorder + network)
def _closure_params(seed):
    """Seeded network parameters, uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), library order."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, 64 * 9) / 3.0, rng.uniform(-1, 1, 64) / 3.0,
             rng.uniform(-1, 1, 64 * 64) / 8.0, rng.uniform(-1, 1, 64) / 8.0,
             rng.uniform(-1, 1, 64) / 8.0, np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)



def run_closure(args, rank, world, local_rank):
    """Moment recorder on a 3D hot-beam state, network inference on 2^20 samples per call and a
    full-batch training step on 2^20 samples.  value = inference samples/s."""
    import torch
    import paper_0808_4078_gb300 as pic

    dist = _init_dist(world, local_rank)
    dev = torch.device("cuda", local_rank)

    def ev_time(fn, stream, reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    # recorder
    L = build_load(argparse.Namespace(**{**vars(args), "workload": "hot3d", "ppc": args.rec_ppc}), rank)
    wl = L.workload
    eng = pic.Engine(3, wl.nx, wl.ny, wl.nz, dx=wl.dx, dt=wl.dt, capacity=[sp.n for sp in wl.species],
                     sort_interval=args.sort, diag_interval=0, flags=0, device=f"cuda:{local_rank}")
    for i, sp in enumerate(wl.species):
        eng.load_species(i, sp.q, sp.m, sp.w, sp.nu, sp.cell, sp.offset, sp.u)
    npart, ncell = wl.nparticles, wl.ncell
    L.close()
    eng.step(4)
    import ctypes
    nbytes = ctypes.c_size_t(0)
    pic._check(pic.lib().pic_record_moments_scratch_bytes(eng._ctx, 0, 4, 4, ctypes.byref(nbytes)), eng._ctx)
    nc = (wl.nx // 4) * (wl.ny // 4)
    out = torch.empty((pic.PIC_MOM_ROWS, nc), dtype=torch.float32, device=dev)
    scratch = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
    n64 = ctypes.c_int64(0)

    def record():
        pic._check(pic.lib().pic_record_moments(eng._ctx, 0, 4, 4, ctypes.c_void_p(out.data_ptr()), out.numel(),
                                                ctypes.c_void_p(scratch.data_ptr()), nbytes.value,
                                                ctypes.byref(n64)), eng._ctx)
    rec_ms = ev_time(record, eng.stream, max(3, args.steps // 4))
    eng.close()
    del eng, scratch
    torch.cuda.empty_cache()

    # network
    n = args.samples
    g = torch.Generator(device=dev).manual_seed(5)
    x = torch.randn((9, n), generator=g, device=dev, dtype=torch.float32)
    t = torch.randn((n,), generator=g, device=dev, dtype=torch.float32)
    net = pic.ClosureNet(_closure_params(1), [0.0] * 9, [1.0] * 9, device=dev)
    y = torch.empty(n, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    lib = pic.lib()

    def infer():
        pic._check(lib.pic_mlp_forward(ctypes.c_void_p(net.params.data_ptr()), ctypes.byref(net.norm),
                                       ctypes.c_void_p(x.data_ptr()), n, n, ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(net.stream.cuda_stream)))
    with Clocks(local_rank) as clk:
        inf_ms = ev_time(infer, net.stream, args.steps)
    pic._check(lib.pic_mlp_status(1))
    step = [0]

    def train():
        step[0] += 1
        pic._check(lib.pic_mlp_train_step(ctypes.c_void_p(net.params.data_ptr()), ctypes.c_void_p(net.m.data_ptr()),
                                          ctypes.c_void_p(net.v.data_ptr()), step[0], 1e-4, ctypes.byref(net.norm),
                                          ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(t.data_ptr()), n,
                                          None, ctypes.c_void_p(net._scratch.data_ptr()), net._scratch.numel(),
                                          ctypes.c_void_p(net.stream.cuda_stream)))
    train_ms = ev_time(train, net.stream, max(3, args.steps // 4))
    pic._check(lib.pic_mlp_status(1))

    # end to end: host features -> device, inference, host result
    xh = x.cpu().pin_memory()
    yh = torch.empty(n, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(net.stream):
            x.copy_(xh, non_blocking=True)
            infer()
            yh.copy_(y, non_blocking=True)
    net.stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps

    if rank == 0:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except Exception:
            pass
        bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
        flops = 2.0 * n * (16 * 64 + 64 * 64)          # the two tensor-core products (K padded to 16)
        tflops = flops / (inf_ms / 1e3) / 1e12
        rec_bytes = npart * 36 + ncell * 32           # pass 1 reads u, pass 2 o + u; field columns
        line = {
            "metric": "closure inference samples/s", "value": n / (inf_ms / 1e3), "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": inf_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": f"closure_mlp_9x64x64x1_{n}samples", "samples_per_call": n,
                       "recorder_state": f"hot_beam_3d_{wl.nx}x{wl.ny}x{wl.nz}_ppc{args.rec_ppc}",
                       "l2": "features 37.7 MB < L2: inference inputs may be L2-resident between calls"},
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": tflops / bf16_peak, "traffic": 37.8e6 * n / (1 << 20),
                         "traffic_source": "ncu DRAM bytes, profiles/mlp_forward_closure.md",
                         "kernel": "mlp_forward",
                         "peak_kind": "measured" if "bf16_tflops" in peaks else "fallback",
                         "flops_per_launch": flops, "mean_launch_ms": inf_ms},
            "recorder": {"ms_per_snapshot": rec_ms, "coarse_cells": nc, "particles": npart,
                         "alg_bytes": rec_bytes, "achieved_gbs": rec_bytes / (rec_ms / 1e3) / 1e9},
            "train": {"ms_per_step": train_ms, "samples_per_s": n / (train_ms / 1e3)},
            "e2e": {"value": n / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": 36 * n,
                    "d2h_bytes_per_step": 4 * n},
            "gpu_launches": 1,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- hybrid model
HYB_BYTES_PER_PARTICLE = 44     # read cell, ox, oy, ux, uy, P (24 B); write cell, ox, oy, ux, uy (20 B)
HYB_BYTES_PER_NODE = 24         # read the FP32 (a, beta_p) pair once; J and N (int64) written once
# DRAM bytes per particle of the hybrid push (ncu, 1024^2 nodes x 8 ppc, scaled by particles):
# profiles/hybrid_push_deposit_1024x1024.md
HYB_NCU_TRAFFIC_PER_PARTICLE = (226.725632e6 + 126.075904e6) / 8388608


def _hybrid_load(args, rank=0):
    import pic_inputs as pi
    return pi.hybrid_beam_load(nx=args.n, ny=args.n, ppc=args.ppc, seed=6 + 1000 * rank)


def cpu_baseline_hybrid(args, seconds=15.0):
    """The FP64 hybrid oracle (numpy + sparse LU) on a 128 x 128 crop of the same load."""
    import pic_inputs as pi
    from oracle import hybrid
    L = pi.hybrid_beam_load(nx=128, ny=128, ppc=args.ppc, seed=6)
    sim = hybrid.HybridSim(L.nx, L.ny, L.dx, L.dx, L.dt, n0=1.0, nu=L.nu, w=L.w)
    sim.load(L.X, L.Y, L.ux, L.uy, L.uz, L.beta_p0)
    sim.step(1)
    t0 = time.perf_counter()
    steps = 0
    while True:
        sim.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": L.n * steps / el, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"128x128 crop, {args.ppc} ppc ({L.n} particles), {steps} steps in {el:.1f} s, "
                      f"FP64 numpy + scipy sparse LU, single-threaded"}


def run_hybrid(args, rank, world, local_rank):
    """The quasi-neutral hybrid model: push/deposit, variable-density field solve, update.
    value = beam particle-steps/s; the roofline is taken on the push/deposit kernel."""
    import torch
    import paper_0808_4078_gb300 as pic

    dist = _init_dist(world, local_rank)

    def barrier():
        if dist is not None:
            dist.barrier()

    L = _hybrid_load(args, rank)
    n, nx, ny = L.n, L.nx, L.ny
    nc = nx * ny

    def make(flags):
        return pic.HybridEngine(nx, ny, L.dx, L.dx, L.dt, 1.0, L.nu, L.w, n, max_iter=args.cg_iter,
                                flags=flags, sort_interval=args.hybrid_sort, device=f"cuda:{local_rank}")

    # ---------------- end to end through the public API from host buffers
    eng = make(0)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    eng.load(L.X, L.Y, L.ux, L.uy, L.uz, L.beta_p0)
    eng.step(args.steps)
    en = eng.energies()
    e2e_s = time.perf_counter() - t0
    h2d = n * 24 + nc * 16              # FP32 cell/offsets/momenta and the (a, beta_p) pair
    d2h = 3 * 8
    assert np.isfinite(en).all()

    # ---------------- device-resident timing of the graph-replayed step
    eng.step(args.warmup)
    eng.sync()
    l0 = eng.launch_count()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    with Clocks(local_rank) as clk:
        start.record(eng.stream)
        eng.step(args.steps)
        stop.record(eng.stream)
        stop.synchronize()
    barrier()
    ms = start.elapsed_time(stop)
    launches = eng.launch_count() - l0
    st = eng.stats()
    eng.close()

    # ---------------- phase split (CUDA events per phase, direct launches)
    eng = make(pic.PIC_FLAG_PROFILE)
    eng.load(L.X, L.Y, L.ux, L.uy, L.uz, L.beta_p0)
    eng.step(args.warmup)
    base = eng.kernel_times()
    eng.step(args.steps)
    times = eng.kernel_times()
    eng.close()
    phase = {k: (times[k][1] - base[k][1]) / args.steps for k in times}
    t_max, e2e_max = _max_over_ranks(dist, [ms, e2e_s])

    if rank == 0:
        peak, peak_kind = _peaks()
        alg = n * HYB_BYTES_PER_PARTICLE + nc * HYB_BYTES_PER_NODE
        push_ms = phase["push_deposit"]
        achieved = alg / (push_ms / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": world * n * args.steps / (t_max / 1e3), "unit": METRIC,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"hybrid_beam_2d_{nx}x{ny}_ppc{args.ppc}", "grid": [nx, ny],
                       "ppc": args.ppc, "particles_per_gpu": n, "cg_max_iter": args.cg_iter,
                       "sort_interval": args.hybrid_sort or 16,
                       "parallelism": f"replicas{world}",
                       "l2": f"particles {n * 24 / 1e9:.2f} GB > L2, no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": HYB_NCU_TRAFFIC_PER_PARTICLE * n,
                         "traffic_source": "ncu DRAM bytes of the 8-ppc case scaled by particles: "
                                           "profiles/hybrid_push_deposit_1024x1024.md",
                         "kernel": "hybrid push_deposit",
                         "peak_kind": peak_kind, "alg_bytes_per_launch": alg,
                         "mean_launch_ms": push_ms},
            "phase_ms_per_step": phase,
            "solver": {"cg_iterations_per_step": st["cg_iterations"] / max(1, st["steps"]),
                       "unconverged_steps": st["unconverged_steps"]},
            "e2e": {"value": world * n * args.steps / e2e_max, "unit": METRIC,
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_hybrid(args)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="warm2d", choices=["warm2d", "hot3d", "scan", "closure", "hybrid"])
    ap.add_argument("--cg-iter", type=int, default=16, help="hybrid: conjugate-gradient iterations per step")
    ap.add_argument("--hybrid-sort", type=int, default=0, help="hybrid: steps between sorts by cell (0 = 16)")
    ap.add_argument("--j-filter", type=int, default=0, choices=[0, 1],
                    help="warm2d / hot3d: binomial current filter before the E update")
    ap.add_argument("--n", type=int, default=1024, help="2D grid side (warm2d)")
    ap.add_argument("--grid3", type=lambda t: tuple(int(x) for x in t.split(",")),
                    default=(256, 256, 512), help="3D grid nx,ny,nz (hot3d)")
    ap.add_argument("--runs", type=int, default=256, help="runs of the scan")
    ap.add_argument("--ppc", type=int, default=None,
                    help="particles per cell per species (default 64 / 8 / 32)")
    ap.add_argument("--sort", type=int, default=8)
    ap.add_argument("--tile", type=lambda t: tuple(int(x) for x in t.split("x")), default=(0, 0),
                    help="2D particle-kernel tile, e.g. 32x8 (0x0 = default)")
    ap.add_argument("--ctas", type=int, default=0, help="2D particle kernel: CTAs per SM (2, 3 or 4; 0 = default)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="2D: keep the default kernel variant instead of timing them all first")
    ap.add_argument("--diag", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-run", action="store_true", help="scan: skip the per-run baseline")
    ap.add_argument("--samples", type=int, default=1 << 20, help="closure: network samples per call")
    ap.add_argument("--rec-ppc", type=int, default=8, help="closure: particles per cell of the recorder state")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.ppc is None:
        args.ppc = {"warm2d": 64, "hot3d": 8, "scan": 32, "closure": 8, "hybrid": 16}[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "scan":
        run_scan(args, rank, world, local_rank)
    elif args.workload == "closure":
        run_closure(args, rank, world, local_rank)
    elif args.workload == "hybrid":
        run_hybrid(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
