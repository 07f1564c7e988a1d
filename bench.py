"""Throughput of the 2D3V Weibel PIC step on GB300, one JSON line on stdout.

Workload (default): 1024 x 1024 cells, 64 particles per cell per species (134,217,728
particles), gamma = 3 beam (nb = 0.1) with T_perp = 0.1, background T = 0.001 with Krook
nu = 0.1, dx = 0.1, dt = 0.05; synthetic seeded load.  A step is the whole hot path: fused
gather/Boris/drag/move/Esirkepov deposit, Yee update, step finalisation, and the counting sort
every 8 steps.

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
BYTES_PER_CELL = 64


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


def build_workload(args, rank):
    import pic_inputs
    return pic_inputs.warm_beam_krook_2d(n=args.n, ppc=args.ppc, seed=2 + 1000 * rank)


def cpu_baseline(args, seconds=15.0):
    """The oracle as it is, single-threaded, on a 128 x 128 crop of the same physics."""
    import oracle
    import pic_inputs
    wl = pic_inputs.warm_beam_krook_2d(n=128, ppc=args.ppc, seed=2)
    sim = oracle.Simulation.from_workload(wl)
    sim.step(1, record=False)   # warm-up (page-in)
    t0 = time.perf_counter()
    steps = 0
    while True:
        sim.step(1, record=True)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    v = wl.nparticles * steps / el
    return {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"128x128 crop, {args.ppc} ppc/species ({wl.nparticles} particles), "
                      f"{steps} steps in {el:.1f} s, FP64 single-threaded C"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(args, seconds=max(5.0, 3.0 * args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"warm_beam_krook_2d_{args.n}x{args.n}_ppc{args.ppc}",
                       "oracle_sample": "128x128 crop"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": cb["sample"],
                             "value": cb["value"], "unit": METRIC},
            "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_0808_4078_gb300 as pic

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    wl = build_workload(args, rank)
    npart = wl.nparticles
    ncell = wl.ncell
    cap = [s.n for s in wl.species]
    eng = pic.Engine(2, wl.nx, wl.ny, dx=wl.dx, dt=wl.dt, capacity=cap, sort_interval=args.sort,
                     diag_interval=args.diag, diag_capacity=4096, flags=pic.PIC_FLAG_PROFILE,
                     device=f"cuda:{local_rank}")
    stream = eng.stream
    # ---------------- end to end through the public API from host buffers
    host = []
    for s in wl.species:
        host.append((torch.from_numpy(s.cell).pin_memory(), torch.from_numpy(s.offset).pin_memory(),
                     torch.from_numpy(s.u).pin_memory()))
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
    e2e_local = npart * args.steps / e2e_s

    # ---------------- device-resident timing
    eng.step(args.warmup)
    eng.sync()
    eng.kernel_times()            # drain warm-up timings
    base_times = eng.kernel_times()
    l0 = eng.launch_count()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    with Clocks(local_rank) as clk:
        start.record(stream)
        eng.step(args.steps)
        stop.record(stream)
        stop.synchronize()
    barrier()
    ms = start.elapsed_time(stop)
    launches = eng.launch_count() - l0
    times = eng.kernel_times()
    push_n = times["push_deposit"][0] - base_times["push_deposit"][0]
    push_ms = times["push_deposit"][1] - base_times["push_deposit"][1]
    phase = {k: (times[k][1] - base_times[k][1]) / max(1, args.steps) for k in times}

    t_max = ms
    e2e_max = e2e_s
    if dist is not None:
        tt = torch.tensor([ms, e2e_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max, e2e_max = float(tt[0]), float(tt[1])

    if rank == 0:
        peak, peak_kind = _peaks()
        alg_bytes = npart * BYTES_PER_PARTICLE_2D + ncell * BYTES_PER_CELL
        push_avg_s = push_ms / max(1, push_n) / 1e3
        achieved = alg_bytes / push_avg_s / 1e9
        value = world * npart * args.steps / (t_max / 1e3)
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "grid": [wl.nx, wl.ny], "ppc_per_species": args.ppc,
                       "particles_per_gpu": npart, "sort_interval": args.sort,
                       "diag_interval": args.diag, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (particles 3.2 GB/GPU), no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "push_deposit", "peak_kind": peak_kind,
                         "alg_bytes_per_launch": alg_bytes,
                         "mean_launch_ms": push_avg_s * 1e3},
            "phase_ms_per_step": phase,
            "e2e": {"value": world * npart * args.steps / e2e_max, "unit": METRIC,
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    eng.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--ppc", type=int, default=64)
    ap.add_argument("--sort", type=int, default=8)
    ap.add_argument("--diag", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
