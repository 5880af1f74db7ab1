#!/usr/bin/env python3
"""Benchmark of one suspension time step (MLUPS and HBM roofline fraction).

Default workload: D3Q19, 512^3 periodic box, 16000 spheres of radius 8 (25.6 % solid) at
seeded random positions, velocities N(0, 1e-3), density ratio 1.2, tau 0.6, body force
1e-6, FP32 arithmetic on FP32 deviation storage. A "step" is one full time step of the
method: fused stream + collide + boundary-site transfer over all sites, the per-particle
reduction, particle update and contacts, re-marking, and the internal-site imposition.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Multi-GPU runs are independent replicas (the path is not
decomposed across GPUs); value = sites x steps x ranks / max-over-ranks time.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1105_2904_gb300 import workloads as W  # noqa: E402

METRIC = "MLUPS"
UNIT = "MLUPS"


def config_defaults(argv):
    """Option defaults from a JSON file given as --config PATH (keys are the options' names with
    underscores; options given on the command line still win)."""
    pre = argparse.ArgumentParser(add_help=False)
    pre.add_argument("--config")
    known, _ = pre.parse_known_args(argv)
    if not known.config:
        return {}
    with open(known.config) as f:
        cfg = json.load(f)
    return {k: v for k, v in cfg.items() if k != "description"}


def parse(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    p = argparse.ArgumentParser()
    p.add_argument("--config", help="JSON file of option defaults (bench_configs/)")
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="d3q19_512",
                   choices=["d3q19_512", "d2q9_sedimentation", "d2q9_channel_disk", "ensemble_64", "closure"])
    p.add_argument("--closure-cells", type=int, nargs=2, default=[512, 64],
                   help="closure workload: training and held-out cells (8 spheres each)")
    p.add_argument("--closure-large-cells", type=int, default=0,
                   help="closure workload: also judge the trained network on this many held-out 128^3 "
                        "cells with 200 spheres of radius 3 against their 512^3 radius-12 twins")
    p.add_argument("--closure-large-train", type=int, default=0,
                   help="closure workload: also train a network on this many 128^3 / 200-sphere cells "
                        "and judge it on the held-out large cells")
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    p.add_argument("--edge", type=int, default=0, help="override the 3D box edge (same solid fraction)")
    p.add_argument("--sweep-shape", type=int, default=-1,
                   help="sweep kernel shape (lbm_set_sweep_shape): -1 automatic, 0 one-site, 16/32/64/128 two-site")
    p.add_argument("--streaming", default="pull", choices=["pull", "inplace"],
                   help="streaming scheme (lbm_set_streaming): pull (two buffers) or inplace (one buffer)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-patterns", action="store_true",
                   help="default workload: leave out the 16-bit storages, the batched ensemble and the "
                        "learned closure measured beside the headline line")
    p.add_argument("--pattern-closure-cells", type=int, nargs=2, default=[384, 48],
                   help="training and held-out cells of the closure measured beside the headline line")
    p.add_argument("--cpu-full", action="store_true",
                   help="also time the all-core oracle on the full-size 3D workload for 10 steps "
                        "(on by default for the default 512^3 workload)")
    p.add_argument("--no-cpu-full", action="store_true",
                   help="leave out the full-size oracle timing of the default workload (~2 minutes)")
    cfg = config_defaults(argv)
    unknown = sorted(set(cfg) - {a.dest for a in p._actions})
    if unknown:
        p.error("unknown keys in %s: %s" % (cfg and "--config", ", ".join(unknown)))
    p.set_defaults(**cfg)
    return p.parse_args(argv)


def workload(args):
    if args.workload == "d2q9_sedimentation":
        return W.sedimentation_2d()
    if args.workload == "d2q9_channel_disk":
        return W.channel_disk_2d()
    if args.edge:
        return W.suspension_3d_scaled(args.edge)
    return W.suspension_3d()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value):
    """Maximum of a float over all ranks (identity without a process group). Works with the
    nccl backend (tensor on the current CUDA device) and with gloo (CPU tensor)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value):
    """Sum of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_throughput(sites, steps, ms_local):
    """Whole-job MLUPS of independent ranks: each rank advanced its own `sites` sites by
    `steps` steps (replicas of one problem, or distinct cells of an ensemble); the job counts
    every rank's sites and its time is the slowest rank's."""
    ms = reduce_max(ms_local)
    return reduce_sum(sites) * steps / (ms / 1e3) / 1e6, ms


def source_sha():
    h = hashlib.sha256()
    for f in ("sweep.cuh", "sweep2.cuh", "common.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_1105_2904_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel_key):
    """ncu DRAM bytes per site of the sweep kernel, if taken on the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    rec = d.get(kernel_key)
    if not rec or rec.get("source_sha") != source_sha():
        return None
    return rec


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(wl, target_s=12.0, configs=()):
    """The FP64 oracle, as it stands (one host thread), on a bounded sample of the workload:
    the same suspension scaled to a smaller periodic box with the same solid fraction.
    configs: (precision, sweep shape, streaming) triples; for each, the CUDA path then runs the
    same sample for the same steps in that configuration, and its error against the oracle is
    returned beside the baseline: (baseline, [error per config])."""
    import oracle as O

    edge = 64 if wl.lattice == "D3Q19" else 256
    if wl.lattice == "D3Q19":
        s = W.suspension_3d_scaled(edge)
        c, r, d, v = s.particles()
        sim = O.OracleSim(O.D3Q19, edge, edge, edge, s.tau, body_force=s.body_force,
                          body_force_on_particles=s.body_force_on_particles)
        sample = "D3Q19 %d^3 periodic, %d spheres r=8 (same solid fraction)" % (edge, len(r))
    elif wl.sites <= 2 * edge * edge:
        # a small 2D workload is its own sample
        s = wl
        nx2, ny2 = wl.dims[0], wl.dims[1]
        c, r, d, v = wl.particles()
        sim = O.OracleSim(O.D2Q9, nx2, ny2, 1, wl.tau, body_force=wl.body_force, walls=wl.walls,
                          gravity=wl.gravity, gap=0.0)
        sample = "%s, the whole workload" % wl.name
    else:
        s = wl
        nx2, ny2 = edge, 2 * edge
        n = max(1, int(round(wl.n_particles * (edge * edge * 2) / wl.sites)))
        c, r = W.rsa_centers((edge, 2 * edge), n, wl.radius, seed=wl.seed, min_gap=wl.min_gap, walls=wl.walls)
        d = np.full(n, wl.density_ratio)
        v = None
        sim = O.OracleSim(O.D2Q9, edge, 2 * edge, 1, wl.tau, body_force=wl.body_force, walls=wl.walls,
                          gravity=wl.gravity, gap=0.0)
        sample = "D2Q9 %dx%d closed box, %d disks r=10" % (edge, 2 * edge, n)
    sim.add_particles(c, r, d, v)
    sites = sim.N
    t = time.perf_counter()
    sim.step(1)
    one = time.perf_counter() - t
    steps = max(1, int(target_s / max(one, 1e-6)))
    t = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t
    base = {"value": sites * steps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%s, %d steps, %.1f s, single-threaded FP64 C" % (sample, steps, dt),
            "host": host_info()}
    # The same oracle built with OpenMP over its site loops (identical results), all cores.
    if wl.lattice == "D3Q19":
        par = O.OracleSim(O.D3Q19, edge, edge, edge, s.tau, body_force=s.body_force,
                          body_force_on_particles=s.body_force_on_particles, openmp=True)
    else:
        par = O.OracleSim(O.D2Q9, nx2, ny2, 1, wl.tau, body_force=wl.body_force, walls=wl.walls,
                          gravity=wl.gravity, gap=0.0, openmp=True)
    par.add_particles(c, r, d, v)
    par.step(1)
    t = time.perf_counter()
    par.step(steps)
    dtp = time.perf_counter() - t
    del par
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    base["all_cores"] = {"value": sites * steps / dtp / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "the same sample and steps, %.1f s, FP64 C with OpenMP over the site loops "
                                   "(identical results)" % dtp}
    if not configs:
        return base, []
    from paper_1105_2904_gb300 import lbmp
    _, ur = sim.get_fields()
    pr = sim.get_particles()
    errs = []
    for precision, shape, streaming in configs:
        if wl.lattice == "D3Q19":
            g = lbmp.Simulation(1, edge, edge, edge, s.tau, body_force=s.body_force, precision=precision,
                                body_force_on_particles=s.body_force_on_particles, streaming=streaming)
        else:
            g = lbmp.Simulation(0, nx2, ny2, 1, wl.tau, body_force=wl.body_force, precision=precision,
                                walls=wl.walls, gravity=wl.gravity, streaming=streaming)
        g.set_sweep_shape(shape)
        g.add_particles(c, r, d, v)
        g.step(1 + steps)
        _, ug = g.get_fields()
        pg = g.get_particles()
        g.close()
        errs.append({"velocity": float(np.max(np.abs(ug - ur)) / np.max(np.abs(ur))),
                     "force": float(np.max(np.abs(pg["force"] - pr["force"])) / np.max(np.abs(pr["force"]))),
                     "norm": "max |x - x_oracle| / max |x_oracle| over the field (velocity) or the particles (force)",
                     "sample": "%s, %d steps, %s storage, the timed run's streaming and sweep shape"
                               % (sample, 1 + steps, precision)})
    return base, errs


def host_info():
    """Host cores and CPU model of the machine the baseline ran on."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle as O

    wl = workload(args)
    t0 = time.perf_counter()
    # calibrate the per-site cost, then size the sample so that the run ends in ~1-2 minutes
    s32 = W.suspension_3d_scaled(32)
    c, r, d, v = s32.particles()
    cal = O.OracleSim(O.D3Q19, 32, 32, 32, s32.tau, body_force=s32.body_force, body_force_on_particles=True)
    cal.add_particles(c, r, d, v)
    t = time.perf_counter()
    cal.step(2)
    per_site = (time.perf_counter() - t) / (2 * 32 ** 3)
    budget = 90.0 / max(1, args.steps + args.warmup)
    edge = int(max(24, min(128, (budget / per_site) ** (1.0 / 3.0))))
    s = W.suspension_3d_scaled(edge)
    c, r, d, v = s.particles()
    sim = O.OracleSim(O.D3Q19, edge, edge, edge, s.tau, body_force=s.body_force, body_force_on_particles=True)
    sim.add_particles(c, r, d, v)
    sim.step(args.warmup)
    t = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t
    value = sim.N * args.steps / dt / 1e6
    sample = ("D3Q19 %d^3 periodic, %d spheres r=8 (the %s workload scaled to the same solid fraction), "
              "FP64 oracle, single-threaded" % (edge, len(r), wl.name))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "sample_edge": edge},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1105_2904_gb300 import build as B
    from paper_1105_2904_gb300 import lbmp

    B.build()
    wl = workload(args)
    lattice = 1 if wl.lattice == "D3Q19" else 0
    nx, ny, nz = wl.dims
    N = wl.sites
    c, r, d, v = wl.particles()
    # A dedicated stream (torch's default stream has handle 0): the library enqueues all
    # of its work on it and the timing events are recorded on it.
    stream = torch.cuda.Stream()

    def make():
        sim = lbmp.Simulation(lattice, nx, ny, nz, wl.tau, body_force=wl.body_force, precision=args.precision,
                              walls=wl.walls, gravity=wl.gravity, gap=0.0,
                              body_force_on_particles=wl.body_force_on_particles, cuda_stream=stream.cuda_stream,
                              streaming=args.streaming)
        sim.set_sweep_shape(args.sweep_shape)
        sim.add_particles(c, r, d, v)
        return sim

    sim = make()
    sim.step(args.warmup)
    sim.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    sim.synchronize()   # raises on a device fault recorded during the timed steps
    info = sim.info()
    value, ms = aggregate_throughput(N, args.steps, e0.elapsed_time(e1))

    # Roofline of the dominant kernel (the sweep): per-launch duration with CUDA events.
    # (an even number of steps: the in-place scheme's two phases in equal numbers)
    prof = sim.profile(2 * min(args.steps // 2 if args.steps > 1 else 1, 25))
    # read Q and write Q stored values per site, in either streaming scheme
    Q = 19 if lattice == 1 else 9
    bytes_per_site = 2 * Q * {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[args.precision]
    algo_bytes = bytes_per_site * N
    peak, peak_kind = measured_peaks()
    achieved = algo_bytes / (prof["sweep_ms"] / 1e3) / 1e9
    # which sweep kernel ran: the two-site one for an explicit two-site shape, or by default for
    # every deviation storage (lbm_set_sweep_shape), where nx is even
    shape = args.sweep_shape if args.sweep_shape >= 0 else (0 if args.precision == "fp64" else 16)
    two_site = shape > 0 and args.precision != "fp64" and nx % 2 == 0 and args.streaming == "pull"
    inplace = args.streaming == "inplace"
    kernel_key = "%s_%s_%s" % ("sweep_inplace" if inplace else ("sweep2" if two_site else "sweep"),
                               wl.lattice.lower(), args.precision)
    rec = traffic_record(kernel_key)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (rec["dram_bytes_per_site"] * N if rec else None),
                "kernel": ("k_sweep_inplace (neighbour and local phases in turn, one buffer): fused in-place "
                           "stream" if inplace else
                           ("k_sweep2 (two sites per thread, %d threads along x)" % shape if two_site else "k_sweep")
                           + ": fused pull-stream")
                          + " + IS imposition + collide + BS transfer",
                "algorithmic_bytes_per_launch": algo_bytes, "sweep_ms": prof["sweep_ms"],
                "particle_phase_ms": prof["particle_ms"], "step_ms_ungraphed": prof["step_ms"],
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"}
    del sim
    torch.cuda.synchronize()

    # End to end through the C-ABI with host buffers: create, configure, upload particles,
    # then every step enqueue it and read the particle state (positions, velocities, forces)
    # back to host arrays. The read-backs are asynchronous into two page-locked buffers: the
    # host copies step k's state out while step k + 1 runs.
    e2e = None
    if not args.no_e2e:
        n = len(r)
        host = {k: np.empty((n, 3)) for k in ("x", "u", "omega", "force", "torque")}
        bufs = [torch.empty(15 * n + 1, dtype=torch.float64, pin_memory=True) for _ in range(2)]

        def consume(buf):
            for k, v in lbmp.unpack_particles(buf.numpy(), n).items():
                np.copyto(host[k], v)

        torch.cuda.synchronize()
        barrier()
        t = time.perf_counter()
        s2 = make()
        tickets = [None, None]
        for k in range(args.steps):
            s2.step(1)
            tickets[k % 2] = s2.get_particles_async(bufs[k % 2])
            if k >= 1:
                s2.wait_particles(tickets[(k - 1) % 2])
                consume(bufs[(k - 1) % 2])
        s2.wait_particles(tickets[(args.steps - 1) % 2])
        consume(bufs[(args.steps - 1) % 2])
        dt = time.perf_counter() - t
        s2.close()
        dt = reduce_max(dt)
        h2d = (c.nbytes + r.nbytes + d.nbytes + v.nbytes) / args.steps
        e2e = {"value": N * args.steps * world / dt / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int((15 * n + 1) * 8),
               "includes": "context creation, particle upload and site classification, %d steps each "
                           "followed by a read-back of the particle state to host arrays (asynchronous, "
                           "double-buffered in pinned memory)" % args.steps}

    want_patterns = (rank == 0 and world == 1 and not args.no_patterns and args.workload == "d3q19_512"
                     and not args.edge and args.precision == "fp32" and args.streaming == "pull")
    cpu, err, errs = None, None, []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        configs = [(args.precision, args.sweep_shape, args.streaming)]
        if want_patterns:
            configs += [("fp16", -1, "pull"), ("bf16", -1, "pull")]
        cpu, errs = cpu_baseline(wl, configs=configs)
        err = errs[0]
        full = args.cpu_full or (args.workload == "d3q19_512" and not args.edge)
        if full and not args.no_cpu_full and lattice == 1:
            cpu["full_size"] = cpu_full_size(wl)

    patterns = None
    if want_patterns:
        # The three forms the method is reshaped into, each against the plain FP32 form of this
        # line on the same GPU, with its error stated.
        patterns = {"plain_fp32": {"value": value, "unit": UNIT, "ms_per_step": ms / args.steps,
                                   "error_vs_oracle": err}}
        rp = []
        for k, prec in enumerate(("fp16", "bf16")):
            m = time_storage(wl, prec, args.steps, args.warmup, stream)
            m["error_vs_oracle"] = errs[1 + k] if len(errs) > 1 + k else None
            m["vs_plain_fp32"] = m["value"] / value
            rp.append(m)
        patterns["reduced_precision"] = rp
        ens = measure_ensemble(args.precision, args.steps, args.warmup, rank=0, world=1, with_e2e=False)
        patterns["batched_ensemble"] = {
            "workload": ens["config"]["workload"], "value": ens["value"], "unit": UNIT,
            "ms_per_step": ens["ms_per_step"], "separate_contexts": ens["separate_launches"],
            "vs_separate_contexts": ens["speedup_vs_separate"],
            "sweep_roofline_frac": ens["roofline"]["frac"],
            "error": "bitwise identical to the same cells stepped as separate FP32 contexts; their error "
                     "against the oracle is the FP32 storage error of plain_fp32"}
        ntr, nte = args.pattern_closure_cells
        clo = measure_closure(ntr, nte)
        patterns["learned_closure"] = {
            "workload": clo["config"]["workload"], "value": clo["value"], "unit": clo["unit"],
            "drag_error_vs_fine": clo["drag_error_vs_fine"], "fine_method": clo["fine_method"],
            "speedup_vs_fine_at_drag_accuracy": clo["speedup_vs_fine_at_drag_accuracy"],
            "train_samples": clo["config"]["train_samples"], "test_samples": clo["config"]["test_samples"],
            "seconds": {"generation": clo["generation_seconds"], "training": clo["training_seconds"]}}

    if rank == 0:
        solid = len(r) * (4.0 / 3.0 * math.pi * wl.radius ** 3) / N if lattice == 1 else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": wl.name, "lattice": wl.lattice, "dims": list(wl.dims),
                       "particles": len(r), "radius": wl.radius, "solid_fraction": solid, "tau": wl.tau,
                       "storage": {"fp32": "fp32 deviations", "fp16": "fp16 scaled deviations",
                                   "bf16": "bf16 scaled deviations", "fp64": "fp64"}[args.precision],
                       "streaming": args.streaming,
                       "distribution_bytes": info["bytes_per_site"] * N,
                       "device_bytes": info["device_bytes"],
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: %.1f GB of distributions per step"
                             % (bytes_per_site * N / 1e9)},
            "roofline": roofline, "cpu_baseline": cpu, "error_vs_oracle": err, "e2e": e2e,
            "gpu_launches": int(info["launches_per_step"]) * args.steps,
            "clocks": clk,
        }
        if patterns is not None:
            line["patterns"] = patterns
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def time_storage(wl, precision, steps, warmup, stream):
    """The headline workload in another storage precision (its default sweep kernel): whole-step
    time with CUDA events over `steps` graph replays, and the sweep's per-launch time."""
    import torch
    from paper_1105_2904_gb300 import lbmp

    lattice = 1 if wl.lattice == "D3Q19" else 0
    nx, ny, nz = wl.dims
    c, r, d, v = wl.particles()
    sim = lbmp.Simulation(lattice, nx, ny, nz, wl.tau, body_force=wl.body_force, precision=precision,
                          walls=wl.walls, gravity=wl.gravity, gap=0.0,
                          body_force_on_particles=wl.body_force_on_particles, cuda_stream=stream.cuda_stream)
    sim.add_particles(c, r, d, v)
    sim.step(warmup)
    sim.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    sim.synchronize()
    ms = e0.elapsed_time(e1)
    prof = sim.profile(2 * min(max(steps // 2, 1), 25))
    sim.close()
    Q = 19 if lattice == 1 else 9
    algo = 2 * Q * 2 * wl.sites
    peak, _ = measured_peaks()
    return {"storage": precision + " scaled deviations", "value": wl.sites * steps / (ms / 1e3) / 1e6,
            "unit": UNIT, "ms_per_step": ms / steps, "sweep_ms": prof["sweep_ms"],
            "particle_phase_ms": prof["particle_ms"],
            "sweep_roofline_frac": algo / (prof["sweep_ms"] / 1e3) / 1e9 / peak,
            "kernel": "k_sweep2 (two sites per thread, 16 threads along x)"}


def cpu_full_size(wl):
    """The all-core oracle on the full-size workload: set-up, then 10 steps timed; the per-step
    time is what a full run of the oracle would take per step (extrapolated, not run)."""
    import oracle as O

    c, r, d, v = wl.particles()
    nx, ny, nz = wl.dims
    t = time.perf_counter()
    sim = O.OracleSim(O.D3Q19, nx, ny, nz, wl.tau, body_force=wl.body_force,
                      body_force_on_particles=wl.body_force_on_particles, openmp=True)
    sim.add_particles(c, r, d, v)
    setup = time.perf_counter() - t
    t = time.perf_counter()
    sim.step(10)
    dt = time.perf_counter() - t
    del sim
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": wl.sites * 10 / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%s, full size, 10 steps after %.1f s of set-up, FP64 C with OpenMP over the site "
                      "loops; %.2f s per step, so %.0f s for the workload's %d steps (extrapolated)"
                      % (wl.name, setup, dt / 10, dt / 10 * wl.steps, wl.steps)}


def run_ensemble(args):
    """64 independent periodic D3Q19 cells (edges 32-128, 1-8 spheres of radius 4-10, tau in
    [0.55, 1]) advanced as one batch (one sweep launch over all cells, batched particle
    phase, multi-step graphs, autotuned launch configuration), against the same cells stepped
    as 64 separate contexts (one graph launch per cell per step, each with its default sweep
    kernel). The batch is bit for bit the cells stepped alone with the one-site kernel."""
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    line = measure_ensemble(args.precision, args.steps, args.warmup, rank, world, with_e2e=not args.no_e2e)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_ensemble(prec, steps, warmup, rank, world, with_e2e=True):
    """The ensemble measurement of run_ensemble; returns its JSON line (rank 0) or None."""
    import torch
    from paper_1105_2904_gb300 import autotune as AT
    from paper_1105_2904_gb300 import build as B
    from paper_1105_2904_gb300 import lbmp

    local = int(os.environ.get("LOCAL_RANK", "0"))
    B.build()
    # Ensembles shard by cell: every rank advances its own 64 seeded cells (rank 0 the
    # reference ensemble), with no exchange between ranks.
    e = W.ensemble_cells(seed=4 + rank)
    n_cells = len(e.dims)
    F = [e.body_force] * n_cells

    def make_batch(p):
        b = lbmp.Batch(1, e.dims, e.taus, F, precision=p, gap=0.0, body_force_on_particles=e.body_force_on_particles)
        for k in range(n_cells):
            if len(e.radii[k]):
                b.add_particles(k, e.centers[k], e.radii[k], e.densities[k], e.velocities[k])
        return b

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    b = make_batch(prec)
    spg = max(1, min(50, steps))
    best, trials = AT.tune(b, trial_steps=8, steps_per_graph=spg)
    stream = torch.cuda.ExternalStream(b.stream)
    b.step(warmup)
    b.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    b.synchronize()
    info = b.info()
    value, ms = aggregate_throughput(e.sites, steps, e0.elapsed_time(e1))
    prof = b.profile(min(steps, 30))
    bytes_per_site = {"fp32": 152, "fp16": 76, "bf16": 76, "fp64": 304}[prec]
    algo_bytes = bytes_per_site * e.sites
    peak, peak_kind = measured_peaks()
    achieved = algo_bytes / (prof["sweep_ms"] / 1e3) / 1e9
    rec = traffic_record("sweep_batch_ensemble_%s" % prec)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (rec["dram_bytes_per_site"] * e.sites if rec else None),
                "kernel": "k_sweep_batch (all cells in one launch)",
                "algorithmic_bytes_per_launch": algo_bytes, "sweep_ms": prof["sweep_ms"],
                "particle_phase_ms": prof["particle_ms"], "step_ms_ungraphed": prof["step_ms"],
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"}
    b.close()

    # The same cells as separate contexts, one graph launch per cell per step, on one stream.
    sep_stream = torch.cuda.Stream()
    sims = []
    for k in range(n_cells):
        nx, ny, nz = e.dims[k]
        s_ = lbmp.Simulation(1, nx, ny, nz, e.taus[k], body_force=e.body_force, precision=prec, gap=0.0,
                             body_force_on_particles=e.body_force_on_particles, cuda_stream=sep_stream.cuda_stream)
        s_.set_sweep_shape(0)   # the batch sweep's kernel: results bit for bit those of the batch
        if len(e.radii[k]):
            s_.add_particles(e.centers[k], e.radii[k], e.densities[k], e.velocities[k])
        sims.append(s_)
    for _ in range(warmup):
        for s_ in sims:
            s_.step(1)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(sep_stream)
    for _ in range(steps):
        for s_ in sims:
            s_.step(1)
    f1.record(sep_stream)
    torch.cuda.synchronize()
    sep_ms = f0.elapsed_time(f1)
    for s_ in sims:
        s_.close()
    sep_value, _ = aggregate_throughput(e.sites, steps, sep_ms)

    # End to end through the C-ABI with host buffers: batch creation, particle upload, then
    # every step a read-back of every cell's particle state.
    e2e = None
    if with_e2e:
        torch.cuda.synchronize()
        t = time.perf_counter()
        b2 = make_batch(prec)
        b2.set_tuning(tile_width=best["tile_width"], order=best["order"], grid=best["grid"], steps_per_graph=1)
        views = [b2.cell(k) for k in range(n_cells)]
        hosts = [{q: np.empty((len(e.radii[k]), 3)) for q in ("x", "u", "omega", "force", "torque")}
                 for k in range(n_cells)]
        for _ in range(steps):
            b2.step(1)
            for k in range(n_cells):
                if len(e.radii[k]):
                    lbmp.lbm_get_particles(views[k].h, len(e.radii[k]), hosts[k])
        dt = time.perf_counter() - t
        b2.close()
        dt = reduce_max(dt)
        h2d = sum(c.nbytes + r.nbytes + d.nbytes + v.nbytes
                  for c, r, d, v in zip(e.centers, e.radii, e.densities, e.velocities)) / steps
        e2e = {"value": reduce_sum(e.sites) * steps / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(5 * 3 * 8 * e.n_particles),
               "includes": "batch creation, particle upload and site classification, %d steps each followed "
                           "by a particle-state read-back of every cell" % steps}

    if rank == 0:
        return {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": e.name, "cells": n_cells, "sites": e.sites, "total_cells": n_cells * world, "particles": e.n_particles,
                       "dropped_spheres": int(sum(e.dropped)), "storage": prec,
                       "tuning": {"policy": best["policy"], "order": best["order"], "grid": best["grid"],
                                  "steps_per_graph": spg, "candidates": len(trials)},
                       "parallelism": ("cells sharded: %d distinct seeded cells per GPU" % n_cells) if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: %.1f GB of distributions per step" % (algo_bytes / 1e9)},
            "separate_launches": {"value": sep_value, "unit": UNIT, "ms_per_step": sep_ms / steps,
                                  "launches_per_step": "one step graph per cell (%d)" % n_cells,
                                  "error": "bitwise identical to the batch (the contexts run the one-site sweep, "
                                           "the batch's kernel)"},
            "speedup_vs_separate": value / sep_value,
            "roofline": roofline, "cpu_baseline": None, "e2e": e2e,
            "gpu_launches": int(info["launches_per_step"]) * steps,
            "clocks": clk,
        }
    return None


def run_closure(args):
    """Learned drag closure: paired coarse (r = 3, 32^3 cells) / fine (r = 12, 128^3 cells)
    runs of seeded cells with 8 fixed spheres each, the network trained on the GPU on one set
    of seeds and judged against the fine method on held-out seeds. The value is the drag
    throughput of coarse + closure expressed as fine-lattice site updates per second (the
    fine method's work per drag evaluation over the time the closure path takes for it); the
    fine method's own MLUPS is reported beside it, with the drag errors of both paths."""
    import torch

    world, rank, local = dist_setup()
    if world > 1 and rank != 0:
        return
    torch.cuda.set_device(local)
    ntr, nte = args.closure_cells
    print(json.dumps(measure_closure(ntr, nte, args.closure_large_cells, args.closure_large_train)), flush=True)


def measure_closure(ntr, nte, n_large=0, n_large_train=0):
    """The closure measurement of run_closure on ntr training and nte held-out cells; returns
    its JSON line. n_large > 0: the trained network is also judged on that many held-out
    cells of the large configuration (128^3 coarse cells with 200 spheres of radius 3, 512^3
    fine twins with radius 12; 1.1 % solid against the training cells' 2.8 %)."""
    import torch
    from paper_1105_2904_gb300 import build as B
    from paper_1105_2904_gb300 import closure as CL

    B.build()
    spec = CL.PairSpec()
    t0 = time.perf_counter()
    Xtr, Ttr, ctr, ftr, str_ = CL.generate(spec, ntr, seed=1)
    t_gen = time.perf_counter() - t0
    Xte, Tte, cte, fte, ste = CL.generate(spec, nte, seed=2)
    cl = CL.Closure(seed=0)
    t0 = time.perf_counter()
    cl.fit(Xtr, Ttr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    e_coarse = CL.drag_errors(cte, fte)
    e_closure = CL.drag_errors(cl.corrected(Xte, cte, ste), fte)
    # timing: one batch of held-out cells by each path, CUDA events on the batch stream
    cells = CL.place(spec, nte, seed=2)

    def timed(fine):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        b = CL._run(spec, cells, fine=fine)
        ev[1].record()
        torch.cuda.synchronize()
        f = spec.factor if fine else 1
        sites = (spec.L * f) ** 3 * nte * spec.steps * f * f
        t = ev[0].elapsed_time(ev[1]) / 1e3
        return b, sites, t

    bc, sites_c, t_c = timed(False)
    xin = torch.cat([bc.cell(k).closure_features(spec.n_side, spec.spacing, 1e-3) for k in range(nte)], 0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    cl.net.forward(xin)
    ev[1].record()
    torch.cuda.synchronize()
    t_inf = ev[0].elapsed_time(ev[1]) / 1e3
    bc.close()
    bf, sites_f, t_f = timed(True)
    bf.close()
    value = sites_f / (t_c + t_inf) / 1e6
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS (fine-lattice equivalent)", "n_gpus": 1,
            "steps": spec.steps, "warmup": 0, "higher_is_better": True, "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "closure_d3q19_coarse32_r3_fine128_r12", "spheres_per_cell": spec.n_spheres,
                       "train_samples": int(Xtr.shape[0]), "test_samples": int(Xte.shape[0]),
                       "network": CL.SIZES, "tau": spec.tau, "coarse_steps": spec.steps},
            "drag_error_vs_fine": {"coarse_mean": float(e_coarse.mean()), "coarse_p95": float(np.percentile(e_coarse, 95)),
                                   "closure_mean": float(e_closure.mean()),
                                   "closure_p95": float(np.percentile(e_closure, 95)),
                                   "closure_max": float(e_closure.max())},
            "fine_method": {"value": sites_f / t_f / 1e6, "unit": "MLUPS", "seconds": t_f},
            "closure_path_seconds": {"coarse_runs": t_c, "inference": t_inf},
            "speedup_vs_fine_at_drag_accuracy": t_f / (t_c + t_inf),
            "generation_seconds": t_gen, "training_seconds": t_train}
    if n_large > 0:
        big = CL.PairSpec(L=128, n_spheres=200)
        t0 = time.perf_counter()
        Xb, Tb, cb, fb, sb = CL.generate(big, n_large, seed=3)
        t_big = time.perf_counter() - t0
        eb_coarse = CL.drag_errors(cb, fb)
        eb_closure = CL.drag_errors(cl.corrected(Xb, cb, sb), fb)
        line["large_cells"] = {
            "workload": "128^3 coarse cells, 200 spheres r=3 (512^3 fine twins, r=12), held-out seeds",
            "cells": n_large, "samples": int(Xb.shape[0]),
            "drag_error_vs_fine": {"coarse_mean": float(eb_coarse.mean()),
                                   "coarse_p95": float(np.percentile(eb_coarse, 95)),
                                   "closure_mean": float(eb_closure.mean()),
                                   "closure_p95": float(np.percentile(eb_closure, 95))},
            "trained_on": "the %d small cells above (32^3, 8 spheres each)" % ntr,
            "generation_seconds": t_big}
        if n_large_train > 0:
            t0 = time.perf_counter()
            Xl, Tl, cl_c, fl, sl = CL.generate(big, n_large_train, seed=5)
            t_lg = time.perf_counter() - t0
            cl2 = CL.Closure(seed=0)
            cl2.fit(Xl, Tl)
            e2 = CL.drag_errors(cl2.corrected(Xb, cb, sb), fb)
            # the coarse and fine runs of the held-out large cells, timed (CUDA events)
            cells_b = CL.place(big, n_large, seed=3)

            def timed_big(fine):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                torch.cuda.synchronize()
                ev[0].record()
                b = CL._run(big, cells_b[:1], fine=fine)
                ev[1].record()
                torch.cuda.synchronize()
                b.close()
                return ev[0].elapsed_time(ev[1]) / 1e3
            t_c1, t_f1 = timed_big(False), timed_big(True)
            line["large_cells"]["trained_on_large_cells"] = {
                "cells": n_large_train, "samples": int(Xl.shape[0]),
                "drag_error_vs_fine": {"closure_mean": float(e2.mean()),
                                       "closure_p95": float(np.percentile(e2, 95)),
                                       "closure_max": float(e2.max())},
                "seconds_per_cell": {"coarse": t_c1, "fine": t_f1},
                "generation_seconds": t_lg}
            cl2.close()
    cl.close()
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble_64":
        run_ensemble(args)
    elif args.workload == "closure":
        run_closure(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
