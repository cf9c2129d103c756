#!/usr/bin/env python
"""Throughput benchmark of the fused two-lattice step: MLUPS (one update of
both lattices of one cell) and the HBM-roofline fraction of the step kernel.

Default workload (``--workload batch``): 256 independent 2D drop-on-flat-wall
domains with sides drawn from {64, 128, 256, 512}, contact angles 30-150 deg,
density ratios 1-100 (seed 1; about 24M cells, 3.1 GB of state, larger than
L2), FP16 population storage with FP32 arithmetic, advanced by one persistent
autotuned launch per time step replayed from a CUDA graph.  One bench step =
one time step of every domain.

Other workloads: ``drop_on_cylinder`` (512 x 512, density ratio 100, FP32;
its state fits in L2, so L2 is flushed between individually timed steps),
``static_drop`` (128 x 128, FP64), ``water_entry``, ``annulus`` and
``channel`` (moving particles), ``porous_2d`` (phase separation in random
discs between bounce-back walls) and ``drainage_3d``.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores.  Under torchrun every rank runs an
independent replica (no data-path collective; weak scaling) and rank 0 prints
one JSON line with the max-over-ranks time.
"""
import argparse
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

# algorithmic bytes per cell update: every population read and written once,
# lagged fields (u, S, phi) read and written once, phi0 read once
BYTES_PER_CELL = {
    "p64": 8 * (36 + 11),
    "p32": 4 * (36 + 11),
    "fp16": 2 * 2 * (8 + 9) + 2 * 8 + 4 * 11,
    "bf16": 2 * 2 * (8 + 9) + 2 * 8 + 4 * 11,
}
BYTES_PER_CELL_3D = {
    "p64": 8 * (52 + 15),
    "p32": 4 * (52 + 15),
    "fp16": 2 * 2 * (6 + 19) + 2 * 8 + 4 * 15,
    "bf16": 2 * 2 * (6 + 19) + 2 * 8 + 4 * 15,
}
# arithmetic type of the path (the storage type of the populations goes in config.storage)
DTYPE = {"p64": "f64", "p32": "f32", "fp16": "f32", "bf16": "f32"}
STORAGE = {"p64": "f64", "p32": "f32", "fp16": "f16 populations (int64 rest, f32 lagged fields)",
           "bf16": "bf16 populations (int64 rest, f32 lagged fields)"}


KERNEL_DESC = ["one cell per thread (tiles)", "two cells per thread (tiles)",
               "two cells per thread (tiles), bulk-copy staging",
               "near tiles one cell, far tiles two cells per thread",
               "two cells per thread on strips marched in y (tile = strip width x segment rows), "
               "tensor-copy staging"]

# timed regions of K steps each in the batched workloads; the median is reported
REPEATS = 5
# end-to-end call sequences of the batched workloads; the median is reported
E2E_REPEATS = 5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "drop_on_cylinder", "static_drop", "water_entry",
                             "drainage_3d", "annulus", "porous_2d", "channel", "drops"])
    ap.add_argument("--n3d", type=int, default=256, help="cube side of drainage_3d")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--precision", default=None)
    ap.add_argument("--config", type=int, nargs=4, default=None,
                    metavar=("TILE_X", "TILE_Y", "KERNEL", "CTAS_PER_SM"),
                    help="fix the launch configuration instead of autotuning it")
    ap.add_argument("--phase-model", type=int, default=0, choices=[0, 1],
                    help="order parameter: 0 Cahn-Hilliard (the paper's), 1 conservative Allen-Cahn")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def with_phase_model(c, phase_model):
    """The workload with the order-parameter lattice chosen (0: Cahn-Hilliard,
    1: conservative Allen-Cahn)."""
    if phase_model:
        c["params"] = dict(c["params"], phase_model=phase_model)
        if "desc" in c:
            c["desc"] += "; conservative Allen-Cahn order parameter"
    return c


def batch_workload(count=256, phase_model=0):
    from paper_2311_05097_gb300 import workloads as W
    draws = W.batch_cases(count, seed=1)
    cases = [with_phase_model(W.flat_wall_drop(d["L"], d["theta_deg"], d["rho_ratio"]), phase_model)
             for d in draws]
    return dict(cases=cases, draws=draws, precision="fp16",
                desc="%d independent 2D drop-on-flat-wall domains, sides uniform over "
                     "{64,128,256,512}, theta U[30,150] deg, density ratio log-U[1,100], "
                     "seed 1%s" % (count, "; conservative Allen-Cahn order parameter" if phase_model else ""))


def batch_like(args):
    """The batched workload named by --workload (batch or drops)."""
    if args.workload == "drops":
        return drops_workload(args.batch_count, args.phase_model)
    return batch_workload(args.batch_count, args.phase_model)


def drops_workload(count=256, phase_model=0):
    from paper_2311_05097_gb300 import workloads as W
    draws = W.batch_cases(count, seed=1)
    cases = [with_phase_model(W.periodic_drop(d["L"], d["rho_ratio"]), phase_model) for d in draws]
    return dict(cases=cases, draws=draws, precision="fp16",
                desc="%d independent 2D periodic drop domains (radius L/4, no solid), sides uniform over "
                     "{64,128,256,512}, density ratio log-U[1,100], seed 1%s"
                     % (count, "; conservative Allen-Cahn order parameter" if phase_model else ""))


def single_workload(name, n3d=256, phase_model=0):
    return with_phase_model(_single_workload(name, n3d), phase_model)


def _single_workload(name, n3d=256):
    from paper_2311_05097_gb300 import workloads as W
    if name == "water_entry":
        c = W.water_entry()
        c["precision"] = "bf16"
        c["desc"] = ("2D water entry: particle R=40, rho_p=2, u=-0.02, 1024x2048, pool depth 800, "
                     "density ratio 10, theta 90 deg; force/torque reduction and Newton-Euler "
                     "in FP64 every step")
        return c
    if name == "annulus":
        c = W.annulus_mixing()
        c["precision"] = "p32"
        c["desc"] = ("2D annulus mixing (Sec. 4.5 layout): 512x512, outer wall, inner cylinder R=64 "
                     "rotating at 1e-4 rad/step, 15 free wetting particles (R 20-30, own contact angles "
                     "45-135 deg), repulsion, gravity on particles; force/torque reduction and "
                     "Newton-Euler in FP64 every step")
        return c
    if name == "channel":
        c = W.channel_displacement()
        c["precision"] = "p32"
        c["desc"] = ("2D displacement in a complex channel (Sec. 4.6 layout): 1280x256, bottom wall with two "
                     "cavities, bounce-back walls at both ends of y, a drop of fluid 1 in the small cavity, "
                     "16 free particles (R 16-20, own contact angles 80-100 deg), body force 3e-7, "
                     "particle-particle and particle-wall repulsion; force/torque reduction and Newton-Euler "
                     "in FP64 every step")
        return c
    if name == "porous_2d":
        c = W.porous_phase_separation_2d(n=1024, theta_deg=45.0)
        c["precision"] = "p32"
        c["desc"] = ("2D phase separation in a porous medium (Sec. 4.1 setting), 1024x1024, random discs "
                     "R 6-12 (porosity %.3f), phi = (1 - phi0) U(-1,1), theta 45 deg, sigma 1e-3, M 0.1, "
                     "equal densities; no-flux bounce-back walls at both ends of y" % c["porosity"])
        return c
    if name == "drainage_3d":
        c = W.porous_drainage_3d(n=n3d)
        c["precision"] = "fp16"
        c["desc"] = ("3D drainage, %d^3, random non-overlapping spheres R 8-16 (porosity %.3f), "
                     "theta 120 deg, body force 1e-6, density ratio 10, solid viscosity cap 10x, D3Q19 + D3Q7"
                     % (n3d, c["porosity"]))
        return c
    if name == "drop_on_cylinder":
        c = W.drop_on_cylinder()
        c["precision"] = "p32"
        c["desc"] = ("2D drop (R0=50) on a fixed cylinder (Rp=60) between wall slabs, 512x512, "
                     "density ratio 100, viscosity ratio 100, theta 60 deg")
    else:
        c = W.static_drop()
        c["precision"] = "p64"
        c["desc"] = "2D static drop R=25, 128x128 periodic, density ratio 10, viscosity ratio 10"
    return c


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 power=float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r["sm"] > 0.5 * r["smax"]] or rows
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(r["power"] for r in rows)}


def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def read_traffic(key, config=None):
    """DRAM bytes per launch recorded under profiles/ for this workload and
    precision, or None when there is none or it was taken for another launch
    configuration than the one timed."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        ents = json.load(open(path)).get(key, [])
    except Exception:
        return None
    for ent in ents if isinstance(ents, list) else [ents]:
        if config is None or ent.get("config") is None or list(ent["config"]) == list(config):
            return ent.get("bytes_per_launch")
    return None


# ---------------------------------------------------------------------------------------------
# oracle (CPU) timing: a bounded sample of the workload
# ---------------------------------------------------------------------------------------------
def oracle_steps(args, budget_s):
    """The reference arm: W warm-up and exactly K timed steps of the FP64
    oracle on a bounded sample of the workload -- whole domains taken in order
    from the batch list (a single-domain workload is its one domain), as many
    as keep the K + W steps within about ``budget_s`` seconds.  Returns
    (MLUPS, timed seconds, sampled cells per step, description, threads)."""
    from oracle import oracle as O
    if args.workload in ("batch", "drops"):
        cases = batch_like(args)["cases"]
    else:
        cases = [single_workload(args.workload, args.n3d, args.phase_model)]
    total = max(args.steps, 1) + max(args.warmup, 0)
    sims, cells, t_est = [], 0, 0.0
    for c in cases:
        o = O.OracleSim(c["shape"], O.make_params(**c["params"]))
        if c.get("walls_y"):
            o.set_walls(True)
        for k, pp in enumerate(c.get("particles", [])):
            o.set_particle(k, O.Particle(**pp))
        o.init(c["phi0"], c["phi"], c.get("u"))
        t0 = time.perf_counter()
        o.step(1)  # probe: cost of one step of this domain (part of its warm-up)
        one = time.perf_counter() - t0
        if sims and t_est + one * total > budget_s:
            break
        sims.append((o, c))
        cells += int(math.prod(c["shape"]))
        t_est += one * total
    for o, _ in sims:
        o.step(max(args.warmup - 1, 0))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for o, _ in sims:
            o.step(1)
    dt = time.perf_counter() - t0
    desc = ("FP64 C oracle (OpenMP) on %d whole domain(s) of the workload (%s; %d cells), %d warm-up + "
            "%d timed steps" % (len(sims), ", ".join("x".join(map(str, c["shape"])) for _, c in sims[:8])
                                + (", ..." if len(sims) > 8 else ""), cells, args.warmup, args.steps))
    return cells * args.steps / dt / 1e6, dt, cells, desc, O.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    v, dt, sample_cells, desc, cores = oracle_steps(args, 90.0)
    if args.workload in ("batch", "drops"):
        bw = batch_like(args)
        cells = sum(int(math.prod(c["shape"])) for c in bw["cases"])
        cfg = {"workload": args.workload, "domains": len(bw["cases"]), "cells": cells,
               "precision": "p64 (oracle)", "desc": bw["desc"]}
    else:
        c = single_workload(args.workload, args.n3d, args.phase_model)
        cells = int(math.prod(c["shape"]))
        cfg = {"workload": args.workload, "cells": cells, "precision": "p64 (oracle)",
               "desc": c["desc"]}
    # each step advances the sampled cells only: ms_per_step is the time of one
    # such step, so ms_per_step x steps is the timed region that ran
    line = {"impl": "reference", "metric": "MLUPS", "value": round(v, 4), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / max(args.steps, 1) * 1e3, 3),
            "sampled": True, "sample_cells_per_step": sample_cells,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, order_parameter="allen-cahn" if args.phase_model else "cahn-hilliard"),
            "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def setup_dist():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return dist, int(os.environ.get("RANK", "0")), world, local


def max_over_ranks(dist, value):
    """Maximum of ``value`` over the ranks of the default process group (NCCL
    on the GPUs; any CPU backend such as gloo reduces a host tensor)."""
    if not dist:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank, steps, world, slowest_ms):
    """Whole-job throughput of ``world`` replicas that each advance
    ``cells_per_rank`` cells by ``steps`` steps, timed by the slowest rank."""
    return cells_per_rank * steps * world / (slowest_ms * 1e-3) / 1e6


def run_batch(args, dist, rank, world, local):
    import ctypes as C

    import numpy as np
    import torch
    from paper_2311_05097_gb300 import pf

    bw = batch_like(args)
    cases = bw["cases"]
    prec = args.precision or bw["precision"]
    cells = sum(int(math.prod(c["shape"])) for c in cases)
    stream = torch.cuda.Stream()
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision=prec,
                 stream=stream.cuda_stream)
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"])
    if args.config:
        b.set_config(*args.config)
    # warm-up: the first long call runs the launch-configuration autotuner
    b.step(256 + max(args.warmup, 3))
    b.sync()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    n0 = pf.launch_count()
    # REPEATS timed regions of exactly K steps each (barrier + synchronize on
    # both sides); the headline is the median region, max over ranks
    reps_ms = []
    t_wall = time.perf_counter()
    for _ in range(REPEATS):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        reps_ms.append(e0.elapsed_time(e1))
    t_wall = time.perf_counter() - t_wall
    launches = (pf.launch_count() - n0) // REPEATS
    b.sync()
    clk = clocks.stop()
    total_ms = max_over_ranks(dist, statistics.median(reps_ms))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    mlups = whole_job_mlups(cells, args.steps, world, total_ms)
    bpc = BYTES_PER_CELL[prec]
    avg_s = total_ms * 1e-3 / args.steps  # one step-kernel launch per step
    achieved = bpc * cells / avg_s / 1e9
    tx, ty, cps, cpt = b.config()

    e2e = None
    if not args.no_e2e:
        S = 100
        hosts = [(torch.from_numpy(np.ascontiguousarray(c["phi0"])).pin_memory(),
                  torch.from_numpy(np.ascontiguousarray(c["phi"])).pin_memory(),
                  torch.empty(c["phi"].shape, dtype=torch.float64).pin_memory()) for c in cases]
        L = pf.load()
        nd = len(hosts)
        t_phi0 = (C.c_void_p * nd)(*[h[0].data_ptr() for h in hosts])
        t_phi = (C.c_void_p * nd)(*[h[1].data_ptr() for h in hosts])
        t_out = (C.c_void_p * nd)(*[h[2].data_ptr() for h in hosts])
        # E2E_REPEATS call sequences, each on a batch created for it (outside the
        # timed region); the median is reported
        dts = []
        for _ in range(E2E_REPEATS):
            e2e_b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases],
                             precision=prec, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = L.pf_batch_init_all(e2e_b._h, C.cast(t_phi0, C.c_void_p), C.cast(t_phi, C.c_void_p), None, None,
                                     pf.PF_HOST)
            if rc:
                raise pf.PfError(rc, pf.last_error())
            e2e_b.step(S)
            rc = L.pf_batch_get_macros_all(e2e_b._h, C.cast(t_out, C.c_void_p), None, None, None, None,
                                           pf.PF_HOST)
            if rc:
                raise pf.PfError(rc, pf.last_error())
            dts.append(time.perf_counter() - t0)
            e2e_b.close()
        dt = statistics.median(dts)
        e2e = {"value": round(cells * S / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": 16 * cells // S, "d2h_bytes_per_step": 8 * cells // S,
               "h2d_bytes_per_call": 16 * cells, "d2h_bytes_per_call": 8 * cells,
               "steps_per_call": S,
               "desc": "each call sequence: pf_batch_init_all (every domain from pinned host phi0, "
                       "phi); pf_batch_step(%d) (includes the autotuner's timed steps when the "
                       "configuration is not cached); pf_batch_get_macros_all (phi of every domain "
                       "to pinned host); wall clock, median of %d sequences (ms: %s)"
                       % (S, E2E_REPEATS, ", ".join("%.1f" % (v * 1e3) for v in dts))}
    b.close()
    cfg = {"workload": args.workload, "domains": len(cases), "cells": cells, "precision": prec,
           "desc": bw["desc"], "l2": "state (%.2f GB) larger than L2 (129 MB); no flush"
                                   % (cells * bpc / 1e9),
           "tile": [tx, ty], "ctas_per_sm": cps, "kernel": cpt, "cells_per_thread": 2 if cpt else 1,
           "kernel_desc": KERNEL_DESC[cpt],
           "parallelism": "independent replicas per GPU" if world > 1 else "single GPU"}
    cfg["timing"] = ("median of %d timed regions of %d steps each (ms: %s)"
                     % (REPEATS, args.steps, ", ".join("%.2f" % v for v in reps_ms)))
    return dict(mlups=mlups, total_ms=total_ms, achieved=achieved, bpc=bpc, prec=prec, cfg=cfg,
                clk=clk, launches=launches, e2e=e2e, t_wall=t_wall,
                kernel=step_kernel_name(2, cpt), launch_config=[tx, ty, cpt])


def step_kernel_name(dim, variant):
    """The step kernel(s) of a launch variant (the roofline's dominant kernel)."""
    if dim == 3:
        return "k_step3d"
    return ["k_step2d", "k_step2d_pair", "k_step2d_stage", "k_step2d_pair+k_step2d", "k_step2d_strip"][variant]


def run_single(args, dist, rank, world, local):
    import numpy as np
    import ctypes as C

    import torch
    from paper_2311_05097_gb300 import pf

    case = single_workload(args.workload, args.n3d, args.phase_model)
    prec = args.precision or case["precision"]
    cells = int(math.prod(case["shape"]))
    dim = len(case["shape"])
    bpc = (BYTES_PER_CELL if dim == 2 else BYTES_PER_CELL_3D)[prec]
    in_l2 = cells * bpc < 256e6  # state small enough to stay in the 129 MB L2 between steps
    stream = torch.cuda.Stream()
    sim = pf.Sim(case["shape"], precision=prec, stream=stream.cuda_stream,
                 walls_y=case.get("walls_y", False), **case["params"])
    for k, pp in enumerate(case.get("particles", [])):
        sim.set_particle(k, **pp)
    sim.init(case["phi0"], case["phi"], case.get("u"))
    if args.config:
        sim.set_config(*args.config)
    else:
        # the autotuner times its candidates on a scratch copy of the workload
        # so the timed run starts at step 0 (the water entry diverges after
        # ~300 steps at its parameters)
        scratch = pf.Sim(case["shape"], precision=prec, stream=stream.cuda_stream,
                         walls_y=case.get("walls_y", False), **case["params"])
        for k, pp in enumerate(case.get("particles", [])):
            scratch.set_particle(k, **pp)
        scratch.init(case["phi0"], case["phi"], case.get("u"))
        scratch.autotune()
        tx, ty, cps, kern = scratch.config()
        scratch.close()
        sim.set_config(tx, ty, kern, cps)
    tx, ty, cps, kern = sim.config()
    launch = {"tile": [tx, ty], "ctas_per_sm": cps, "kernel": kern,
              "kernel_desc": ["one cell per thread", "two cells per thread", "two cells per thread, staged",
                              "near tiles one cell, far tiles two cells per thread",
                              "two cells per thread on strips marched in y, tensor-copy staging"][kern]}
    if not in_l2:
        return run_single_large(args, dist, rank, world, local, case, prec, cells, bpc, sim, stream, launch)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    scrub = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_l2():
        # write 512 MiB (evicts the state), then read 256 MiB so the dirty
        # flush lines are written back before, not during, the timed step
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            scrub.sum()

    for _ in range(max(args.warmup, 3)):
        flush_l2()
        sim.step(1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    n0 = pf.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush_l2()
        ev[k][0].record(stream)
        sim.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = pf.launch_count() - n0
    sim.sync()
    clk = clocks.stop()
    total_ms = max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in ev))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    mlups = whole_job_mlups(cells, args.steps, world, total_ms)
    achieved = bpc * cells / (total_ms * 1e-3 / args.steps) / 1e9

    e2e = None
    if not args.no_e2e:
        S, iters = 20, 5
        phi0_h = torch.from_numpy(case["phi0"]).pin_memory()
        phi_h = torch.from_numpy(case["phi"]).pin_memory()
        u0 = case.get("u")
        u_h = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory() if u0 is not None else None
        out_h = torch.empty(cells, dtype=torch.float64).pin_memory()
        L = pf.load()
        s2 = pf.Sim(case["shape"], precision=prec, stream=stream.cuda_stream,
                 walls_y=case.get("walls_y", False), **case["params"])
        parts = case.get("particles", [])
        for k, pp in enumerate(parts):
            s2.set_particle(k, **pp)
        s2.init(case["phi0"], case["phi"], case.get("u"))
        s2.set_config(tx, ty, kern, cps)  # the timed run's launch configuration (kept across inits)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(iters):
            # the same workload as the timed run: particles reset, initial flow
            for k, pp in enumerate(parts):
                s2.set_particle(k, **pp)
            rc = L.pf_init_fields(s2._h, C.c_void_p(phi0_h.data_ptr()), C.c_void_p(phi_h.data_ptr()),
                                  C.c_void_p(u_h.data_ptr()) if u_h is not None else None, None,
                                  pf.PF_HOST)
            if rc:
                raise pf.PfError(rc, pf.last_error())
            s2.step(S)
            rc = L.pf_get_macros(s2._h, C.c_void_p(out_h.data_ptr()), None, None, None, None,
                                 pf.PF_HOST)
            if rc:
                raise pf.PfError(rc, pf.last_error())
        dt = time.perf_counter() - t0
        s2.close()
        h2d = (16 + (8 * dim if u_h is not None else 0)) * cells + C.sizeof(pf.pf_particle) * len(parts)
        e2e = {"value": round(cells * S * iters / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d // S, "d2h_bytes_per_step": 8 * cells // S,
               "h2d_bytes_per_call": h2d, "d2h_bytes_per_call": 8 * cells,
               "steps_per_call": S,
               "desc": "per call: pf_particle_state(set) of every particle + pf_init_fields(pinned host "
                       "phi0, phi%s) + pf_step(%d) + pf_get_macros(phi to pinned host); wall clock"
                       % (", u" if u_h is not None else "", S)}
    sim.close()
    cfg = {"workload": args.workload, "cells": cells, "precision": prec, "desc": case["desc"],
           "l2": "flushed between timed steps: 512 MiB write, then a 256 MiB read so the "
                 "write-back happens outside the timed step", **launch,
           "parallelism": "independent replicas per GPU" if world > 1 else "single GPU"}
    return dict(mlups=mlups, total_ms=total_ms, achieved=achieved, bpc=bpc, prec=prec, cfg=cfg,
                clk=clk, launches=launches, e2e=e2e, t_wall=t_wall,
                kernel=step_kernel_name(dim, launch["kernel"]))


def run_single_large(args, dist, rank, world, local, case, prec, cells, bpc, sim, stream, launch):
    """A single domain whose state exceeds L2: K steps timed together (graph
    replay), no flush needed."""
    import ctypes as C

    import numpy as np
    import torch
    from paper_2311_05097_gb300 import pf

    sim.step(max(args.warmup, 3))
    sim.sync()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    n0 = pf.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = pf.launch_count() - n0
    sim.sync()
    clk = clocks.stop()
    total_ms = max_over_ranks(dist, e0.elapsed_time(e1))
    if dist:
        dist.barrier()
    mlups = whole_job_mlups(cells, args.steps, world, total_ms)
    nker = round(launches / args.steps)
    achieved = bpc * cells / (total_ms * 1e-3 / args.steps) / 1e9
    e2e = None
    if not args.no_e2e:
        S = 20
        phi0_h = torch.from_numpy(np.ascontiguousarray(case["phi0"])).pin_memory()
        phi_h = torch.from_numpy(np.ascontiguousarray(case["phi"])).pin_memory()
        u0 = case.get("u")
        u_h = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory() if u0 is not None else None
        out_h = torch.empty(cells, dtype=torch.float64).pin_memory()
        parts = case.get("particles", [])
        L = pf.load()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the same workload as the timed run: particles reset, initial flow
        for k, pp in enumerate(parts):
            sim.set_particle(k, **pp)
        rc = L.pf_init_fields(sim._h, C.c_void_p(phi0_h.data_ptr()), C.c_void_p(phi_h.data_ptr()),
                              C.c_void_p(u_h.data_ptr()) if u_h is not None else None, None, pf.PF_HOST)
        if rc:
            raise pf.PfError(rc, pf.last_error())
        sim.step(S)
        rc = L.pf_get_macros(sim._h, C.c_void_p(out_h.data_ptr()), None, None, None, None, pf.PF_HOST)
        if rc:
            raise pf.PfError(rc, pf.last_error())
        dt = time.perf_counter() - t0
        dim = len(case["shape"])
        h2d = (16 + (8 * dim if u_h is not None else 0)) * cells + C.sizeof(pf.pf_particle) * len(parts)
        e2e = {"value": round(cells * S / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d // S, "d2h_bytes_per_step": 8 * cells // S,
               "h2d_bytes_per_call": h2d, "d2h_bytes_per_call": 8 * cells,
               "steps_per_call": S,
               "desc": "pf_particle_state(set) of every particle + pf_init_fields(pinned host phi0, "
                       "phi%s) + pf_step(%d) + pf_get_macros(phi to pinned host); wall clock"
                       % (", u" if u_h is not None else "", S)}
    sim.close()
    cfg = {"workload": args.workload, "cells": cells, "precision": prec, "desc": case["desc"],
           "l2": "state (%.2f GB) larger than L2 (129 MB); no flush" % (cells * bpc / 1e9), **launch,
           "kernels_per_step": nker,
           "parallelism": "independent replicas per GPU" if world > 1 else "single GPU"}
    kernel = step_kernel_name(len(case["shape"]), launch["kernel"])
    return dict(mlups=mlups, total_ms=total_ms, achieved=achieved, bpc=bpc, prec=prec, cfg=cfg,
                clk=clk, launches=launches, e2e=e2e, t_wall=t_wall, kernel=kernel)


# FP64 instructions per 2D cell update of the FP64 step (DADD + DMUL + DFMA thread
# instructions per cell from ncu on the batched workload, kernel 0)
FP64_INST_PER_CELL_2D = 422.1
GB300_SMS = 152
FP64_INST_PER_CLK_PER_SM = 2  # DFMA/DADD/DMUL issue rate of one SM (ncu peak_sustained)


def roofline_entry(args, r, peak, peak_src):
    """HBM roofline of the step; the FP64 2D step is bound by the FP64 pipe
    instead: achieved FP64 instructions per second against the pipe's rate at
    the SM clock measured during the timed region."""
    dim3 = r["kernel"] == "k_step3d"
    if r["prec"] == "p64" and not dim3:
        mhz = (r.get("clk") or {}).get("sm_mhz") or 2070.0
        peak_i = GB300_SMS * FP64_INST_PER_CLK_PER_SM * mhz * 1e-3  # G instructions / s
        ach = FP64_INST_PER_CELL_2D * r["mlups"] * 1e-3
        return {"bound": "alu", "achieved": round(ach, 1), "peak": round(peak_i, 1),
                "unit": "G FP64 inst/s", "frac": round(ach / peak_i, 4), "traffic": None,
                "fp64_inst_per_cell": FP64_INST_PER_CELL_2D, "kernel": r["kernel"],
                "peak_source": "152 SMs x 2 FP64 instructions/clock x SM clock (unit counts and clocks)",
                "hbm_frac": round(r["achieved"] / peak, 4)}
    return {"bound": "hbm", "achieved": round(r["achieved"], 1), "peak": peak,
            "unit": "GB/s", "frac": round(r["achieved"] / peak, 4),
            "traffic": read_traffic("%s/%s%s" % (args.workload, r["prec"], "/allen-cahn" if args.phase_model else ""),
                                    r.get("launch_config")),
            "bytes_per_cell": r["bpc"], "kernel": r["kernel"], "peak_source": peak_src}


def run_ours(args):
    dist, rank, world, local = setup_dist()
    from paper_2311_05097_gb300 import build as B
    if rank == 0 or not dist:
        B.build()
    if dist:
        dist.barrier()
    if args.workload in ("batch", "drops"):
        r = run_batch(args, dist, rank, world, local)
    else:
        r = run_single(args, dist, rank, world, local)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline:
        v, _, _, desc, cores = oracle_steps(argparse.Namespace(**dict(vars(args), steps=2, warmup=1)), 15.0)
        cpu = {"value": round(v, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": desc}
    peaks = read_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)"
    if peak is None:
        peak, peak_src = 6800.0, "fallback"
    line = {
        "metric": "MLUPS", "value": round(r["mlups"], 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[r["prec"]], "data": "synthetic",
        "config": dict(r["cfg"], storage=STORAGE[r["prec"]],
                       order_parameter="allen-cahn" if args.phase_model else "cahn-hilliard"),
        "roofline": roofline_entry(args, r, peak, peak_src),
        "clocks": r["clk"], "e2e": r["e2e"], "gpu_launches": r["launches"], "cpu_baseline": cpu,
        "wall_s": round(r["t_wall"], 3),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
