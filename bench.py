#!/usr/bin/env python
"""Throughput benchmark of the fused two-lattice step (MLUPS, both lattices
per cell update) with its HBM-roofline fraction.

Default workload: 2D drop resting on a fixed cylinder, 512 x 512 cells,
density ratio 1000, viscosity ratio 100, contact angle 60 deg, FP32 storage
and arithmetic.  One bench step = one time step of the whole domain
(the fused step kernel).  The state (~70 MB) fits in L2, so L2 is flushed
(a 512 MiB device write) between timed steps and each step is timed alone
with CUDA events on the library's stream.

Other workloads (--workload): static_drop (128^2, FP64), batch (256
uneven domains, FP16 storage), water_entry (1024 x 2048 with a particle,
BF16 storage).

--impl reference times the FP64 CPU oracle on the same workload (bounded
sample) on the host cores.  Under torchrun each rank runs an independent
replica (no data-path collective); rank 0 prints one JSON line.
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

# algorithmic bytes per cell update: populations read + written once, lagged
# fields (u, S, phi) read + written once, phi0 read once
BYTES_PER_CELL = {
    ("2d", "p64"): 8 * (36 + 11),
    ("2d", "p32"): 4 * (36 + 11),
    ("2d", "fp16"): 2 * 2 * (8 + 9) + 2 * 8 + 4 * 11,
    ("2d", "bf16"): 2 * 2 * (8 + 9) + 2 * 8 + 4 * 11,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="drop_on_cylinder",
                    choices=["drop_on_cylinder", "static_drop"])
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(name):
    from paper_2311_05097_gb300 import workloads as W
    if name == "drop_on_cylinder":
        c = W.drop_on_cylinder()
        c["precision"] = "p32"
        c["desc"] = ("2D drop (R0=50) on a fixed cylinder (Rp=60) between wall slabs, 512x512, "
                     "density ratio 1000, viscosity ratio 100, theta 60 deg")
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
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
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
                "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# oracle (CPU) timing
# ---------------------------------------------------------------------------------------------
def oracle_mlups(case, budget_s=12.0, max_steps=None):
    from oracle import oracle as O
    o = O.OracleSim(case["shape"], O.make_params(**case["params"]))
    o.init(case["phi0"], case["phi"])
    cells = int(math.prod(case["shape"]))
    t0 = time.perf_counter()
    o.step(1)
    dt1 = time.perf_counter() - t0
    n = max(1, int(budget_s / max(dt1, 1e-6)))
    if max_steps:
        n = min(n, max_steps)
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return cells * n / dt / 1e6, n, O.num_threads()


def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    case = workload(args.workload)
    cells = int(math.prod(case["shape"]))
    from oracle import oracle as O
    o = O.OracleSim(case["shape"], O.make_params(**case["params"]))
    o.init(case["phi0"], case["phi"])
    o.step(max(args.warmup, 0) and 1)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    k = min(args.steps, max(1, int(120.0 / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    v = cells * k / dt / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": round(v, 4), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / k * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "cells": cells, "desc": case["desc"]},
            "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": O.num_threads(),
                             "kind": "oracle",
                             "sample": "%d full time steps of the %s workload (FP64 C oracle, OpenMP)"
                                       % (k, args.workload)},
            "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2311_05097_gb300 import build as B
    B.build()
    from paper_2311_05097_gb300 import pf

    case = workload(args.workload)
    prec = args.precision or case["precision"]
    cells = int(math.prod(case["shape"]))
    stream = torch.cuda.Stream()
    sim = pf.Sim(case["shape"], precision=prec, stream=stream.cuda_stream, **case["params"])
    sim.init(case["phi0"], case["phi"])
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
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    torch.cuda.synchronize()
    mlups = cells * args.steps * world / (total_ms * 1e-3) / 1e6
    # roofline of the step kernel (one launch per step)
    bpc = BYTES_PER_CELL[("2d", prec)]
    avg_s = statistics.mean(step_ms) * 1e-3
    achieved = bpc * cells / avg_s / 1e9
    peaks = read_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        tr = json.load(open(tpath)).get("%s/%s" % (args.workload, prec))
        if tr:
            traffic = tr.get("bytes_per_launch")

    # end to end through the public API with host buffers
    e2e = None
    if rank == 0 or True:
        S = 20
        iters = 5
        phi0_h = torch.from_numpy(case["phi0"]).pin_memory().numpy()
        phi_h = torch.from_numpy(case["phi"]).pin_memory().numpy()
        out_h = torch.empty(cells, dtype=torch.float64).pin_memory().numpy()
        e2e_sim = pf.Sim(case["shape"], precision=prec, stream=stream.cuda_stream, **case["params"])
        e2e_sim.init(phi0_h, phi_h)
        e2e_sim.step(S)
        e2e_sim.sync()
        import ctypes as C
        L = pf.load()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(iters):
            e2e_sim.init(phi0_h, phi_h)
            e2e_sim.step(S)
            rc = L.pf_get_macros(e2e_sim._h, C.c_void_p(out_h.ctypes.data), None, None, None, None,
                                 pf.PF_HOST)
            if rc:
                raise pf.PfError(rc, pf.last_error())
        dt = time.perf_counter() - t0
        e2e = {"value": round(cells * S * iters / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": 2 * 8 * cells, "d2h_bytes_per_step": 8 * cells,
               "steps_per_call": S,
               "desc": "pf_init_fields(host phi0, phi) + pf_step(%d) + pf_get_macros(host phi) per "
                       "iteration, wall clock" % S}
        e2e_sim.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline:
        v, n, cores = oracle_mlups(case, budget_s=10.0)
        cpu = {"value": round(v, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "%d full time steps of the %s workload (FP64 C oracle, OpenMP)"
                         % (n, args.workload)}
    line = {
        "metric": "MLUPS", "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"p64": "f64", "p32": "f32", "fp16": "f16 storage / f32 arithmetic",
                  "bf16": "bf16 storage / f32 arithmetic"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "cells": cells, "precision": prec,
                   "desc": case["desc"], "l2": "flushed between timed steps: 512 MiB write, then a 256 MiB read so the write-back happens outside the timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "bytes_per_cell": bpc, "kernel": "k_step2d"},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "cpu_baseline": cpu,
        "wall_s": round(t_wall, 3),
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
