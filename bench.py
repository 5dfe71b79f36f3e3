"""Benchmark of the DUGKS time step on one GB300 (or N replicas under torchrun).

Default workload: the 256 x 256 slotted disk under rigid rotation (FP32,
order-3 isotropic upwind reconstruction, two-stage DUGKS, M = 0.002, W = 4,
cfl = 0.8). One benchmark step = one pass of the whole hot path: the fused
DUGKS step kernel (cell quantities, gradients, face reconstruction, face
distribution, meso-flux update, per-tile mass partials) plus the global FP64
mass reduction. The state (2.6 MB) fits in L2, so L2 is flushed (512 MiB write)
before every timed step and only the step itself is timed, with CUDA events on
the solver's stream.

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle instead
(the baseline program for this method) on the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2007_07760_gb300 import workloads as WL  # noqa: E402

METRIC = "D2Q9 cell-updates/s"
UNIT = "cell-updates/s"
BYTES_PER_CELL = {"fp64": 160, "fp32": 80, "fp16f": 48}   # two-stage, with d(phi u)/dt
L2_FLUSH_BYTES = 512 << 20

# DRAM traffic of the step kernel from one ncu capture, keyed by the hash of the
# kernel sources it was taken on (reported as null once the sources change).
NCU_TRAFFIC = {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_07760_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def workload(name: str, precision: str):
    if name == "slotted_disk256":
        prob = WL.slotted_disk256(order=3, flux=0, stages=2)
    elif name.startswith("vortex"):
        n = int(name[len("vortex"):] or 1024)
        prob = WL.vortex1024(order=3, flux=0, stages=2, n=n)
        prob.name = name
    elif name == "drop64":
        prob = WL.drop64()
    else:
        raise SystemExit(f"unknown workload {name}")
    desc = {"workload": f"{prob.name}_{precision}_p{prob.order}_{'upwind' if prob.flux == 0 else 'central'}"
                        f"_{prob.stages}stage",
            "nx": prob.nx, "ny": prob.ny, "order": prob.order,
            "flux": "upwind" if prob.flux == 0 else "central", "stages": prob.stages,
            "precision": precision, "W": prob.W, "M": prob.M, "cfl": prob.cfl, "velocity": prob.vel_kind}
    return prob, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(prob, budget_s: float = 20.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the
    same workload (the full grid, as many whole steps as fit the budget)."""
    import oracle as O
    O.build()
    p = O.Params(prob.nx, prob.ny, W=prob.W, M=prob.M, cfl=prob.cfl, order=prob.order, flux=prob.flux,
                 stages=prob.stages, dtphiu=prob.dtphiu, vel_kind=prob.vel_kind, vel=prob.vel)
    s = O.State(p, prob.phi0)
    t0 = time.perf_counter()
    s.run(1)
    one = time.perf_counter() - t0
    nsteps = max(1, min(1000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    s.run(nsteps)
    dt = time.perf_counter() - t0
    return {"value": prob.cells * nsteps / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{nsteps} full steps of the {prob.nx}x{prob.ny} grid in FP64 ({dt:.1f} s)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob, desc = workload(args.workload, args.precision)
    import oracle as O
    O.build()
    p = O.Params(prob.nx, prob.ny, W=prob.W, M=prob.M, cfl=prob.cfl, order=prob.order, flux=prob.flux,
                 stages=prob.stages, dtphiu=prob.dtphiu, vel_kind=prob.vel_kind, vel=prob.vel)
    s = O.State(p, prob.phi0)
    t0 = time.perf_counter()
    s.run(1)
    one = time.perf_counter() - t0
    # bounded sample: every step is one full oracle step; at most ~90 s of timed work
    warm = min(args.warmup, 3)
    s.run(warm)
    k = max(1, min(args.steps, int(90.0 / max(one, 1e-6))))
    t0 = time.perf_counter()
    s.run(k)
    dt = time.perf_counter() - t0
    value = prob.cells * k / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": k, "warmup": warm, "ms_per_step": 1e3 * dt / k, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{k} full steps of the {prob.nx}x{prob.ny} grid in FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2007_07760_gb300 import native as N

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prob, desc = workload(args.workload, args.precision)
    # cpu baseline first (oracle process-local, before heavy GPU use), rank 0, N = 1 only
    cpu = cpu_baseline(prob) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    stream = torch.cuda.Stream()
    solver = N.Solver.from_problem(prob, precision=args.precision, stream=stream.cuda_stream)
    mass_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step():
        N.dugks_step(solver.ctx, 1)
        N.dugks_mass_device(solver.ctx, mass_dev.data_ptr())

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            one_step()
    stream.synchronize()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(K):
                flush.zero_()
                ev[i][0].record(stream)
                N.dugks_step(solver.ctx, 1)
                ev[i][1].record(stream)
                N.dugks_mass_device(solver.ctx, mass_dev.data_ptr())
                ev[i][2].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    clocks = clk.summary()
    step_ms = [a.elapsed_time(b) for a, b, _ in ev]
    total_ms = sum(a.elapsed_time(c) for a, _, c in ev)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    if N.dugks_status(solver.ctx) != 0:
        raise SystemExit("device error: " + N.dugks_last_error(solver.ctx))
    mass = float(mass_dev.item())
    if not math.isfinite(mass):
        raise SystemExit("non-finite mass")

    value = prob.cells * K * world / (total_ms * 1e-3)
    avg_step_ms = sum(step_ms) / K
    peak, peak_kind = measured_peak_hbm()
    achieved = BYTES_PER_CELL[args.precision] * prob.cells / (avg_step_ms * 1e-3) / 1e9
    sha = kernel_source_hash()
    traffic = NCU_TRAFFIC.get((sha, desc["workload"]))

    # end to end through the C ABI with host buffers: per step the state comes
    # from pinned host memory, one step runs, phi is read back to host
    nbytes = N.dugks_state_bytes(solver.ctx)
    host_state = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    idx = N.dugks_save_state(solver.ctx, host_state)
    phi_host = np.empty((prob.ny, prob.nx))
    Ke = max(10, min(K, 500))
    for _ in range(3):
        N.dugks_load_state(solver.ctx, host_state, idx)
        N.dugks_step(solver.ctx, 1)
        N.dugks_read_phi(solver.ctx, phi_host)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(Ke):
        N.dugks_load_state(solver.ctx, host_state, idx)
        N.dugks_step(solver.ctx, 1)
        N.dugks_read_phi(solver.ctx, phi_host)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    tsize = 8 if args.precision == "fp64" else 4
    e2e = {"value": prob.cells * Ke * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": prob.cells * tsize, "steps": Ke,
           "path": "dugks_load_state(pinned host) + dugks_step + dugks_read_phi(host)"}
    solver.close()

    if rank == 0:
        launches_per_step = 2 if prob.stages == 2 else 3
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16f": "f32 (f16 storage)"}[args.precision],
            "data": "synthetic",
            "config": dict(desc, l2="flushed before every timed step (512 MiB write, untimed)",
                           replicas=world, parallelism="replicas" if world > 1 else "single"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "step_kernel (fused two-stage DUGKS step)",
                         "bytes_per_cell": BYTES_PER_CELL[args.precision], "peak_source": peak_kind,
                         "avg_kernel_ms": avg_step_ms},
            "e2e": e2e,
            "gpu_launches": launches_per_step * K,
            "clocks": clocks,
            "final_mass": mass,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="slotted_disk256")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16f"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
