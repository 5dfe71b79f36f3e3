"""Benchmark of the DUGKS time step on one GB300 (or N replicas under torchrun).

Default workload: single-vortex deformation of a drop on a 1024 x 1024 grid
(FP32, order-3 isotropic upwind reconstruction, two-stage DUGKS, M = 0.02,
W = 4, cfl = 0.8, amplitude 0.05, reversal period 8192 steps). One benchmark
step = one pass of the whole hot path: the fused DUGKS step kernel (cell
quantities, gradients, face reconstruction, face distribution, meso-flux
update, per-tile FP64 mass partials) plus the global FP64 mass reduction. The
state (92 MB) fits in L2, so L2 is flushed (512 MiB write) before every timed
step and only the step itself is timed, with CUDA events on the solver's stream.

Beside the main line (N = 1 only) the same JSON line carries, under "also": the
4096^2 vortex (state far larger than L2), the 512-grid batch (one graph-replayed
launch per step over all grids), the main workload without the L2 flush (state
resident in L2), the 256 x 256 slotted-disk rotation (latency-bound: one partial
wave of tiles), the plain single-grid FP64 GPU step (the generic kernel), the
three-stage, order-4, DVM and LBM steps, each with its own roofline fraction, and
a bounded served measurement (the first 100 arrivals of the request trace, as
recorded and at 70% load: p50/p99 time-to-result, solves/s, cell-updates/s).

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
# Algorithmic bytes per cell-update (the roofline's numerator): the state read once
# and written once per step. Two-stage with d(phi u)/dt: 9 distribution values read
# and written plus phi of the older level read and phi of the new level written.
BYTES_PER_CELL = {"fp64": 160, "fp32": 80, "fp16f": 48}
# three-stage, two kernels per step: 56 values moved between them
BYTES_PER_CELL_T3 = {"fp64": 448, "fp32": 224}
# What this build's kernels actually move per cell (FP32 and FP16 storage keep phi
# of the state as a plane of its own, read as well: +4 B; three-stage: the phi
# planes of tilde f' and of the accumulator as well)
BYTES_PER_CELL_ACTUAL = {("fp64", 2): 160, ("fp32", 2): 84, ("fp16f", 2): 48, ("fp64", 3): 456, ("fp32", 3): 248,
                         ("fp64", 1): 160, ("fp32", 1): 80}
# the streaming-collision DVM (stages = 1) moves the same state as the two-stage step:
# 9 values read and written, phi of the older level read, the new phi written


def bytes_per_cell(precision: str, stages: int) -> int:
    return BYTES_PER_CELL[precision] if stages <= 2 else BYTES_PER_CELL_T3[precision]
L2_FLUSH_BYTES = 512 << 20

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, bytes) of one step
# kernel launch from one ncu capture, keyed by the hash of the kernel sources it
# was taken on and the workload (reported as null once the sources change). The
# writes of a 1024^2 step stay in L2 (129 MB) during the launch and reach DRAM
# later, so the figure is the read traffic plus the evictions.
NCU_TRAFFIC = {
    ("ec6fb138f47ce3e2", "vortex1024_fp32_p3_upwind_2stage"): 49932288,     # mean of two launches
    ("ec6fb138f47ce3e2", "vortex4096_fp32_p3_upwind_2stage"): 1383666688,   # state 11x the L2
    ("ec6fb138f47ce3e2", "batch512_fp32_p3_upwind_2stage"): 3279676416,     # 1.20x: halos of small grids
}


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
        # vortex<n>[_p<order>][_central][_t3 | _dvm | _lbm]: the three-stage scheme at cfl 0.5 (it needs
        # dt < 12 tau); the streaming-collision DVM at cfl 0.8, the LBM (the DVM at cfl 1)
        parts = name.split("_")
        n = int(parts[0][len("vortex"):] or 1024)
        order = next((int(q[1:]) for q in parts[1:] if q.startswith("p")), 3)
        flux = 1 if "central" in parts[1:] else 0
        stages = 3 if "t3" in parts[1:] else 1 if ("dvm" in parts[1:] or "lbm" in parts[1:]) else 2
        cfl = 0.5 if stages == 3 else 1.0 if "lbm" in parts[1:] else 0.8
        prob = WL.vortex1024(order=order, flux=flux, stages=stages, cfl=cfl, n=n)
        prob.name = parts[0] + ("_lbm" if "lbm" in parts[1:] else "_dvm" if "dvm" in parts[1:] else "")
    elif name == "drop64":
        prob = WL.drop64()
    else:
        raise SystemExit(f"unknown workload {name}")
    scheme = (f"{'upwind' if prob.flux == 0 else 'central'}_{prob.stages}stage" if prob.stages > 1 else
              "streaming_collision")
    desc = {"workload": f"{prob.name}_{precision}_p{prob.order}_{scheme}",
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


def max_over_ranks(x: float, dist=None) -> float:
    """The job's time is its slowest rank's: all-reduce MAX over the process group
    (a CUDA tensor under NCCL, a host tensor under gloo); x itself without one."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: the units all ranks processed
    over the slowest rank's time."""
    return units_per_rank * world / seconds


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


def time_single(solver, stream, warmup: int, K: int, dist=None, local: int = 0, flush_l2: bool = True):
    """W untimed and K timed steps of one solver, L2 flushed before each (unless
    flush_l2 is false: a state larger than L2, or the L2-resident comparison). One
    step = the step kernel (per-tile FP64 mass partials) + the kernel that sums
    them; the second is launched as a programmatic dependent of the first, so no
    event sits between them in the timed pass. A second pass of K steps, with
    events around the step kernel alone, gives its duration for the roofline."""
    import torch
    from paper_2007_07760_gb300 import native as N

    mass_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4 if flush_l2 else 1, dtype=torch.float32, device="cuda")

    def ev():
        return torch.cuda.Event(enable_timing=True)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            if flush_l2:
                flush.zero_()
            N.dugks_step(solver.ctx, 1)
            N.dugks_mass_device(solver.ctx, mass_dev.data_ptr())
    stream.synchronize()
    whole = [(ev(), ev()) for _ in range(K)]
    kern = [(ev(), ev()) for _ in range(K)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for a, b in whole:
                if flush_l2:
                    flush.zero_()
                a.record(stream)
                N.dugks_step(solver.ctx, 1)
                N.dugks_mass_device(solver.ctx, mass_dev.data_ptr())
                b.record(stream)
            for a, b in kern:
                if flush_l2:
                    flush.zero_()
                a.record(stream)
                N.dugks_step(solver.ctx, 1)
                b.record(stream)
                N.dugks_mass_device(solver.ctx, mass_dev.data_ptr())
        stream.synchronize()
    torch.cuda.synchronize()
    clocks = clk.summary()
    del flush
    if N.dugks_status(solver.ctx) != 0:
        raise SystemExit("device error: " + N.dugks_last_error(solver.ctx))
    mass = float(mass_dev.item())
    if not math.isfinite(mass):
        raise SystemExit("non-finite mass")
    return {"total_ms": sum(a.elapsed_time(b) for a, b in whole),
            "avg_step_ms": sum(a.elapsed_time(b) for a, b in kern) / K, "clocks": clocks, "mass": mass}


def also_single(name: str, precision: str, K: int, generic: bool = False, flush_l2: bool = True,
                tune: bool = False):
    """Secondary single-grid measurement for the "also" list of the JSON line."""
    import torch
    from paper_2007_07760_gb300 import native as N

    prob, desc = workload(name, precision)
    stream = torch.cuda.Stream()
    variant = None
    if tune and not generic:
        from paper_2007_07760_gb300 import autotune
        with N.Solver.from_problem(prob, precision=precision, stream=stream.cuda_stream) as solver:
            variant = autotune.tune(solver, "single", prob.cells)
    with N.Solver.from_problem(prob, precision=precision, stream=stream.cuda_stream) as solver:
        if generic:
            solver.set_variant(-1)
        elif variant is not None:
            solver.set_variant(variant)
        r = time_single(solver, stream, 10, K, flush_l2=flush_l2)
    peak, _ = measured_peak_hbm()
    bpc = bytes_per_cell(precision, prob.stages)
    achieved = bpc * prob.cells / (r["avg_step_ms"] * 1e-3) / 1e9
    state_mb = BYTES_PER_CELL_ACTUAL[(precision, prob.stages)] * prob.cells / 1e6
    # the recorded traffic holds for the regime it was captured in: a flushed L2, or a
    # state too large for L2 to matter (an L2-resident run reads far less DRAM)
    traffic = (NCU_TRAFFIC.get((kernel_source_hash(), desc["workload"]))
               if not generic and (flush_l2 or state_mb > 400) else None)
    out = {"workload": desc["workload"] + ("_generic_kernel" if generic else ""), "bytes_per_cell": bpc,
           "bytes_per_cell_actual": BYTES_PER_CELL_ACTUAL[(precision, prob.stages)],
           "value": prob.cells * K / (r["total_ms"] * 1e-3), "unit": UNIT, "steps": K,
           "ms_per_step": r["total_ms"] / K,
           "l2": ("flushed before every timed step" if flush_l2 else
                  f"not flushed: steps back to back ({state_mb:.0f} MB of state"
                  + (", far larger than the 129 MB L2)" if state_mb > 400 else ", L2-resident)")),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": traffic, "avg_kernel_ms": r["avg_step_ms"]},
           "clocks": r["clocks"]}
    if variant is not None:
        out["tile_variant"] = variant
    return out


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

    if args.workload.startswith("batch"):
        run_batch(args, dist, world, rank, local)
        if dist:
            dist.destroy_process_group()
        return
    prob, desc = workload(args.workload, args.precision)
    # cpu baseline first (oracle process-local, before heavy GPU use), rank 0, N = 1 only
    cpu = cpu_baseline(prob) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    stream = torch.cuda.Stream()
    solver = N.Solver.from_problem(prob, precision=args.precision, stream=stream.cuda_stream)
    if args.generic:
        solver.set_variant(-1)
        desc["kernel"] = "generic step_kernel (plain comparison path)"
    elif args.variant is not None:
        solver.set_variant(args.variant)
        desc["tile_variant"] = args.variant
    elif prob.stages == 2 and prob.order <= 3:
        from paper_2007_07760_gb300 import autotune
        desc["tile_variant"] = autotune.tune(solver, "single", prob.cells)
        # the tuning steps advanced the state: start the timed run from the initial field
        solver.close()
        solver = N.Solver.from_problem(prob, precision=args.precision, stream=stream.cuda_stream)
        solver.set_variant(desc["tile_variant"])
    K = args.steps
    res = time_single(solver, stream, args.warmup, K, dist, local)
    total_ms, avg_step_ms, clocks, mass = res["total_ms"], res["avg_step_ms"], res["clocks"], res["mass"]
    total_ms = max_over_ranks(total_ms, dist)
    if dist:
        dist.barrier()

    value = job_rate(prob.cells * K, world, total_ms * 1e-3)
    peak, peak_kind = measured_peak_hbm()
    bpc = bytes_per_cell(args.precision, prob.stages)
    achieved = bpc * prob.cells / (avg_step_ms * 1e-3) / 1e9
    sha = kernel_source_hash()
    traffic = NCU_TRAFFIC.get((sha, desc["workload"]))

    # end to end through the C ABI with host buffers: per step the state comes
    # from pinned host memory, one step runs, phi is read back to host
    nbytes = N.dugks_state_bytes(solver.ctx)
    host_state = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    idx = N.dugks_save_state(solver.ctx, host_state)
    phi_host = torch.empty((prob.ny, prob.nx), dtype=torch.float64, pin_memory=True).numpy()
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
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    tsize = 8 if args.precision == "fp64" else 4
    e2e = {"value": job_rate(prob.cells * Ke, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": prob.cells * tsize, "steps": Ke,
           "path": "dugks_load_state(pinned host) + dugks_step + dugks_read_phi(host)"}
    solver.close()

    if rank == 0:
        launches_per_step = 3 if prob.stages == 3 else 2
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16f": "f32 (f16 storage)"}[args.precision],
            "data": "synthetic",
            "config": dict(desc, l2="flushed before every timed step (512 MiB write, untimed); the step's 88 MB "
                                    "of writes then stay in L2 during the launch and reach DRAM during the next "
                                    "flush, so the DRAM traffic of a launch is its reads (see the 4096^2 line in "
                                    "'also' for a state far larger than L2)",
                           mass="FP64 per-tile partials in the step kernel + fixed-order sum kernel",
                           replicas=world, parallelism="replicas" if world > 1 else "single"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": desc.get("kernel", "step_fast_kernel (TMA-staged fused two-stage DUGKS step)"
                                            if prob.stages == 2 else
                                            "step_fast_kernel KIND_T3A + KIND_T3B (the two kernels of a three-stage step)"
                                            if prob.stages == 3 else "dvm_step_kernel (streaming-collision DVM)"),
                         "bytes_per_cell": bpc,
                         "bytes_per_cell_actual": BYTES_PER_CELL_ACTUAL[(args.precision, prob.stages)],
                         "peak_source": peak_kind, "avg_kernel_ms": avg_step_ms},
            "e2e": e2e,
            "gpu_launches": launches_per_step * K,
            "clocks": clocks,
            "final_mass": mass,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if world == 1 and not args.no_also:
            line["also"] = [also_single("vortex4096", "fp32", 30, flush_l2=False, tune=True),
                            also_batch(512, "fp32", 64),
                            also_single(args.workload, args.precision, 100, flush_l2=False),
                            also_single("slotted_disk256", "fp32", 300),
                            also_single(args.workload, "fp64", 20, generic=True),
                            also_single("vortex1024_t3", "fp32", 50), also_single("vortex1024_p4", "fp32", 50),
                            also_single("vortex1024_dvm", "fp32", 50), also_single("vortex1024_lbm", "fp32", 50),
                            also_serve(100)]
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measure_batch(count: int, precision: str, warmup: int, K: int, dist=None, local: int = 0):
    """Many independent grids (sides log-uniform 64..512, 1-8 drops, uniform velocity
    |u| <= 0.05) advanced together: one launch per step over a work list of tiles
    of all grids, replayed as CUDA graphs, tile variant picked by the autotuner.
    The state of 512 grids (2.3 GB in FP32) is far larger than L2, so no flush is
    needed between steps."""
    import torch
    from paper_2007_07760_gb300 import autotune
    from paper_2007_07760_gb300 import native as N

    probs = WL.random_batch(count=count)
    p0 = probs[0]
    stream = torch.cuda.Stream()
    desc = {"workload": f"batch{count}_{precision}_p{p0.order}_upwind_2stage", "grids": count,
            "sides": "log-uniform 64..512 (seeded)", "precision": precision, "order": p0.order,
            "flux": "upwind", "stages": 2, "M": p0.M, "cfl": p0.cfl, "W": p0.W,
            "velocity": "uniform, random angle, |u| <= 0.05"}
    cells = sum(q.cells for q in probs)
    desc["cells"] = cells
    t_e2e0 = time.perf_counter()
    batch = N.Batch(precision=precision, W=p0.W, M=p0.M, cfl=p0.cfl, order=p0.order, flux=0, stages=2,
                    stream=stream.cuda_stream)
    ids = [batch.add(q.phi0, q.vel_kind, q.vel) for q in probs]
    t_add = time.perf_counter() - t_e2e0
    variant = autotune.tune(batch, "batch", cells)
    desc["tile_variant"] = variant
    desc["l2"] = "no flush: the state of all grids is larger than L2"
    batch.step(warmup)
    batch.status()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            batch.step(K)
            ev1.record(stream)
        stream.synchronize()
    clocks = clk.summary()
    total_ms = ev0.elapsed_time(ev1)
    if batch.status() != 0:
        raise SystemExit("device error: " + N.dugks_batch_last_error(batch.b))
    # end to end: host fields in (dugks_batch_add), the same K steps, every phi back to host
    t0 = time.perf_counter()
    outs = [batch.phi(i) for i in ids]
    t_read = time.perf_counter() - t0
    batch.close()
    del outs
    return {"desc": desc, "cells": cells, "total_ms": total_ms, "clocks": clocks,
            "e2e_s": t_add + total_ms * 1e-3 + t_read}


def run_batch(args, dist, world, rank, local):
    import torch

    count = int(args.workload[len("batch"):] or 512)
    K = args.steps
    r = measure_batch(count, args.precision, args.warmup, K, dist, local)
    total_ms, cells, desc = r["total_ms"], r["cells"], r["desc"]
    total_ms = max_over_ranks(total_ms, dist)
    e2e_s = max_over_ranks(r["e2e_s"], dist)
    value = job_rate(cells * K, world, total_ms * 1e-3)
    peak, peak_kind = measured_peak_hbm()
    bpc = BYTES_PER_CELL[args.precision]
    achieved = bpc * cells / (total_ms / K * 1e-3) / 1e9
    tsize = 8 if args.precision == "fp64" else 4
    traffic = NCU_TRAFFIC.get((kernel_source_hash(), desc["workload"]))
    e2e = {"value": job_rate(cells * K, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(cells * 8 / K), "d2h_bytes_per_step": int(cells * tsize / K),
           "path": "dugks_batch_add from host fields + K steps + dugks_batch_read_phi of every grid, amortised over K"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16f": "f32 (f16 storage)"}[args.precision],
            "data": "synthetic", "config": desc,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "kernel": "batch_fast_kernel + batch_advance_kernel (graph-replayed)",
                         "bytes_per_cell": bpc, "bytes_per_cell_actual": BYTES_PER_CELL_ACTUAL[(args.precision, 2)],
                         "peak_source": peak_kind},
            "e2e": e2e, "gpu_launches": 2 * K, "clocks": r["clocks"],
        }
        print(json.dumps(line), flush=True)


def also_batch(count: int, precision: str, K: int):
    r = measure_batch(count, precision, 8, K)
    peak, _ = measured_peak_hbm()
    achieved = BYTES_PER_CELL[precision] * r["cells"] / (r["total_ms"] / K * 1e-3) / 1e9
    traffic = NCU_TRAFFIC.get((kernel_source_hash(), r["desc"]["workload"]))
    return {"workload": r["desc"]["workload"], "value": r["cells"] * K / (r["total_ms"] * 1e-3), "unit": UNIT,
            "steps": K, "ms_per_step": r["total_ms"] / K, "cells": r["cells"],
            "tile_variant": r["desc"]["tile_variant"], "bytes_per_cell": BYTES_PER_CELL[precision],
            "bytes_per_cell_actual": BYTES_PER_CELL_ACTUAL[(precision, 2)],
            "l2": "no flush: the state of all grids is larger than L2",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic},
            "clocks": r["clocks"]}


# serving lanes, highest priority first: (work limit in cell-updates, slice steps,
# stream priority); the resident grid runs alone in a lowest-priority lane
SERVE_LANES = ((1e8, 256, -3), (2e9, 128, -2), (None, 64, -1))
RESIDENT_LANE = (32, 0)


def serve_passes(requests: int, budget_gb: float, resident: bool, local: int) -> dict:
    """Continuous-batching server on a seeded Poisson trace of `requests` arrivals
    (200 requests/s, sides log-uniform 64..2048, 500..20000 steps, rotation or
    vortex), FP32 order-3 upwind, with a resident 4096^2 vortex grid. Requests are
    served in priority lanes by work (cells x steps), each lane a batch on its own
    stream running one CTA per tile. The trace offers far more work than one GPU
    does, so it is replayed twice: as recorded (overloaded: the latencies are
    mostly queueing) and with arrivals stretched so that the offered load is 70%
    of the throughput measured in the first pass."""
    import torch
    from paper_2007_07760_gb300 import native as N
    from paper_2007_07760_gb300 import server as S

    trace = S.poisson_trace(requests, rate=200.0)
    # a request arrives with its field: the clients' fields are made before the replay
    trace = [S.Request(r.rid, r.arrival, r.n, r.steps, r.kind, S.request_field(r)[0]) for r in trace]
    work = sum(r.cells * r.steps for r in trace)
    common = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2, precision="fp32")
    warm = WL.drops(64, 64, [(32.0, 40.0)], [12.0], 4.0)
    passes = {}
    for name, scale in (("recorded", 1.0), ("load70", None)):
        if scale is None:
            cap = passes["recorded"]["cell_updates_per_s"]
            offered = work / trace[-1].arrival
            scale = min(1.0, 0.7 * cap / offered)
        specs = [(lim, sl, pr) for lim, sl, pr in SERVE_LANES]
        if resident:
            specs.append((None, RESIDENT_LANE[0], RESIDENT_LANE[1]))
        streams = [torch.cuda.Stream(priority=pr) for _, _, pr in specs]
        batches = [N.Batch(stream=st.cuda_stream, **common) for st in streams]
        try:
            for b in batches:
                b.set_ctas(-1)
                # first use of each kernel outside the replay (module loading waits for the device)
                g = b.add(warm, "vortex", (64.0, 0.05, 100.0), 8)
                b.step(8)
                b.retire(g)
                b.collect(g, wait=True)
            lanes = [S.Lane(b, lim, sl) for b, (lim, sl, _) in zip(batches, specs)]
            srv = S.Server(lanes, budget_bytes=int(budget_gb * (1 << 30)), max_slots=512)
            if resident:
                big = WL.vortex1024(n=4096)
                srv.add_resident(big.phi0, big.vel_kind, big.vel)
            with ClockSampler(local) as clk:
                st = srv.run(trace, time_scale=scale)
            st["clocks"] = clk.summary()
            st["time_scale"] = scale
            st["offered_cell_updates_per_s"] = work / (trace[-1].arrival / scale)
            passes[name] = st
        finally:
            for b in batches:
                b.close()
    return {"trace": {"requests": requests, "rate_per_s": 200.0, "sides": "log-uniform 64..2048",
                      "steps": "log-uniform 500..20000", "request_cell_updates": work},
            "lanes": [{"max_work": lim, "slice_steps": sl, "stream_priority": pr} for lim, sl, pr in SERVE_LANES]
            + ([{"resident": "4096x4096 vortex", "slice_steps": RESIDENT_LANE[0],
                 "stream_priority": RESIDENT_LANE[1]}] if resident else []),
            "budget_gb": budget_gb, "passes": passes}


def also_serve(requests: int) -> dict:
    """Bounded served measurement for the "also" list: the first `requests`
    arrivals of the trace, recorded and at 70% load."""
    r = serve_passes(requests, 32.0, True, 0)
    rec, l70 = r["passes"]["recorded"], r["passes"]["load70"]
    keep = ("requests", "failed", "wall_s", "solves_per_s", "cell_updates_per_s", "p50_s", "p99_s", "mean_s",
            "time_scale", "offered_cell_updates_per_s", "status", "lanes", "clocks")
    return {"workload": f"serve{requests}_fp32_p3_upwind_2stage", "metric": "served D2Q9 cell-updates/s",
            "value": rec["cell_updates_per_s"], "unit": UNIT, "solves_per_s": rec["solves_per_s"],
            "p50_s": rec["p50_s"], "p99_s": rec["p99_s"],
            "load70": {k: l70[k] for k in keep if k in l70}, "recorded": {k: rec[k] for k in keep if k in rec},
            "trace": r["trace"], "lanes": r["lanes"]}


def run_serve(args, local):
    """The served line of its own (bench.py --workload serve --requests R)."""
    r = serve_passes(args.requests, args.budget_gb, not args.no_resident, local)
    rec = r["passes"]["recorded"]
    line = {"metric": "served D2Q9 cell-updates/s", "value": rec["cell_updates_per_s"], "unit": UNIT,
            "n_gpus": 1, "steps": None, "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"serve{args.requests}_fp32_p3_upwind_2stage", "requests": args.requests,
                       "rate_per_s": 200.0, "sides": "log-uniform 64..2048", "steps": "log-uniform 500..20000",
                       "resident_grid": None if args.no_resident else "4096x4096 vortex",
                       "budget_gb": args.budget_gb, "lanes": r["lanes"]},
            "serving": r["passes"],
            "clocks": rec["clocks"], "gpu_launches": None}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vortex1024")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16f"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-also", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--variant", type=int, default=None, help="fixed tile variant (default: autotuned)")
    ap.add_argument("--generic", action="store_true", help="time the generic (plain) kernel instead")
    ap.add_argument("--requests", type=int, default=48, help="serve workload: requests in the trace")
    ap.add_argument("--budget-gb", type=float, default=32.0, help="serve workload: device-memory budget")
    ap.add_argument("--no-resident", action="store_true", help="serve workload: no standing 4096^2 grid")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        run_serve(args, int(os.environ.get("LOCAL_RANK", "0")))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
