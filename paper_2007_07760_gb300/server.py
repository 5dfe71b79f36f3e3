"""Continuous-batching request server for Allen-Cahn interface-tracking solves.

Requests (grid size, number of steps, velocity field) arrive over time. The
server keeps every admitted grid's state resident on the device inside one
batch (``native.Batch``): all admitted grids advance together, one launch per
step over the tiles of all of them, each grid stopping by itself at its own
step target. At every slice boundary the server

* admits queued requests in arrival order while the device-memory budget and
  the slot limit allow (a request that does not fit waits; later, smaller ones
  are not let past it),
* collects the grids that reached their target (phi copied back, slot freed),
* launches the next slice.

A request whose grid cannot be added fails alone: a non-finite initial field
(DUGKS_ENONFINITE) or any other refusal is recorded as that request's result,
with its status code, and the others go on; DUGKS_ENOMEM is transient while
grids that will finish hold memory, so the request goes back to the head of
the queue until they do; with nothing running but resident grids (which never
finish) it fails at once, as does a request that fits the budget only without
the resident grids.

Time-to-result = completion time - arrival time (queueing included). A grid's
result does not depend on what else is in the batch (bitwise; see the tests).
The backend is any object with the Batch interface, so the policy runs on the
CPU in the tests with a stand-in backend.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import workloads as WL
from .native import DUGKS_ENOMEM


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the trace
    n: int                  # grid side (n x n cells)
    steps: int
    kind: str               # "rotation" (slotted disk) or "vortex" (single vortex)
    phi0: np.ndarray | None = field(default=None, repr=False)   # caller's field (else synthetic)

    @property
    def cells(self) -> int:
        return self.n * self.n


@dataclass
class Result:
    rid: int
    n: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    phi: np.ndarray | None = field(default=None, repr=False)
    error: int = 0          # status code of a request that failed (0: solved)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def poisson_trace(count: int, rate: float = 200.0, seed: int = WL.SEED_BASE + 4, nmin: int = 64,
                  nmax: int = 2048, smin: int = 500, smax: int = 20000) -> list[Request]:
    """Poisson arrivals at `rate` per second; side and step count log-uniform;
    rotation or vortex velocity with probability 1/2 each."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        steps = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        kind = "rotation" if rng.uniform() < 0.5 else "vortex"
        out.append(Request(i, t, n, steps, kind))
    return out


def request_field(req: Request, cfl: float = 0.8, W: float = 4.0, umax: float = 0.05):
    """Initial field and velocity of a request: the slotted disk scaled to the grid
    under rigid rotation, or the drop in the single vortex reversed at the
    request's last step. The rotation makes one revolution over the request's
    steps unless that would exceed the peak speed umax at the box corners (the
    scheme needs |u| well below the lattice speed); then it turns more slowly."""
    n = req.n
    phi0 = req.phi0   # the caller's field, with the kind's velocity; else the synthetic one
    if req.kind == "rotation":
        s = n / 256.0
        if phi0 is None:
            phi0 = WL.slotted_disk(n, 128 * s, 160 * s, 64 * s, 16 * s, 80 * s, W)
        omega = min(2.0 * math.pi / (req.steps * cfl), umax * math.sqrt(2.0) / n)
        return phi0, "rotation", (n / 2, n / 2, omega)
    if phi0 is None:
        phi0 = WL.drops(n, n, [(0.5 * n, 0.75 * n)], [0.15 * n], W)
    return phi0, "vortex", (float(n), umax, req.steps * cfl)


class Server:
    """Admission by device-memory budget and slot count, continuous batching,
    per-request time-to-result."""

    def __init__(self, backend, budget_bytes: int, max_slots: int = 256, slice_steps: int = 64,
                 keep_fields: bool = False, clock=time.perf_counter, sleep=time.sleep, cfl: float = 0.8,
                 W: float = 4.0):
        self.b = backend
        self.budget = budget_bytes
        self.max_slots = max_slots
        self.slice = slice_steps
        self.keep = keep_fields
        self.clock = clock
        self.sleep = sleep
        self.cfl = cfl
        self.W = W
        self.used = 0
        self.peak_used = 0
        self.active = {}          # grid id -> (request, admitted time, bytes)
        self.resident = []        # grid ids that never finish (e.g. a standing large grid)
        self.results: list[Result] = []
        self.cell_updates = 0

    def add_resident(self, phi0: np.ndarray, vel_kind: str, vel) -> int:
        ny, nx = phi0.shape
        nbytes = self.b.grid_bytes(nx, ny)
        if self.used + nbytes > self.budget:
            raise ValueError("resident grid exceeds the budget")
        gid = self.b.add(phi0, vel_kind, vel, -1)
        self.used += nbytes
        self.peak_used = max(self.peak_used, self.used)
        self.resident.append((gid, nx * ny))
        return gid

    def _admit(self, queue: deque, now: float):
        while queue and len(self.active) + len(self.resident) < self.max_slots:
            req = queue[0]
            nbytes = self.b.grid_bytes(req.n, req.n)
            if nbytes > self.budget:
                raise ValueError(f"request {req.rid} can never fit the budget")
            if self.used + nbytes > self.budget:
                if self.active:
                    break   # waits for running grids to free memory
                # only resident grids hold memory and they never finish: it can never fit
                queue.popleft()
                self.results.append(Result(req.rid, req.n, req.steps, req.arrival, now, now, None, DUGKS_ENOMEM))
                continue
            queue.popleft()
            phi0, kind, vel = request_field(req, self.cfl, self.W)
            try:
                gid = self.b.add(phi0, kind, vel, req.steps)
            except Exception as e:   # the backend's error carries the status code
                code = getattr(e, "code", None)
                if code is None:
                    raise
                if code == DUGKS_ENOMEM and self.active:
                    # transient while grids that will finish hold memory: retry once they have
                    # (resident grids never finish, so with only those it fails now)
                    queue.appendleft(req)
                    break
                self.results.append(Result(req.rid, req.n, req.steps, req.arrival, now, now, None, int(code)))
                continue
            self.used += nbytes
            self.peak_used = max(self.peak_used, self.used)
            self.active[gid] = (req, now, nbytes)

    def _collect(self):
        done = [gid for gid, (req, _, _) in self.active.items() if self.b.step_index(gid) >= req.steps]
        for gid in done:
            req, admitted, nbytes = self.active.pop(gid)
            phi = self.b.phi(gid)               # waits for the device
            fin = self.clock() - self.t0
            self.results.append(Result(req.rid, req.n, req.steps, req.arrival, admitted, fin,
                                       phi if self.keep else None))
            self.b.remove(gid)
            self.used -= nbytes

    def run(self, trace: list[Request], time_scale: float = 1.0, max_wall: float | None = None) -> dict:
        """Replays `trace` (arrival times divided by time_scale) until every request
        has finished. Returns throughput and latency statistics."""
        pending = deque(sorted((Request(r.rid, r.arrival / time_scale, r.n, r.steps, r.kind, r.phi0) for r in trace),
                               key=lambda r: r.arrival))
        queue: deque = deque()
        self.t0 = self.clock()
        slices = 0
        while pending or queue or self.active:
            now = self.clock() - self.t0
            if max_wall is not None and now > max_wall:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            self._admit(queue, now)
            if not self.active:
                if pending:
                    self.sleep(max(0.0, min(pending[0].arrival - (self.clock() - self.t0), 0.05)))
                continue
            # cells that advance in this slice (each grid stops at its own target)
            n = self.slice
            for gid, (req, _, _) in self.active.items():
                self.cell_updates += req.cells * max(0, min(n, req.steps - self.b.step_index(gid)))
            for _, cells in self.resident:
                self.cell_updates += cells * n
            self.b.step(n)
            slices += 1
            self._collect()
        wall = self.clock() - self.t0
        status = self.b.status() if hasattr(self.b, "status") else 0
        solved = [r for r in self.results if r.error == 0]
        lat = np.array([r.latency for r in solved]) if solved else np.zeros(1)
        return {"requests": len(self.results), "failed": len(self.results) - len(solved), "wall_s": wall,
                "slices": slices, "solves_per_s": len(solved) / wall if wall > 0 else 0.0,
                "cell_updates_per_s": self.cell_updates / wall if wall > 0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "peak_bytes": self.peak_used, "budget_bytes": self.budget,
                "status": int(status)}
