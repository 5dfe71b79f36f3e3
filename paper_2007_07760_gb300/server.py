"""Continuous-batching request server for Allen-Cahn interface-tracking solves.

Requests (grid size, number of steps, velocity field) arrive over time. Every
admitted grid's state stays resident on the device inside a batch
(``native.Batch``): one launch per step advances all grids of a batch over the
tiles of all of them, each grid stopping by itself at its own step target.

Requests are served in lanes: each lane is a batch on its own CUDA stream, and a
request goes to the first lane whose work limit (cells x steps) it fits. The
lanes' streams carry decreasing priority and their kernels run one CTA per tile,
so the GPU takes the tiles of a higher lane first as soon as tiles of a lower
one finish: short solves are not held to the step rate of the large grids
(nor of a resident grid that never finishes, which sits in the lowest lane).
Within a lane all grids advance together.

The host never waits for the device while serving. For each lane it keeps at
most `depth` slices (a slice: `slice_steps` steps of the lane) in flight, with a
fence after each; a grid whose target falls within a queued slice is retired at
once (its read-out queued behind that slice into pinned host memory) and its
result collected, and its memory released, once the read-out has landed. Between
polls the server admits queued requests in arrival order while the
device-memory budget and the slot limit allow (a request that does not fit
waits; later, smaller ones are not let past it).

A request whose grid cannot be added fails alone: a non-finite initial field
(DUGKS_ENONFINITE) or any other refusal is recorded as that request's result,
with its status code, and the others go on; DUGKS_ENOMEM is transient while
grids that will finish hold memory, so the request goes back to the head of
the queue until they do; with nothing running but resident grids (which never
finish) it fails at once, as does a request that fits the budget only without
the resident grids.

Time-to-result = completion time - arrival time (queueing included). A grid's
result does not depend on what else is in the batch or on its lane (bitwise;
see the tests). The backend is any object with the Batch interface, so the
policy runs on the CPU in the tests with a stand-in backend.
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
        omega = min(2.0 * math.pi / (max(req.steps, 1) * cfl), umax * math.sqrt(2.0) / n)
        return phi0, "rotation", (n / 2, n / 2, omega)
    if phi0 is None:
        phi0 = WL.drops(n, n, [(0.5 * n, 0.75 * n)], [0.15 * n], W)
    return phi0, "vortex", (float(n), umax, max(req.steps, 1) * cfl)   # (a zero-step request: T of one step)


@dataclass
class Lane:
    """One batch on one stream: requests of at most `max_work` cell-updates
    (None: any), advanced `slice_steps` steps per slice."""
    backend: object
    max_work: float | None = None
    slice_steps: int = 64
    active: dict = field(default_factory=dict)      # grid id -> (request, admitted time, bytes)
    retiring: dict = field(default_factory=dict)    # grid id -> (request, admitted time, bytes)
    resident: list = field(default_factory=list)    # (grid id, cells) of grids that never finish
    inflight: deque = field(default_factory=deque)  # fence tickets of queued slices
    slices: int = 0
    resident_steps: int = 0

    def has_work(self) -> bool:
        return bool(self.active or self.resident)


class Server:
    """Admission by device-memory budget and slot count, continuous batching in
    priority lanes, per-request time-to-result.

    `backend` is one batch (a single lane) or a list of lanes, highest priority
    first: Lane objects or (batch, max_work) / (batch, max_work, slice_steps)
    tuples; the last lane takes any request and the resident grids."""

    def __init__(self, backend, budget_bytes: int, max_slots: int = 256, slice_steps: int = 64,
                 keep_fields: bool = False, clock=time.perf_counter, sleep=time.sleep, cfl: float = 0.8,
                 W: float = 4.0, depth: int = 2, poll_s: float = 2e-4):
        lanes = backend if isinstance(backend, (list, tuple)) else [backend]
        self.lanes = []
        for ln in lanes:
            if isinstance(ln, Lane):
                self.lanes.append(ln)
            elif isinstance(ln, tuple):
                self.lanes.append(Lane(ln[0], ln[1], ln[2] if len(ln) > 2 else slice_steps))
            else:
                self.lanes.append(Lane(ln, None, slice_steps))
        self.lanes[-1].max_work = None
        self.budget = budget_bytes
        self.max_slots = max_slots
        self.keep = keep_fields
        self.clock = clock
        self.sleep = sleep
        self.cfl = cfl
        self.W = W
        self.depth = depth
        self.poll_s = poll_s
        self.used = 0
        self.peak_used = 0
        self.results: list[Result] = []
        self.cell_updates = 0

    # grids admitted and not yet collected, over all lanes
    def _live(self) -> int:
        return sum(len(ln.active) + len(ln.retiring) for ln in self.lanes)

    def _slots(self) -> int:
        return self._live() + sum(len(ln.resident) for ln in self.lanes)

    def _lane_for(self, req: Request) -> Lane:
        work = req.cells * req.steps
        for ln in self.lanes:
            if ln.max_work is None or work <= ln.max_work:
                return ln
        return self.lanes[-1]

    def add_resident(self, phi0: np.ndarray, vel_kind: str, vel) -> int:
        ny, nx = phi0.shape
        ln = self.lanes[-1]
        nbytes = ln.backend.grid_bytes(nx, ny)
        if self.used + nbytes > self.budget:
            raise ValueError("resident grid exceeds the budget")
        gid = ln.backend.add(phi0, vel_kind, vel, -1)
        self.used += nbytes
        self.peak_used = max(self.peak_used, self.used)
        ln.resident.append((gid, nx * ny))
        return gid

    def _admit(self, queue: deque, now: float):
        while queue and self._slots() < self.max_slots:
            req = queue[0]
            ln = self._lane_for(req)
            nbytes = ln.backend.grid_bytes(req.n, req.n)
            if nbytes > self.budget:
                raise ValueError(f"request {req.rid} can never fit the budget")
            if self.used + nbytes > self.budget:
                if self._live():
                    break   # waits for running grids to free memory
                # only resident grids hold memory and they never finish: it can never fit
                queue.popleft()
                self.results.append(Result(req.rid, req.n, req.steps, req.arrival, now, now, None, DUGKS_ENOMEM))
                continue
            queue.popleft()
            phi0, kind, vel = request_field(req, self.cfl, self.W)
            try:
                gid = ln.backend.add(phi0, kind, vel, req.steps)
            except Exception as e:   # the backend's error carries the status code
                code = getattr(e, "code", None)
                if code is None:
                    raise
                if code == DUGKS_ENOMEM and self._live():
                    # transient while grids that will finish hold memory: retry once they have
                    # (resident grids never finish, so with only those it fails now)
                    queue.appendleft(req)
                    break
                self.results.append(Result(req.rid, req.n, req.steps, req.arrival, now, now, None, int(code)))
                continue
            self.used += nbytes
            self.peak_used = max(self.peak_used, self.used)
            ln.active[gid] = (req, now, nbytes)

    def _collect(self) -> bool:
        """Results whose read-out has landed (no wait)."""
        got = False
        for ln in self.lanes:
            for gid in list(ln.retiring):
                phi = ln.backend.collect(gid)
                if phi is None:
                    continue
                req, admitted, nbytes = ln.retiring.pop(gid)
                fin = self.clock() - self.t0
                self.results.append(Result(req.rid, req.n, req.steps, req.arrival, admitted, fin,
                                           phi if self.keep else None))
                self.used -= nbytes
                got = True
        return got

    def _feed(self, ln: Lane) -> bool:
        """Queues one more slice of lane `ln` if it has work and room in flight."""
        b = ln.backend
        while ln.inflight and b.reached(ln.inflight[0]):
            ln.inflight.popleft()
        if not ln.has_work() or len(ln.inflight) >= self.depth:
            return False
        n = ln.slice_steps
        for gid, (req, _, _) in ln.active.items():
            self.cell_updates += req.cells * max(0, min(n, req.steps - b.step_index(gid)))
        for _, cells in ln.resident:
            self.cell_updates += cells * n
        ln.resident_steps += n if ln.resident else 0
        b.step(n)
        ln.inflight.append(b.fence())
        ln.slices += 1
        # grids whose target falls in this slice: read-out queued behind it
        for gid in [g for g, (req, _, _) in ln.active.items() if b.step_index(g) >= req.steps]:
            b.retire(gid)
            ln.retiring[gid] = ln.active.pop(gid)
        return True

    def run(self, trace: list[Request], time_scale: float = 1.0, max_wall: float | None = None) -> dict:
        """Replays `trace` (arrival times divided by time_scale) until every request
        has finished. Returns throughput and latency statistics."""
        pending = deque(sorted((Request(r.rid, r.arrival / time_scale, r.n, r.steps, r.kind, r.phi0) for r in trace),
                               key=lambda r: r.arrival))
        queue: deque = deque()
        self.t0 = self.clock()
        while pending or queue or self._live():
            now = self.clock() - self.t0
            if max_wall is not None and now > max_wall:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            self._admit(queue, now)
            busy = self._collect()
            for ln in self.lanes:
                busy = self._feed(ln) or busy
            if not busy:
                if pending and not queue and not any(ln.has_work() or ln.retiring for ln in self.lanes):
                    self.sleep(max(0.0, min(pending[0].arrival - (self.clock() - self.t0), 0.05)))
                else:
                    self.sleep(self.poll_s)
        # the slices still queued (resident grids) are part of the measured work
        while any(ln.inflight for ln in self.lanes):
            for ln in self.lanes:
                while ln.inflight and ln.backend.reached(ln.inflight[0]):
                    ln.inflight.popleft()
            if any(ln.inflight for ln in self.lanes):
                self.sleep(self.poll_s)
        wall = self.clock() - self.t0
        status = 0
        for ln in self.lanes:
            st = ln.backend.status() if hasattr(ln.backend, "status") else 0
            status = status or int(st)
        solved = [r for r in self.results if r.error == 0]
        lat = np.array([r.latency for r in solved]) if solved else np.zeros(1)
        lanes = []
        for i, ln in enumerate(self.lanes):
            mine = [r for r in solved if self._lane_for(Request(0, 0.0, r.n, r.steps, "")) is ln]
            ll = np.array([r.latency for r in mine]) if mine else np.zeros(1)
            lanes.append({"max_work": ln.max_work, "slice_steps": ln.slice_steps, "solved": len(mine),
                          "slices": ln.slices, "p50_s": float(np.percentile(ll, 50)),
                          "p99_s": float(np.percentile(ll, 99)),
                          "resident_steps_per_s": ln.resident_steps / wall if ln.resident and wall > 0 else None})
        return {"requests": len(self.results), "failed": len(self.results) - len(solved), "wall_s": wall,
                "slices": sum(ln.slices for ln in self.lanes),
                "solves_per_s": len(solved) / wall if wall > 0 else 0.0,
                "cell_updates_per_s": self.cell_updates / wall if wall > 0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "peak_bytes": self.peak_used, "budget_bytes": self.budget,
                "lanes": lanes, "status": int(status)}
