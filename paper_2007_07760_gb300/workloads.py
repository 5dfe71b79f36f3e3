"""Seeded synthetic inputs shaped like the paper's interface-tracking tests.

This module only builds initial order-parameter fields and velocity-field
parameters (Sec. III: translation of a circular interface, Zalesak's slotted disk
under rigid rotation, the extension of a circle in a reversed shear flow, a
reversing vortex). It contains none of the DUGKS
arithmetic and is the one module both the CUDA path's callers and the oracle's
tests draw their inputs from.

Coordinates are in cells: cell (i, j) has its centre at (i + 1/2, j + 1/2);
arrays are (ny, nx), x fastest. The interface profile is the equilibrium
tanh profile of Sec. II.A, phi = 1/2 + 1/2 tanh(2 s / W) for a signed distance s
that is positive inside phase A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2007077600


def centres(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    return np.meshgrid(x, y)          # X[j, i], Y[j, i]


def tanh_profile(s: np.ndarray, W: float) -> np.ndarray:
    return 0.5 + 0.5 * np.tanh(2.0 * s / W)


def periodic_delta(a: np.ndarray, c: float, n: int) -> np.ndarray:
    d = a - c
    return d - n * np.round(d / n)


def drops(nx: int, ny: int, centers, radii, W: float) -> np.ndarray:
    """Union of circular drops on the periodic box (minimum-image distance)."""
    X, Y = centres(nx, ny)
    s = np.full((ny, nx), -np.inf)
    for (cx, cy), R in zip(centers, radii):
        dx = periodic_delta(X, cx, nx)
        dy = periodic_delta(Y, cy, ny)
        s = np.maximum(s, R - np.sqrt(dx * dx + dy * dy))
    return tanh_profile(s, W)


def slotted_disk(n: int, cx: float, cy: float, R: float, slot_w: float, slot_h: float,
                 W: float) -> np.ndarray:
    """Zalesak's disk: a disk with a rectangular slot opening downward (Sec. III.B)."""
    X, Y = centres(n, n)
    s_disk = R - np.hypot(X - cx, Y - cy)
    x0, x1 = cx - slot_w / 2, cx + slot_w / 2
    y0, y1 = cy - R, cy - R + slot_h
    # signed distance to the slot rectangle, positive outside it
    dx = np.maximum(np.maximum(x0 - X, X - x1), 0.0)
    dy = np.maximum(np.maximum(y0 - Y, Y - y1), 0.0)
    outside = np.hypot(dx, dy)
    inside = np.minimum(np.minimum(X - x0, x1 - X), np.minimum(Y - y0, y1 - Y))
    s_slot = np.where((dx > 0) | (dy > 0), outside, -inside)
    return tanh_profile(np.minimum(s_disk, s_slot), W)


def planar_slab(n: int, W: float) -> np.ndarray:
    """phi = 1/2 [tanh(2(x - n/4)/W) - tanh(2(x - 3n/4)/W)], uniform in y."""
    X, _ = centres(n, n)
    return 0.5 * (np.tanh(2.0 * (X - n / 4) / W) - np.tanh(2.0 * (X - 3 * n / 4) / W))


@dataclass
class Problem:
    """One simulation: grid, method parameters, velocity and initial field."""
    name: str
    nx: int
    ny: int
    W: float
    M: float
    cfl: float
    order: int
    flux: int               # 0 upwind, 1 central
    stages: int
    vel_kind: str           # uniform | rotation | vortex
    vel: tuple
    phi0: np.ndarray = field(repr=False)
    steps: int = 1000
    dtphiu: int = 1

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def drop64(order: int = 2, flux: int = 0, stages: int = 2, cfl: float = 0.8,
           n: int = 64, steps: int = 1000) -> Problem:
    """64x64 periodic circular drop R = 16, W = 4, M = 0.01, u = (0.02, 0.02)."""
    phi0 = drops(n, n, [(n / 2, n / 2)], [n / 4], 4.0)
    return Problem("drop64", n, n, 4.0, 0.01, cfl, order, flux, stages, "uniform",
                   (0.02, 0.02), phi0, steps)


def slotted_disk256(order: int = 3, flux: int = 0, stages: int = 2, cfl: float = 0.8,
                    n: int = 256, steps: int = 16384) -> Problem:
    """256x256 slotted disk R = 64 centred at (128, 160), slot 16 x 80, W = 4,
    rigid rotation about the box centre, one revolution in 16384 steps, M = 0.002."""
    s = n / 256.0
    phi0 = slotted_disk(n, 128 * s, 160 * s, 64 * s, 16 * s, 80 * s, 4.0)
    omega = 2.0 * math.pi / (16384 * cfl)
    return Problem("slotted_disk256", n, n, 4.0, 0.002, cfl, order, flux, stages, "rotation",
                   (n / 2, n / 2, omega), phi0, steps)


def vortex1024(order: int = 3, flux: int = 0, stages: int = 2, cfl: float = 0.8,
               n: int = 1024, steps: int = 8192, umax: float = 0.05) -> Problem:
    """Single-vortex deformation on the unit box mapped to n x n cells: drop
    R = 0.15 at (0.5, 0.75), reversed by cos(pi t / T) with T = steps * dt.
    Reading: the peak speed is scaled to umax lattice units (stability)."""
    phi0 = drops(n, n, [(0.5 * n, 0.75 * n)], [0.15 * n], 4.0)
    return Problem("vortex1024", n, n, 4.0, 0.02, cfl, order, flux, stages, "vortex",
                   (float(n), umax, steps * cfl), phi0, steps)


def random_batch(count: int = 512, seed: int = SEED_BASE + 3, nmin: int = 64, nmax: int = 512,
                 order: int = 3, cfl: float = 0.8, steps: int = 1000):
    """Independent periodic grids: side log-uniform in [nmin, nmax], 1-8 drops
    (R uniform in [8, min(64, N/4)], W = 4), uniform velocity of random angle and
    |u| <= 0.05, M = 0.02, upwind, two-stage."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        k = int(rng.integers(1, 9))
        rmax = min(64.0, n / 4)
        radii = rng.uniform(8.0, rmax, size=k)
        cents = rng.uniform(0.0, n, size=(k, 2))
        ang = rng.uniform(0.0, 2 * math.pi)
        sp = rng.uniform(0.0, 0.05)
        phi0 = drops(n, n, [tuple(c) for c in cents], radii, 4.0)
        out.append(Problem(f"batch{g}", n, n, 4.0, 0.02, cfl, order, 0, 2, "uniform",
                           (sp * math.cos(ang), sp * math.sin(ang)), phi0, steps))
    return out


def extension(Pe: float, cfl: float, L0: int = 256, M: float = 0.02, W: float = 4.0):
    """Interface extension in a shear flow (Sec. III.C): circle R = L0/5 centred at
    (0.5 L0, 0.3 L0), cell-centre velocity u = U0 pi sin(pi x/L0) cos(pi y/L0),
    v = -U0 pi cos(pi x/L0) sin(pi y/L0) with U0 = Pe M / L0, reversed after
    T_f = L0/U0 and run for another T_f. Returns (phi0, u, v, steps per half)."""
    U0 = Pe * M / L0
    X, Y = centres(L0, L0)
    u = U0 * math.pi * np.sin(math.pi * X / L0) * np.cos(math.pi * Y / L0)
    v = -U0 * math.pi * np.cos(math.pi * X / L0) * np.sin(math.pi * Y / L0)
    phi0 = drops(L0, L0, [(0.5 * L0, 0.3 * L0)], [L0 / 5], W)
    return phi0, u, v, int(round(L0 / U0 / cfl))


def zalesak_disk(L0: int = 256) -> np.ndarray:
    """Zalesak's slotted disk of Sec. III.B as a step function: phi = 1 at the cell
    centres inside the disk (radius 0.4 L0, centred in the L0 x L0 domain) and
    outside the slot (0.08 L0 wide, opening downward), 0 elsewhere. Reading: the
    slot length is unstated; it runs from the bottom of the disk to 0.25 R above
    the centre (length 1.25 R), the proportions of the slotted-disk workload."""
    R, w = 0.4 * L0, 0.08 * L0
    X, Y = centres(L0, L0)
    c = 0.5 * L0
    inside = (X - c) ** 2 + (Y - c) ** 2 < R * R
    slot = (np.abs(X - c) < 0.5 * w) & (Y < c + 0.25 * R)
    return (inside & ~slot).astype(np.float64)


def zalesak(Pe: float, cfl: float, M: float = 0.02, L0: int = 256, Cn: float = 4.0 / 256):
    """Zalesak's disk rotation (Sec. III.B): rigid rotation about the domain centre
    with u = -(U0 pi / L0)(y - L0/2), v = (U0 pi / L0)(x - L0/2), U0 = Pe M / L0,
    one revolution in T = 2 T_f = 2 L0 / U0; W = Cn L0. Returns the problem (its
    steps = one revolution)."""
    U0 = Pe * M / L0
    om = U0 * math.pi / L0
    steps = int(round(2.0 * L0 / U0 / cfl))
    return Problem(f"zalesak{L0}", L0, L0, Cn * L0, M, cfl, 3, 0, 2, "rotation", (0.5 * L0, 0.5 * L0, om),
                   zalesak_disk(L0), steps)


def deformation(Pe: float, cfl: float, M: float = 0.02, L0: int = 512, Cn: float = 4.0 / 512):
    """Smoothed deformation (Sec. III.D): a circle in the centre of the L0 x L0
    domain in the shear flow u = -U0 sin(4 pi x/L0) sin(4 pi y/L0) cos(pi t/T_f),
    v = -U0 cos(4 pi x/L0) cos(4 pi y/L0) cos(pi t/T_f), U0 = Pe M / L0, run to
    t = T_f = L0 / U0 (the displacement integral of cos(pi t / T_f) vanishes there).
    Reading: the circle's radius is unstated; R = L0/5 as in the paper's other
    tests. Returns the problem (its steps reach T_f)."""
    U0 = Pe * M / L0
    Tf = L0 / U0
    steps = int(round(Tf / cfl))
    phi0 = drops(L0, L0, [(0.5 * L0, 0.5 * L0)], [L0 / 5], Cn * L0)
    return Problem(f"deformation{L0}", L0, L0, Cn * L0, M, cfl, 3, 0, 2, "deformation", (float(L0), U0, steps * cfl),
                   phi0, steps)


def translation(n: int, order: int, flux: int, stages: int, cfl: float,
                Pe: float = 128.0, Cn: float = 1.0 / 32, M: float = 0.02) -> Problem:
    """Diagonal translation of a circle R = L0/5 (Sec. III.A): U0 = Pe M / L0,
    W = Cn L0, one period T_f = L0 / U0."""
    U0 = Pe * M / n
    W = Cn * n
    phi0 = drops(n, n, [(n / 2, n / 2)], [n / 5], W)
    steps = int(round(n / U0 / cfl))
    return Problem(f"translation{n}", n, n, W, M, cfl, order, flux, stages, "uniform",
                   (U0, U0), phi0, steps)
