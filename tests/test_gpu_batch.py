"""Batches of independent grids (one launch per step over a work list of tiles).

* every grid of a mixed batch matches the FP64 oracle and the single-grid path;
* a grid's result is bitwise the same alone and in a mix, also when it joins a
  batch that is already running, and with or without CUDA-graph replay;
* per-grid step targets freeze a grid; removal frees its slot.
"""
import numpy as np
import pytest

from paper_2007_07760_gb300 import native as N
from paper_2007_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

COMMON = dict(W=4.0, M=0.02, cfl=0.8, order=3, flux=0, stages=2)


def mixed_grids(seed=1):
    rng = np.random.default_rng(WL.SEED_BASE + seed)
    out = []
    for (nx, ny), kind in zip([(45, 27), (64, 64), (33, 40), (100, 80)],
                              ["uniform", "rotation", "vortex", "uniform"]):
        cents = [tuple(rng.uniform(0, [nx, ny])) for _ in range(2)]
        phi0 = WL.drops(nx, ny, cents, [min(nx, ny) / 5, min(nx, ny) / 6], 4.0)
        if kind == "uniform":
            vel = (float(rng.uniform(-0.04, 0.04)), float(rng.uniform(-0.04, 0.04)))
        elif kind == "rotation":
            vel = (nx / 2, ny / 2, 2e-3)
        else:
            vel = (float(nx), 0.04, 40.0)
        out.append((phi0, kind, vel))
    return out


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_batch_matches_single_grid_path(precision, tol):
    grids = mixed_grids()
    with N.Batch(precision=precision, **COMMON) as b:
        ids = [b.add(phi0, kind, vel) for phi0, kind, vel in grids]
        b.step(20)
        for gid, (phi0, kind, vel) in zip(ids, grids):
            ny, nx = phi0.shape
            with N.Solver(nx, ny, phi0, vel_kind=kind, vel=vel, precision=precision, **COMMON) as s:
                s.step(20)
                assert rel(b.phi(gid), s.phi()) < tol
                assert abs(b.mass(gid) - s.mass()) / s.mass() < (1e-13 if precision == "fp64" else 1e-6)


def test_batch_matches_oracle_fp64(oracle):
    grids = mixed_grids(seed=2)
    with N.Batch(precision="fp64", **COMMON) as b:
        ids = [b.add(phi0, kind, vel) for phi0, kind, vel in grids]
        b.step(12)
        for gid, (phi0, kind, vel) in zip(ids, grids):
            ny, nx = phi0.shape
            p = oracle.Params(nx, ny, vel_kind=kind, vel=vel, **COMMON)
            ref = oracle.State(p, phi0).run(12)
            assert rel(b.phi(gid), ref.phi()) < 1e-12


@pytest.mark.parametrize("precision", ["fp32", "fp16f"])
def test_alone_equals_in_mix_bitwise(precision):
    grids = mixed_grids(seed=3)
    phi0, kind, vel = grids[1]
    with N.Batch(precision=precision, **COMMON) as alone:
        g = alone.add(phi0, kind, vel)
        alone.step(17)
        ref = alone.phi(g)
        mref = alone.mass(g)
    with N.Batch(precision=precision, **COMMON) as mix:
        others = [mix.add(p0, k, v) for p0, k, v in grids[:1] + grids[2:]]
        mix.step(5)                          # the mix is already running
        g = mix.add(phi0, kind, vel)         # joins at its own step 0
        mix.step(17)
        assert mix.step_index(g) == 17 and all(mix.step_index(o) == 22 for o in others)
        assert np.array_equal(mix.phi(g), ref)
        assert mix.mass(g) == mref


def test_graph_replay_equals_single_launches():
    grids = mixed_grids(seed=4)
    res = []
    for chunks in ([16], [1] * 16):
        with N.Batch(precision="fp32", **COMMON) as b:
            ids = [b.add(p0, k, v) for p0, k, v in grids]
            for c in chunks:
                b.step(c)
            res.append([b.phi(i) for i in ids])
    for a, c in zip(*res):
        assert np.array_equal(a, c)


def test_targets_freeze_grids_and_removal_reuses_slots():
    grids = mixed_grids(seed=5)
    with N.Batch(precision="fp32", **COMMON) as b:
        g0 = b.add(grids[0][0], grids[0][1], grids[0][2], target_steps=5)
        g1 = b.add(grids[1][0], grids[1][1], grids[1][2])
        b.step(3)
        frozen_at_3 = b.phi(g0)
        b.step(10)
        assert b.step_index(g0) == 5 and b.step_index(g1) == 13
        after = b.phi(g0)
        b.step(9)
        assert np.array_equal(b.phi(g0), after) and not np.array_equal(after, frozen_at_3)
        assert b.active_cells() == grids[1][0].size
        b.remove(g0)
        g2 = b.add(grids[2][0], grids[2][1], grids[2][2])
        assert g2 == g0
        b.step(2)
        assert b.step_index(g2) == 2 and b.status() == 0
