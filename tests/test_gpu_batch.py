"""Batched ensemble (ic_batch_*): every box of a batch evolves bit for bit as
it does under its own ic_step, for boxes of different sizes, seeds and
particle sets (the heterogeneous ensembles whose averages the method
measures, Sec. 6)."""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def make_boxes(prec, stream=None):
    from paper_1307_0702_gb300 import Grid

    specs = [(16, 3, 0), (24, 7, 1), (16, 0, 2), (20, 12, 3)]
    grids, inputs = [], []
    for n, npart, box in specs:
        gp, parts = W.many_particle_config(n, max(npart, 1), kT=1e-3, wave_amp=2e-3, seed=box, precision=prec,
                                           k_spring=0.4 if box % 2 else 0.0)
        gp["box"] = box
        rho, g = W.standing_wave_fields(gp)
        grid = Grid(gp, stream=stream)
        grid.set_state(rho, g)
        grid.init_thermal(100 + box)
        if npart:
            grid.add_particles(parts["q"][:npart], parts["m_e"][:npart], parts["kappa_ratio"][:npart],
                               parts["k_spring"][:npart])
        grids.append(grid)
        inputs.append((gp, rho, g, parts, npart, box))
    return grids, inputs


def snapshot(grid):
    rho, g = grid.get_state()
    out = [rho] + g
    if grid.n_particles:
        out += list(grid.forces())
        f, lam, a2 = grid.time_average()
        out += [f, lam, np.array([a2])]
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_equals_individual_steps(prec):
    from paper_1307_0702_gb300 import Batch

    w = np.linspace(0.2, 1.0, 7)
    a_grids, _ = make_boxes(prec)
    with Batch(a_grids) as batch:
        batch.step(3, w[:3])
        batch.step(4, w[3:])
        batched = [snapshot(g) for g in a_grids]
    b_grids, _ = make_boxes(prec)
    for g in b_grids:
        g.step(7, w)
    single = [snapshot(g) for g in b_grids]
    for x, y in zip(batched, single):
        assert len(x) == len(y)
        for u, v in zip(x, y):
            assert np.array_equal(u, v)
    for g in a_grids + b_grids:
        g.close()


def test_batch_boxes_sharing_one_stream():
    import torch

    from paper_1307_0702_gb300 import Batch

    a_grids, _ = make_boxes("fp32", stream=torch.cuda.Stream())
    with Batch(a_grids) as batch:
        batch.step(4, np.ones(4))
    b_grids, _ = make_boxes("fp32")
    for g in b_grids:
        g.step(4, np.ones(4))
    for ga, gb in zip(a_grids, b_grids):
        for u, v in zip(snapshot(ga), snapshot(gb)):
            assert np.array_equal(u, v)
    for g in a_grids + b_grids:
        g.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_tiling_leaves_results_unchanged(prec):
    """Every stage-kernel tiling gives the same fields, particles and forces
    bit for bit (only the reduction order of A(t) changes)."""
    from paper_1307_0702_gb300 import Grid

    runs = []
    # (tile_x, zchunk, staging of the wide tile): x edge 40 admits the row modes in FP32
    for tile_x, zchunk, copy in [(32, 32, "rows16"), (16, 8, "rows16"), (32, 8, "bulk"), (16, 16, "thread"),
                                 (32, 16, "thread")]:
        gp, parts = W.many_particle_config((40, 20, 18), 9, kT=1e-3, wave_amp=2e-3, seed=5, precision=prec,
                                           k_spring=0.3)
        rho, g = W.standing_wave_fields(gp)
        with Grid(gp) as grid:
            grid.set_tile(tile_x, zchunk)
            grid.set_stage_copy(copy)
            assert grid.tile()[0] == tile_x and grid.tile()[2] == min(zchunk, 18)
            assert grid.stage_copy() == (copy if prec == "fp32" and tile_x == 32 else "thread")
            grid.set_state(rho, g)
            grid.init_thermal(4)
            grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
            grid.step(6, np.ones(6))
            runs.append(snapshot(grid))
    for other in runs[1:]:
        for u, v in zip(runs[0][:-1], other[:-1]):
            assert np.array_equal(u, v)
        assert np.allclose(runs[0][-1], other[-1], rtol=1e-5 if prec == "fp32" else 1e-12, atol=0)


def test_autotune_keeps_state_and_results():
    from paper_1307_0702_gb300 import Batch, Grid

    def fresh():
        gp, parts = W.many_particle_config(24, 5, kT=1e-3, wave_amp=2e-3, seed=8, precision="fp32")
        rho, g = W.standing_wave_fields(gp)
        grid = Grid(gp)
        grid.set_state(rho, g)
        grid.init_thermal(1)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"])
        return grid

    a, b = fresh(), fresh()
    a.step(2, np.ones(2))
    b.step(2, np.ones(2))
    before = snapshot(a)
    choice = a.autotune(reps=2)
    assert choice[0] in (16, 24, 32) and choice[2] in (8, 16, 24)
    for u, v in zip(before, snapshot(a)):
        assert np.array_equal(u, v)
    a.step(3, np.ones(3))
    b.step(3, np.ones(3))
    for u, v in zip(snapshot(a)[:-1], snapshot(b)[:-1]):
        assert np.array_equal(u, v)
    c = fresh()
    c.step(5, np.ones(5))
    with Batch([a, c]) as batch:
        tiles = batch.autotune(reps=1)
        assert tiles[0] == tiles[1]
        batch.step(2, np.ones(2))
    b.step(2, np.ones(2))
    for u, v in zip(snapshot(a)[:-1], snapshot(b)[:-1]):
        assert np.array_equal(u, v)
    for g in (a, b, c):
        g.close()


def test_batch_as_one_graph_equals_individual_steps(monkeypatch):
    from paper_1307_0702_gb300 import Batch

    monkeypatch.setenv("IC_BATCH_GRAPH", "1")
    w = np.linspace(0.3, 1.0, 5)
    a_grids, _ = make_boxes("fp32")
    with Batch(a_grids) as batch:
        batch.step(5, w)
    monkeypatch.delenv("IC_BATCH_GRAPH")
    b_grids, _ = make_boxes("fp32")
    for g in b_grids:
        g.step(5, w)
    for ga, gb in zip(a_grids, b_grids):
        for u, v in zip(snapshot(ga), snapshot(gb)):
            assert np.array_equal(u, v)
    for g in a_grids + b_grids:
        g.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("fp64", 1e-11)])
def test_batch_boxes_against_the_oracle(prec, tol):
    """Every box of a heterogeneous batch (edges 16, 24, 32 and 48, 0 to 20
    particles, their own Philox seeds and box ids, tethered and free) against
    the oracle run of the same box, field by field and particle by particle."""
    from pairs import compare, run_oracle

    from paper_1307_0702_gb300 import Batch, Grid

    specs = [(16, 0, 11), (24, 7, 12), (32, 20, 13), (48, 13, 14)]
    w = np.linspace(0.5, 1.0, 3)
    grids, inputs = [], []
    for n, npart, box in specs:
        gp, parts = W.many_particle_config(n, max(npart, 1), kT=1e-3, wave_amp=2e-3, seed=box, precision=prec,
                                           k_spring=0.4 if box % 2 else 0.0)
        gp["box"] = box
        rho, g = W.standing_wave_fields(gp)
        grid = Grid(gp)
        grid.set_state(rho, g)
        grid.init_thermal(200 + box, add=True)
        sub = {k: v[:npart] for k, v in parts.items()} if npart else None
        if npart:
            grid.add_particles(sub["q"], sub["m_e"], sub["kappa_ratio"], sub["k_spring"])
        grids.append(grid)
        inputs.append((gp, rho, g, sub))
    with Batch(grids) as batch:
        batch.step(3, w)
    for grid, (gp, rho, g, sub) in zip(grids, inputs):
        out = {}
        out["rho"], out["g"] = grid.get_state()
        if sub is not None:
            out["lam"], out["u"], out["q"] = grid.forces()
            out["f_avg"], out["lam_avg"], out["a2"] = grid.time_average()
        sim = run_oracle(gp, rho, g, sub, nsteps=3, weights=w, thermal_seed=200 + gp["box"])
        errs = compare(out, sim, gp, q0=None if sub is None else sub["q"])
        bad = {k: v for k, v in errs.items() if not v <= tol}
        assert not bad, (gp["nx"], errs)
        grid.close()
