"""Batched ensemble (ic_batch_*): every box of a batch evolves bit for bit as
it does under its own ic_step, for boxes of different sizes, seeds and
particle sets (the heterogeneous ensembles whose averages the method
measures, Sec. 6)."""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def make_boxes(prec):
    from paper_1307_0702_gb300 import Grid

    specs = [(16, 3, 0), (24, 7, 1), (16, 0, 2), (20, 12, 3)]
    grids, inputs = [], []
    for n, npart, box in specs:
        gp, parts = W.many_particle_config(n, max(npart, 1), kT=1e-3, wave_amp=2e-3, seed=box, precision=prec,
                                           k_spring=0.4 if box % 2 else 0.0)
        gp["box"] = box
        rho, g = W.standing_wave_fields(gp)
        grid = Grid(gp)
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
