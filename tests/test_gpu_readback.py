"""Pipelined read-back of the constraint forces (ic_forces_async /
ic_forces_collect) against the blocking ic_forces, bit for bit: each step's
lambda queued into one of two pinned slots and read while the next step runs
equals lambda read after a synchronisation; refusals of bad slots."""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def boxes(prec):
    from paper_1307_0702_gb300 import Grid

    out = []
    for _ in range(2):
        gp, parts = W.many_particle_config(24, 12, kT=1e-3, wave_amp=3e-3, seed=4, precision=prec)
        rho, g = W.standing_wave_fields(gp)
        grid = Grid(gp)
        grid.set_state(rho, g)
        grid.init_thermal(2)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"])
        out.append(grid)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pipelined_readback_equals_forces(prec):
    a, b = boxes(prec)
    w = np.ones(1)
    nsteps = 7
    piped = []
    for i in range(nsteps):
        a.step(1, w)
        a.forces_async(i & 1)
        if i:
            piped.append(a.forces_collect((i - 1) & 1))
    piped.append(a.forces_collect((nsteps - 1) & 1))
    blocking = []
    for i in range(nsteps):
        b.step(1, w)
        blocking.append(b.forces()[0])
    for x, y in zip(piped, blocking):
        assert np.array_equal(x, y)
        assert np.any(x != 0.0)
    for g in (a, b):
        g.close()


def test_readback_slot_refusals():
    from paper_1307_0702_gb300.ic import ICError

    a, b = boxes("fp32")
    with pytest.raises(ICError) as e:
        a.forces_collect(0)          # nothing queued
    assert e.value.status == -6
    with pytest.raises(ICError) as e:
        a.forces_async(2)
    assert e.value.status == -1
    a.step(1)
    a.forces_async(1)
    a.forces_collect(1)
    with pytest.raises(ICError):
        a.forces_collect(1)          # collected once
    for g in (a, b):
        g.close()
