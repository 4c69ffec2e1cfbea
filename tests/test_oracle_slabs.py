"""Domain decomposition of one box into z-slabs (multi-GPU scheme 2), in the
oracle: the slab-split step with halo exchange over gloo ranks reproduces the
unsplit step bit for bit -- fields, particles and accumulators -- with
particles on and next to the slab boundaries, thermal noise, springs and the
mode drive."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import ic as oic
from oracle import slabs


def case(nz):
    p = oic.GridParams(nx=10, ny=8, nz=nz, kT=1e-3, wave_amp=3e-3, forcing="mode", wave_axis=0, seed=21,
                       box=3, zeta=0.2)
    rng = np.random.default_rng(5)
    zs = np.array([0.05, nz / 2 - 0.02, nz / 2 + 0.03, nz - 0.1, nz / 3 + 0.5, 2 * nz / 3 - 0.49, 1.6])
    q = np.column_stack([rng.uniform(0, 10, zs.size), rng.uniform(0, 8, zs.size), zs])
    m_e = rng.uniform(-2.0, 6.0, zs.size)
    kappa = rng.uniform(0.3, 2.0, zs.size)
    k_s = np.where(np.arange(zs.size) % 2 == 0, 0.4, 0.0)
    th_drho, th_g = oic.thermal_fluctuation(p, 77)
    rho, g = oic.standing_wave(p)
    return p, rho - p.rho0 + th_drho, [g[a] + th_g[a] for a in range(3)], (q, m_e, kappa, k_s)


def serial(nz, nsteps, weights):
    p, drho, g, (q, m_e, kappa, k_s) = case(nz)
    sim = oic.Simulation(p, g=g, drho=drho)
    sim.add_particles(q, m_e, kappa, k_s)
    u0 = sim.parts.u.copy()
    sim.run(nsteps, weights)
    return sim, u0


def slab_run(comm, nz, nsteps, weights, u0):
    p, drho, g, (q, m_e, kappa, k_s) = case(nz)
    sl = slabs.SlabSimulation(p, comm, drho, g)
    sl.add_particles(q, m_e, kappa, k_s, u0)
    sl.run(nsteps, weights)
    drho, g = sl.gather_fields()
    return dict(drho=drho, g=g, q=sl.parts.q, u=sl.parts.u, lam=sl.lam, sw=sl.acc.sw, sa2=sl.acc.sa2,
                sf=sl.acc.sf, sl=sl.acc.sl)


def check(res, sim):
    assert np.array_equal(res["drho"], sim.drho)
    for a in range(3):
        assert np.array_equal(res["g"][a], sim.g[a])
    assert np.array_equal(res["q"], sim.parts.q)
    assert np.array_equal(res["u"], sim.parts.u)
    assert np.array_equal(res["lam"], sim.lam)
    assert res["sw"] == sim.acc.sw and res["sa2"] == sim.acc.sa2
    assert np.array_equal(res["sf"], sim.acc.sf) and np.array_equal(res["sl"], sim.acc.sl)


def test_slab_bounds_partition():
    for nz, world in [(16, 2), (18, 3), (17, 4), (9, 1)]:
        b = [slabs.slab_bounds(nz, world, r) for r in range(world)]
        assert b[0][0] == 0 and b[-1][1] == nz
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
        assert max(z1 - z0 for z0, z1 in b) - min(z1 - z0 for z0, z1 in b) <= 1


def test_single_slab_with_periodic_ghosts_equals_serial():
    w = np.linspace(0.5, 1.0, 4)
    sim, u0 = serial(8, 4, w)
    check(slab_run(slabs.SelfComm(), 8, 4, w, u0), sim)


def worker(rank, world, port, nz, nsteps, weights, u0, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = slab_run(slabs.GlooComm(), nz, nsteps, weights, u0)
        q.put((rank, res))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world,nz", [(2, 16), (3, 18)])
def test_slabs_over_gloo_ranks_equal_serial(world, nz):
    w = np.linspace(0.5, 1.0, 4)
    sim, u0 = serial(nz, 4, w)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, nz, 4, w, u0, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = [q.get(timeout=300) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for _, res in results:
        check(res, sim)


def test_planted_mistake_is_caught():
    """A slab whose ghosts are not refreshed (one halo plane short) must differ."""
    w = np.linspace(0.5, 1.0, 3)
    sim, u0 = serial(8, 3, w)

    class StaleComm(slabs.SelfComm):
        def exchange(self, top, bottom):
            lower, upper = super().exchange(top, bottom)
            lower[:, 0] = 0.0
            return lower, upper

    res = slab_run(StaleComm(), 8, 3, w, u0)
    assert not np.array_equal(res["drho"], sim.drho)
