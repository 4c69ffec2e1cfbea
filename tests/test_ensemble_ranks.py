"""Ensemble over ranks (world size 2, gloo, CPU): each rank runs its own box in
the oracle; the combined sums equal the serial combination of both boxes."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import ic as oic


def box_sums(rank):
    p = oic.GridParams(nx=8, ny=8, nz=8, kT=1e-3, wave_amp=2e-3, forcing="mode", seed=11, box=rank)
    s = oic.Simulation(p)
    rng = np.random.default_rng(rank)
    s.add_particles(rng.uniform(0, 8, (2 + rank, 3)), 4.0, 0.5, 0.3)
    s.run(6, np.linspace(0.5, 1.0, 6))
    return {"sw": s.acc.sw, "sa2": s.acc.sa2, "sf": s.acc.sf.copy(), "sl": s.acc.sl.copy()}


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1307_0702_gb300 import ensemble

    ens = ensemble.ensemble_sums(box_sums(rank))
    q.put((rank, ens["sw"], ens["sa2"], ens["sf"], ens["sl"], ensemble.ensemble_force(ens)))
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_ensemble_sums_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted([q.get(timeout=300) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    serial = [box_sums(0), box_sums(1)]
    sw = serial[0]["sw"] + serial[1]["sw"]
    sf = np.concatenate([serial[0]["sf"], serial[1]["sf"]])
    for rank, r_sw, r_sa2, r_sf, r_sl, force in results:
        assert r_sw == sw
        assert r_sa2 == serial[0]["sa2"] + serial[1]["sa2"]
        assert np.array_equal(r_sf, sf)
        assert np.array_equal(r_sl, np.concatenate([serial[0]["sl"], serial[1]["sl"]]))
        per = np.concatenate([serial[b]["sf"] / serial[b]["sw"] for b in range(2)])
        assert np.allclose(force, -per.mean(axis=0), rtol=0, atol=1e-18)
    # the two boxes draw different noise (box id in the Philox counter)
    assert not np.array_equal(serial[0]["sf"][:2], serial[1]["sf"][:2])
