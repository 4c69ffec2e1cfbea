"""Gradients of an ensemble of deterministic boxes over ranks (world size 2,
gloo, CPU): each rank differentiates its own box with the oracle's adjoint;
the combined gradient equals the serial combination of both boxes, and the
A-gradient of the ensemble objective equals central differences of the sum
of the two boxes' objectives."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import adjoint as oadj
from oracle import ic as oic


def box(rank, A=3e-3):
    p = oic.GridParams(nx=8, ny=7, nz=6, forcing="mode", wave_amp=A, zeta=0.2, wave_phase=0.3 * rank)
    rng = np.random.default_rng(10 + rank)
    drho = 2e-3 * rng.uniform(-1, 1, p.shape)
    g = [2e-3 * rng.uniform(-1, 1, p.shape) for _ in range(3)]
    n = 2 + rank
    parts = oadj.make_parts(rng.uniform(0.5, 5.5, (n, 3)), 1e-3 * rng.normal(size=(n, 3)), rng.uniform(1, 5, n),
                            rng.uniform(0.4, 1.2, n), 0.6, p.c)
    return p, drho, g, parts, np.linspace(0.5, 1.0, 6), np.tile([1.0, 0.0, 0.0], (n, 1))


def box_gradient(rank):
    p, drho, g, parts, w, d = box(rank)
    return oadj.rollout_gradient(p, drho, g, parts, w, d, checkpoint_every=4)


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1307_0702_gb300 import ensemble

    phi, gr = box_gradient(rank)
    ens = ensemble.ensemble_gradient(phi, gr)
    q.put((rank, ens["phi"], ens["A"], ens["m_e"], ens["kappa_ratio"], ens["boxes"]))
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_ensemble_gradient_over_two_ranks():
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
    serial = [box_gradient(0), box_gradient(1)]
    for rank, phi, gA, gm, gk, boxes in results:
        assert boxes == 2
        assert phi == serial[0][0] + serial[1][0]
        assert gA == serial[0][1]["A"] + serial[1][1]["A"]
        assert np.array_equal(gm, np.concatenate([serial[0][1]["m_e"], serial[1][1]["m_e"]]))
        assert np.array_equal(gk, np.concatenate([serial[0][1]["kappa_ratio"], serial[1][1]["kappa_ratio"]]))

    # the drive amplitude shared by both boxes: central differences of the ensemble objective
    def phi_ens(A):
        tot = 0.0
        for r in range(2):
            p, drho, g, parts, w, d = box(r, A)
            tot += oadj.rollout(p, drho, g, parts, w, d)[0]
        return tot

    e = 1e-4          # relative: A moves by 3e-7, well above the rounding of the positions
    fd = (phi_ens(3e-3 * (1 + e)) - phi_ens(3e-3 * (1 - e))) / (2 * e * 3e-3)
    assert abs(results[0][2] - fd) <= 1e-5 * abs(fd)
