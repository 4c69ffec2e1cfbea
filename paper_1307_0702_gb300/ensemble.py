"""Ensembles of independent boxes spread over ranks (one box per GPU).

The gradients of a differentiable rollout (one box per rank) are combined
the same way at the end, by ``ensemble_gradient``.

The IC step of one box needs no communication: every rank advances its own
box (its own Philox ``box`` id) and the only exchange is at the end, where the
weighted sums behind the time averages (sum_n w_n F_n, sum_n w_n lambda_n,
sum_n w_n, sum_n w_n A_n^2) of every box are combined in FP64.  The ensemble
average of the radiation force is the mean over all particles of each
particle's time average -(sum w F)/(sum w) (the estimator of Sec. 6 applied
to the ensemble).
"""
import numpy as np


def ensemble_sums(sums, group=None):
    """Combine the weighted sums of one box per rank over the ranks of ``group``.

    sums: {"sw": float, "sa2": float, "sf": (np, 3), "sl": (np, 3)} of this
    rank's box.  Returns, identically on every rank, {"sw": total weight,
    "sa2": total, "sf", "sl": particle sums of all boxes stacked in rank order,
    "sw_p": (n_total,) weight sum of each particle's box, "boxes": ranks}.
    """
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    mine = {"sw": float(sums["sw"]), "sa2": float(sums["sa2"]),
            "sf": np.ascontiguousarray(sums["sf"], dtype=np.float64).reshape(-1, 3),
            "sl": np.ascontiguousarray(sums["sl"], dtype=np.float64).reshape(-1, 3)}
    if world > 1:
        parts = [None] * world
        dist.all_gather_object(parts, mine, group=group)
    else:
        parts = [mine]
    return {"sw": float(sum(p["sw"] for p in parts)),     # summed in rank order on every rank
            "sa2": float(sum(p["sa2"] for p in parts)),
            "sf": np.concatenate([p["sf"] for p in parts], axis=0),
            "sl": np.concatenate([p["sl"] for p in parts], axis=0),
            "sw_p": np.concatenate([np.full(p["sf"].shape[0], p["sw"]) for p in parts]),
            "boxes": world}


def ensemble_force(ens):
    """Mean over the ensemble's particles of the radiation force -<F_spring>_w.

    A statistic of the ensemble, taken on the host over the boxes' results:
    each box's time averages are the library's (ic_time_average); averaging
    independent realizations is outside the method's step."""
    return -np.mean(ens["sf"] / ens["sw_p"][:, None], axis=0)


def ensemble_a2(ens):
    """Ensemble mean of <A^2>_w."""
    return ens["sa2"] / ens["sw"]


def ensemble_gradient(phi, grad, group=None):
    """Combine the rollout gradients of one box per rank (``Rollout.backward``
    or the oracle's) for the ensemble objective Phi_ens = sum over boxes of
    each box's Phi.

    phi: this rank's Phi; grad: dict with m_e, kappa_ratio (n,) and A.
    Returns, identically on every rank, {"phi": sum of Phi, "m_e",
    "kappa_ratio": per-particle gradients of all boxes stacked in rank order
    (a particle belongs to one box), "A": summed over boxes (a drive
    amplitude shared by the ensemble), "boxes": ranks}.
    """
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    mine = {"phi": float(phi), "A": float(grad["A"]),
            "m_e": np.ascontiguousarray(grad["m_e"], dtype=np.float64).reshape(-1),
            "kappa_ratio": np.ascontiguousarray(grad["kappa_ratio"], dtype=np.float64).reshape(-1)}
    if world > 1:
        parts = [None] * world
        dist.all_gather_object(parts, mine, group=group)
    else:
        parts = [mine]
    return {"phi": float(sum(p["phi"] for p in parts)), "A": float(sum(p["A"] for p in parts)),
            "m_e": np.concatenate([p["m_e"] for p in parts]),
            "kappa_ratio": np.concatenate([p["kappa_ratio"] for p in parts]), "boxes": world}
