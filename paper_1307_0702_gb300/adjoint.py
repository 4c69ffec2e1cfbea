"""Differentiable deterministic rollout of the IC method.

The observable of Sec. 6 is the time-averaged force on tethered particles,
whose closed form (Eq. (eq:acousticForce2)) depends on the particle's excess
compressibility (f_1, Eq. (f1)) and excess mass (f_2, Eq. (f2)) and on the
square of the wave amplitude.  ``Rollout`` runs N deterministic steps of a
``Grid`` and returns

    Phi = sum_p d_p . <F_p>_w,    <F>_w = sum_n w_n F^{n+1/2} / sum_n w_n,

and ``Rollout.backward`` its gradient with respect to every particle's m_e
and kappa_p/kappa_f, the drive amplitude and the initial state, by the
library's adjoint kernels: states are kept on the device every
``checkpoint_every`` steps; each segment is then run forward again from its
checkpoint, every step recording its tape (ic_step_record_tape), and the
tapes are reversed last first (ic_adjoint_step_tape).  With ``tapes=False``
the segment keeps one snapshot per step instead, and each step is recorded
again just before it is reversed (a third forward pass, K snapshots instead
of K tapes of ~19 fields).

``time_averaged_force`` wraps it as a torch.autograd.Function.
"""
import numpy as np

from .ic import Grid


class Rollout:
    """Checkpointed forward and reverse sweeps of one deterministic box.

    grid: a Grid with kT = 0 and its particles added; kappa_ratio: the
    particles' kappa_p/kappa_f (n,), for the chain rule from epsilon_pf.
    """

    def __init__(self, grid, kappa_ratio, checkpoint_every=50, tapes=True):
        if grid.params.get("kT", 0.0) != 0.0:
            raise ValueError("the adjoint covers the deterministic step (kT = 0)")
        self.grid = grid
        self.kappa = np.asarray(kappa_ratio, dtype=np.float64).reshape(-1)
        self.K = int(checkpoint_every)
        if self.K < 1:
            raise ValueError("checkpoint_every must be >= 1")
        self.tapes = bool(tapes)
        self.checkpoints = []
        self.weights = None
        grid.adjoint_enable()

    def forward(self, weights, direction=None):
        """Run len(weights) steps; returns Phi."""
        g = self.grid
        self.weights = np.asarray(weights, dtype=np.float64).reshape(-1)
        self.direction = None if direction is None else np.asarray(direction, float).reshape(-1, 3)
        n = len(self.weights)
        W = float(np.sum(self.weights))
        if n == 0 or W == 0.0:
            raise ValueError("the weights must be non-empty and sum to a non-zero value")
        try:
            g.time_average(reset=True)
        except Exception:       # no sums yet
            pass
        self.checkpoints = []
        for start in range(0, n, self.K):
            buf = g.new_snapshot()
            g.snapshot_save(buf)
            self.checkpoints.append(buf)
            stop = min(start + self.K, n)
            g.step(stop - start, weights=self.weights[start:stop])
        return g.objective(self.direction, reset=True)

    def backward(self):
        """Gradients of the last forward's Phi: dict m_e, kappa_ratio, eps (n,),
        A (drive amplitude, through the drive only), rho, g (initial fields),
        q, u (initial particle state)."""
        g = self.grid
        n = len(self.weights)
        W = float(np.sum(self.weights))
        g.adjoint_reset(self.direction)
        if self.tapes:
            tapes = [g.new_tape() for _ in range(min(self.K, n))]
            for seg in range(len(self.checkpoints) - 1, -1, -1):
                start = seg * self.K
                stop = min(start + self.K, n)
                g.snapshot_load(self.checkpoints[seg])
                for j in range(stop - start):
                    g.step_record_tape(tapes[j])
                for j in range(stop - start - 1, -1, -1):
                    g.adjoint_step_tape(tapes[j], self.weights[start + j] / W)
            return self._read()
        pool = [g.new_snapshot() for _ in range(min(self.K, n) - 1)]
        for seg in range(len(self.checkpoints) - 1, -1, -1):
            start = seg * self.K
            stop = min(start + self.K, n)
            # the segment's states: its checkpoint, then one snapshot per recomputed step
            states = [self.checkpoints[seg]] + pool[:stop - start - 1]
            g.snapshot_load(states[0])
            for j in range(1, stop - start):
                g.step(1)
                g.snapshot_save(states[j])
            for j in range(stop - start - 1, -1, -1):
                g.snapshot_load(states[j])
                g.step_record()
                g.adjoint_step(self.weights[start + j] / W)
        return self._read()

    def _read(self):
        g = self.grid
        out = g.adjoint_read()
        out["kappa_ratio"] = g.adjoint_read_kappa()
        return out


def time_averaged_force(params, q, m_e, kappa_ratio, k_spring, wave_amp, rho, g=None, u=None, weights=None,
                        direction=None, checkpoint_every=50):
    """Phi = sum_p d_p . <F_p>_w of a deterministic rollout, differentiable in
    m_e, kappa_ratio (n,), wave_amp (scalar, the drive amplitude), rho (the
    initial density, [z, y, x]), g (the three initial momentum fields) and u
    (initial particle velocities, (n, 3); default zero).  All torch tensors
    (float64); params as for ``Grid`` (kT must be 0); weights (N,) the
    averaging weight of each step."""
    import torch

    class _F(torch.autograd.Function):
        @staticmethod
        def forward(ctx, m_e_t, kappa_t, amp_t, rho_t, gx_t, gy_t, gz_t, u_t):
            p = dict(params)
            p["wave_amp"] = float(amp_t)
            grid = Grid(p)
            grid.set_state(rho_t.detach().cpu().numpy(),
                           [x.detach().cpu().numpy() for x in (gx_t, gy_t, gz_t)])
            grid.add_particles(np.asarray(q, float), m_e_t.detach().cpu().numpy(),
                               kappa_t.detach().cpu().numpy(), np.asarray(k_spring, float),
                               u=u_t.detach().cpu().numpy())
            roll = Rollout(grid, kappa_t.detach().cpu().numpy(), checkpoint_every)
            phi = roll.forward(weights, direction)
            ctx.roll = roll
            return torch.tensor(phi, dtype=torch.float64)

        @staticmethod
        def backward(ctx, dphi):
            gr = ctx.roll.backward()
            ctx.roll.grid.close()
            s = float(dphi)

            def t(x):
                return torch.as_tensor(np.asarray(x) * s, dtype=torch.float64)

            return (t(gr["m_e"]), t(gr["kappa_ratio"]), t(gr["A"]), t(gr["rho"]), t(gr["g"][0]), t(gr["g"][1]),
                    t(gr["g"][2]), t(gr["u"]))

    n = np.asarray(q).reshape(-1, 3).shape[0]
    shape = tuple(rho.shape)
    zeros = torch.zeros(shape, dtype=torch.float64)
    gx, gy, gz = (zeros, zeros, zeros) if g is None else g
    u = torch.zeros((n, 3), dtype=torch.float64) if u is None else u
    return _F.apply(m_e, kappa_ratio, torch.as_tensor(wave_amp, dtype=torch.float64), rho, gx, gy, gz, u)
