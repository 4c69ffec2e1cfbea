"""One box split into z-slabs over ranks: the IC step with halo exchange (oracle).

TEST INFRASTRUCTURE ONLY, like the rest of this package: it states, in plain
numpy, the data flow of the domain-decomposed form of the step so that a test
can check that splitting a box changes no bit of the result.

Decomposition
-------------
Rank r of R owns the planes z0_r <= z < z1_r (an even split of nz) and keeps
HALO = 3 ghost planes on each side.  One RK3 stage's rates at a plane reach at
most two planes away (the face density and velocity of the plane above, the
flux differences of the plane below), so three ghost planes keep the owned
planes exact; the planes of the padded slab that the periodic rolls of the
flux code wrap around are never used.

Per step, in the order of App. A.2:

* halo exchange of (delta rho, g) before every RK3 stage and after the last
  one (4 per step): each rank sends its top HALO planes to the next rank and
  its bottom HALO planes to the previous one;
* particle state is replicated on every rank.  Each particle is owned by the
  rank whose slab holds its cell plane at q^n; the owner does the particle's
  gathers J (stencils reach two planes past the owned ones, inside the
  ghosts) and the per-particle results are all-gathered in particle order;
* every rank spreads every particle's S contributions (pressure S Omega,
  force S F, impulse S dg) onto its whole padded slab, ghosts included, in
  the serial order (particle, then stencil point), so ghost planes need no
  second exchange;
* the stochastic stress of a ghost cell is drawn from the same counter
  (global cell index) as on its owner;
* the driven-mode amplitude A(t) of the accumulators is taken over the
  gathered density.

Only the 'g' (momentum) form of substep 6 is decomposed.
"""
import numpy as np

from . import fluid, ic, peskin, philox

HALO = 3


def slab_bounds(nz, world, rank):
    """[z0, z1) of rank's slab: nz split as evenly as possible, lower ranks first."""
    base, rem = divmod(nz, world)
    z0 = rank * base + min(rank, rem)
    return z0, z0 + base + (1 if rank < rem else 0)


class SelfComm:
    """World of one rank: the ghosts of the only slab are its own periodic images."""

    rank, world = 0, 1

    def exchange(self, top, bottom):
        """(lower ghosts, upper ghosts) given this rank's top and bottom planes."""
        return top.copy(), bottom.copy()

    def allgather(self, obj):
        return [obj]


class GlooComm:
    """torch.distributed point-to-point and all-gather (gloo, CPU tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, top, bottom):
        import torch

        d = self.dist
        nxt, prv = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        lower = torch.empty(top.shape, dtype=torch.float64)
        upper = torch.empty(bottom.shape, dtype=torch.float64)
        # tag 0: planes moving up (my top -> next rank's lower ghosts); tag 1: moving down
        reqs = [d.isend(torch.from_numpy(np.ascontiguousarray(top)), nxt, self.group, tag=0),
                d.isend(torch.from_numpy(np.ascontiguousarray(bottom)), prv, self.group, tag=1),
                d.irecv(lower, prv, self.group, tag=0),
                d.irecv(upper, nxt, self.group, tag=1)]
        for r in reqs:
            r.wait()
        return lower.numpy(), upper.numpy()

    def allgather(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out


class SlabSimulation:
    """This rank's slab of an ``ic.Simulation`` (same parameters and initial state).

    Fields are held as padded arrays of nloc + 2 HALO planes; plane l of the
    padded slab is the global plane (z0 - HALO + l) mod nz.
    """

    def __init__(self, p: ic.GridParams, comm, drho, g):
        if p.momentum_form != "g":
            raise ValueError("only the momentum form of substep 6 is decomposed")
        self.p, self.comm = p, comm
        self.z0, self.z1 = slab_bounds(p.nz, comm.world, comm.rank)
        self.nloc = self.z1 - self.z0
        if self.nloc < HALO or (comm.world > 1 and self.nloc + 2 * HALO > p.nz):
            raise ValueError("slabs must hold at least HALO planes and their ghosts must not overlap")
        self.npad = self.nloc + 2 * HALO
        self.zg = (self.z0 - HALO + np.arange(self.npad)) % p.nz       # global plane of each padded plane
        # padded copies of each global plane (a plane may appear twice when R = 1)
        self.copies = [[] for _ in range(p.nz)]
        for l, z in enumerate(self.zg):
            self.copies[z].append(l)
        self.ncopy = max(len(c) for c in self.copies)
        self.drho = self._pad_from_global(drho)
        self.g = [self._pad_from_global(a) for a in g]
        self.parts = ic.Particles(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0),
                                  np.zeros(0), np.zeros((0, 3)))
        self.acc = ic.Accumulators(sf=np.zeros((0, 3)), sl=np.zeros((0, 3)))
        self.step_index = 0
        self.lam = np.zeros((0, 3))

    # ------------------------------------------------------------- layout
    @property
    def plane_cells(self):
        return self.p.nx * self.p.ny

    @property
    def pad_shape(self):
        return (self.npad, self.p.ny, self.p.nx)

    def _pad_from_global(self, a):
        return np.array(np.asarray(a, dtype=np.float64)[self.zg])

    def interior(self, a):
        return a[HALO:HALO + self.nloc]

    def _halo_exchange(self, fields):
        """Refresh the ghost planes of the given padded fields (in place)."""
        top = np.stack([f[self.nloc:self.nloc + HALO] for f in fields])   # my topmost owned planes
        bottom = np.stack([f[HALO:2 * HALO] for f in fields])               # my lowest owned planes
        lower, upper = self.comm.exchange(top, bottom)
        for j, f in enumerate(fields):
            f[:HALO] = lower[j]
            f[HALO + self.nloc:] = upper[j]

    def _local_first(self, flat):
        """Global linear indices -> one padded linear index each (any copy)."""
        zg, rest = np.divmod(flat, self.plane_cells)
        local = np.array([self.copies[z][0] if self.copies[z] else -1 for z in range(self.p.nz)])[zg]
        if np.any(local < 0):
            raise RuntimeError("stencil point outside the padded slab")
        return local * self.plane_cells + rest

    def _local_all(self, flat):
        """Global linear indices (n, 27) -> (n, 27, ncopy) padded indices, -1 where absent."""
        zg, rest = np.divmod(flat, self.plane_cells)
        table = np.full((self.p.nz, self.ncopy), -1, dtype=np.int64)
        for z, c in enumerate(self.copies):
            table[z, :len(c)] = c
        local = table[zg]
        return np.where(local >= 0, local * self.plane_cells + rest[..., None], -1)

    def _interp(self, st, rows, field):
        """J field for the particles ``rows`` of stencil set ``st`` (their owner's gather)."""
        if rows.size == 0:
            return np.zeros(0)
        flat = self._local_first(st.flat[rows])
        return np.sum(st.w[rows] * field.reshape(-1)[flat], axis=1)

    def _spread(self, st, values):
        """S values of every particle onto every padded copy, in serial order."""
        out = np.zeros(self.npad * self.plane_cells)
        if st.flat.shape[0]:
            vals = st.w * (np.asarray(values, dtype=np.float64)[:, None] / self.p.h ** 3)
            idx = self._local_all(st.flat)
            vals = np.broadcast_to(vals[..., None], idx.shape)
            keep = idx >= 0
            np.add.at(out, idx[keep], vals[keep])
        return out.reshape(self.pad_shape)

    def _gather_rows(self, owned, values):
        """All-gather per-particle rows computed by their owners into particle order."""
        parts = self.comm.allgather((owned, values))
        n = self.parts.n
        out = None
        for rows, vals in parts:
            if out is None:
                out = np.zeros((n,) + np.asarray(vals).shape[1:])
            out[rows] = vals
        return out

    def _owned(self, q):
        plane = np.floor(q[:, 2] / self.p.h).astype(np.int64) % self.p.nz
        return np.nonzero((plane >= self.z0) & (plane < self.z1))[0]

    def gather_fields(self):
        """(delta rho, [g_x, g_y, g_z]) of the whole box, identical on every rank."""
        slabs = self.comm.allgather([self.interior(self.drho)] + [self.interior(a) for a in self.g])
        return (np.concatenate([s[0] for s in slabs]),
                [np.concatenate([s[1 + a] for s in slabs]) for a in range(3)])

    # ------------------------------------------------------------ particles
    def add_particles(self, q, m_e, kappa_ratio, k_spring, u):
        """Replicated particle state (u given: the serial run's initial velocities)."""
        q = np.mod(np.atleast_2d(np.asarray(q, dtype=np.float64)), self.p.lengths)
        n = q.shape[0]
        self.parts = ic.Particles(q, np.asarray(u, dtype=np.float64).reshape(n, 3),
                                  np.broadcast_to(np.asarray(m_e, float), (n,)).copy(),
                                  ic.epsilon_from_kappa_ratio(np.broadcast_to(np.asarray(kappa_ratio, float), (n,)),
                                                              self.p.c),
                                  np.broadcast_to(np.asarray(k_spring, float), (n,)).copy(), q.copy())
        self.acc.sf = np.zeros((n, 3))
        self.acc.sl = np.zeros((n, 3))

    def velocities(self, drho, g):
        return [g[a] / (self.p.rho0 + 0.5 * (drho + fluid.up(drho, a))) for a in range(3)]

    def spring_force(self, q):
        d = q - self.parts.q_eq
        L = self.p.lengths
        d = d - L * np.round(d / L)
        return -self.parts.k_s[:, None] * d

    # ------------------------------------------------------------------ step
    def step(self, weight=0.0):
        """Substeps 1-7 of App. A.2, decomposed (see the module header)."""
        p, fp, pt = self.p, self.p.fluid(), self.parts
        h, dt, gshape = p.h, p.dt, p.shape
        vol = peskin.kernel_volume(h)
        t_n = self.step_index * dt
        npart = pt.n
        self._halo_exchange([self.drho] + self.g)
        rho_n, g_n = self.drho, self.g
        v_n = self.velocities(rho_n, g_n)

        if npart:
            own = self._owned(pt.q)
            _, faces_n = peskin.all_stencils(pt.q, h, gshape)
            jv_n = np.stack([self._interp(faces_n[a], own, v_n[a]) for a in range(3)], axis=1).reshape(-1, 3)
            q_half_own = np.mod(pt.q[own] + 0.5 * dt * jv_n, p.lengths)
            q_half = self._gather_rows(own, q_half_own)
            force = self.spring_force(q_half)
            centre, faces = peskin.all_stencils(q_half, h, gshape)
            jv_n_half = self._gather_rows(own, np.stack([self._interp(faces[a], own, v_n[a]) for a in range(3)],
                                                        axis=1).reshape(-1, 3))
            face_force = [self._spread(faces[a], force[:, a]) for a in range(3)]
        else:
            force = np.zeros((0, 3))
            face_force = None

        cells = ((self.zg[:, None, None] * p.ny + np.arange(p.ny)[None, :, None]) * p.nx
                 + np.arange(p.nx)[None, None, :]).reshape(-1)
        if p.kT > 0.0:
            z = philox.stress_normals_at(p.seed, p.box, self.step_index, cells)
            w_a, w_b = z[0:6].reshape((6,) + self.pad_shape), z[6:12].reshape((6,) + self.pad_shape)
        normals = None
        rho_s, g_s = rho_n, g_n
        for s in range(3):
            if s > 0:
                self._halo_exchange([rho_s] + g_s)
            extra = ic.external_pressure(p, t_n + fluid.RK3_TIME[s] * dt)
            extra = None if extra is None else self._pad_from_global(extra)
            if npart:
                omega = self._gather_rows(own, pt.eps[own] * vol * self._interp(centre, own, rho_s))
                pp = self._spread(centre, omega)
                extra = pp if extra is None else extra + pp
            if p.kT > 0.0:
                normals = w_a + fluid.RK3_BETA[s] * w_b
            drho, dg = fluid.rates(rho_s, g_s, fp, extra, normals, face_force)
            rho_next = fluid.rk3_combine(s, rho_n, rho_s, dt * drho)
            g_next = [fluid.rk3_combine(s, g_n[a], g_s[a], dt * dg[a]) for a in range(3)]
            rho_s, g_s = rho_next, g_next
        rho_new, g_tilde = rho_s, g_s
        self._halo_exchange([rho_new] + g_tilde)

        if npart:
            v_tilde = self.velocities(rho_new, g_tilde)
            jv_tilde = self._gather_rows(own, np.stack([self._interp(faces[a], own, v_tilde[a]) for a in range(3)],
                                                       axis=1).reshape(-1, 3))
            m_f = vol * (p.rho0 + self._gather_rows(own, self._interp(centre, own, rho_new)))
            me = pt.m_e[:, None]
            mf = m_f[:, None]
            dgp = me * mf / (me + mf) * (jv_tilde - pt.u)
            u_new = pt.u + mf / (me + mf) * (jv_tilde - pt.u)
            g_new = [g_tilde[a] - self._spread(faces[a], dgp[:, a]) for a in range(3)]
            v_new = self.velocities(rho_new, g_new)
            jv_new = self._gather_rows(own, np.stack([self._interp(faces[a], own, v_new[a]) for a in range(3)],
                                                     axis=1).reshape(-1, 3))
            q_new = np.mod(pt.q + 0.5 * dt * (jv_new + jv_n_half), p.lengths)
            lam = dgp / dt - force
            pt.q, pt.u = q_new, u_new
        else:
            g_new = g_tilde
            lam = np.zeros((0, 3))

        self.drho, self.g = rho_new, g_new
        self.step_index += 1
        if weight != 0.0:
            full_drho, _ = self.gather_fields()
            self.acc.sw += weight
            self.acc.sa2 += weight * ic.mode_amplitude(p, full_drho) ** 2
            self.acc.sf += weight * force
            self.acc.sl += weight * lam
        self.lam = lam

    def run(self, nsteps, weights=None):
        for i in range(nsteps):
            self.step(0.0 if weights is None else float(weights[i]))
