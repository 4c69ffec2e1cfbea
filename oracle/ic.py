"""One explicit time step of the inertial-coupling method (oracle).

Follows App. A.2 substeps 1-7 in the paper's order and notation:

 1. q^{n+1/2} = q^n + (dt/2) J^n v^n
 2. F^{n+1/2} = F(q^{n+1/2}, t^{n+1/2})          (here: a tethering spring)
 3. fluid SSP-RK3 from t^n to t^{n+1} with the particle frozen at q^{n+1/2},
    the pressure pi = c^2 rho + S Omega (Eqs. (eq:pressure), (omega)) built from
    each stage's own density, and the momentum source S F^{n+1/2}; no lambda.
 4. dg = dt (lambda + F) = m_e m_f / (m_e + m_f) (J v~^{n+1} - u^n),
    m_f = V J rho^{n+1}
 5. u^{n+1} = u^n + m_f / (m_e + m_f) (J v~^{n+1} - u^n)
 6. momentum-conserving fluid correction
 7. q^{n+1} = q^n + (dt/2) J^{n+1/2} (v^{n+1} + v^n)

Readings where the paper is silent or ambiguous (each also listed in the
project's design notes):

* Substep 6 is applied to the momentum, g^{n+1} = g~^{n+1} - S dg ("g form"),
  so that total momentum m_e u + h^3 sum g changes by exactly dt sum F.  The
  paper writes it for the velocity, v^{n+1} = v~^{n+1} - (V/m_f) S dg; that "v
  form" is kept as an option (``momentum_form='v'``).  Both coincide at zero
  Mach number (footnote in Sec. 7).
* Several particles: every particle takes its impulse from the same v~^{n+1}
  and all spreads are added (the paper only says the generalisation to N
  particles is straightforward, Sec. 4.2).
* The standing wave is held by a body pressure (``forcing='mode'``,
  p_ext = P cos(k x) sin(omega t + phi) with P = 2 Gamma omega A, Gamma = (4 eta/3 +
  zeta)/(2 rho0), omega = (2c/h) sin(kh/2)), which keeps the mode at density
  amplitude A from the exact initial eigenmode rho0 + A cos(kx).  The paper's
  own drive (Eq. (pext)), a pressure on one grid plane, is ``forcing='plane'``
  with Delta p0 = A N Gamma omega.
* The radiation force is read from a spring F = -k_s (q - q_eq) tethering the
  particle (Sec. 6): the reported force is minus the weighted time average of
  the spring force.
"""
from dataclasses import dataclass, field

import numpy as np

from . import fluid, peskin, philox


@dataclass
class GridParams:
    nx: int = 32
    ny: int = 32
    nz: int = 32
    h: float = 1.0
    rho0: float = 1.0
    c: float = 4.0
    eta: float = 0.5
    zeta: float = 0.0
    kT: float = 0.0
    dt: float = 0.025
    seed: int = 0
    box: int = 0
    forcing: str = "none"          # 'none' | 'mode' | 'plane'
    wave_axis: int = 0             # 0 = x, 1 = y, 2 = z
    wave_amp: float = 0.0          # target density amplitude A of the driven mode
    wave_nlambda: int = 1          # wavelengths per box along wave_axis
    plane_index: int = 0           # grid plane driven when forcing == 'plane'
    wave_phase: float = 0.0        # drive phase phi: sin(omega t + phi)
    momentum_form: str = "g"       # 'g' (default) or 'v' (paper's literal form)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def lengths(self):
        return np.array([self.nx, self.ny, self.nz], dtype=np.float64) * self.h

    def fluid(self):
        return fluid.FluidParams(self.h, self.rho0, self.c, self.eta, self.zeta, self.kT, self.dt)


def epsilon_from_kappa_ratio(kappa_ratio, c):
    """epsilon_pf = c_p^2 - c_f^2 with c_p^2 = c_f^2 kappa_f/kappa_p (Eqs. (part_svel), (ke))."""
    return c ** 2 * (1.0 / np.asarray(kappa_ratio, dtype=np.float64) - 1.0)


def wave_numbers(p):
    """(k, discrete k~, omega = c k~, Gamma) of the driven mode."""
    n_ax = (p.nx, p.ny, p.nz)[p.wave_axis]
    k = 2.0 * np.pi * p.wave_nlambda / (n_ax * p.h)
    kd = (2.0 / p.h) * np.sin(0.5 * k * p.h)
    gamma = (4.0 * p.eta / 3.0 + p.zeta) / (2.0 * p.rho0)
    return k, kd, p.c * kd, gamma


def axis_coordinate(p, axis):
    """Cell-centre coordinate along ``axis`` broadcast to the grid shape."""
    n = (p.nx, p.ny, p.nz)[axis]
    x = np.arange(n) * p.h
    shape = [1, 1, 1]
    shape[fluid.AXIS[axis]] = n
    return np.broadcast_to(x.reshape(shape), p.shape)


def external_pressure(p, t):
    """Body pressure of the standing-wave drive at time t (centres)."""
    if p.forcing == "none" or p.wave_amp == 0.0:
        return None
    k, kd, omega, gamma = wave_numbers(p)
    if p.forcing == "mode":
        amp = 2.0 * gamma * omega * p.wave_amp
        return amp * np.cos(k * axis_coordinate(p, p.wave_axis)) * np.sin(omega * t + p.wave_phase)
    if p.forcing == "plane":
        n_ax = (p.nx, p.ny, p.nz)[p.wave_axis]
        dp0 = p.wave_amp * n_ax * gamma * omega
        idx = np.rint(axis_coordinate(p, p.wave_axis) / p.h).astype(np.int64)
        return np.where(idx == p.plane_index, dp0 * np.sin(omega * t + p.wave_phase), 0.0)
    raise ValueError(p.forcing)


def mode_amplitude(p, drho):
    """A(t) = (2/N) sum_i (rho_i - rho0) cos(k x_i) along the wave axis (drho = rho - rho0)."""
    k = wave_numbers(p)[0]
    return 2.0 * np.mean(drho * np.cos(k * axis_coordinate(p, p.wave_axis)))


def standing_wave(p):
    """Initial eigenmode rho = rho0 + A cos(k x), g = 0."""
    k = wave_numbers(p)[0]
    rho = p.rho0 + p.wave_amp * np.cos(k * axis_coordinate(p, p.wave_axis))
    return np.array(rho), [np.zeros(p.shape) for _ in range(3)]


def thermal_fluctuation(p, seed):
    """(delta rho, g) of a sample of the discrete Gibbs state of the linearised fluid.

    delta rho ~ N(0, rho0 kT / (c^2 h^3)), g^alpha ~ N(0, rho0 kT / h^3) from
    Philox purpose 1, with the means removed so that total mass and momentum
    are those of the quiescent fluid.
    """
    n = int(np.prod(p.shape))
    z = philox.thermal_normals(seed, p.box, n)
    vol = p.h ** 3
    drho = np.sqrt(p.rho0 * p.kT / (p.c ** 2 * vol)) * z[0]
    drho -= drho.mean()
    g = []
    for a in range(3):
        ga = np.sqrt(p.rho0 * p.kT / vol) * z[1 + a]
        ga -= ga.mean()
        g.append(ga.reshape(p.shape))
    return drho.reshape(p.shape), g


def thermal_state(p, seed):
    """The Gibbs sample as (rho, g)."""
    drho, g = thermal_fluctuation(p, seed)
    return p.rho0 + drho, g


def particle_pressure(centre, drho, eps, p):
    """S Omega at the cell centres, Omega = epsilon V (J rho - rho0) (Eqs. (eq:pressure), (omega)).

    drho = rho - rho0; J rho - rho0 = J drho because the weights sum to 1 (Eq. (k1)).
    """
    omega = eps * peskin.kernel_volume(p.h) * centre.interp(drho)
    return centre.spread(omega, p.shape, p.h)


@dataclass
class Particles:
    q: np.ndarray                   # (np, 3) positions
    u: np.ndarray                   # (np, 3) velocities
    m_e: np.ndarray                 # (np,) excess mass
    eps: np.ndarray                 # (np,) epsilon_pf
    k_s: np.ndarray                 # (np,) spring constant (0 = free)
    q_eq: np.ndarray                # (np, 3) spring anchor

    @property
    def n(self):
        return self.q.shape[0]


@dataclass
class Accumulators:
    sw: float = 0.0                 # sum of weights
    sa2: float = 0.0                # sum of w A(t)^2
    sf: np.ndarray = None           # (np, 3) sum of w F_spring
    sl: np.ndarray = None           # (np, 3) sum of w lambda


class Simulation:
    """State (rho, g, particles) and the IC step.

    The density is carried as drho = rho - rho0 (``rho`` is a derived view).
    """

    def __init__(self, p: GridParams, rho=None, g=None, drho=None):
        self.p = p
        if drho is None:
            if rho is None:
                rho, g = standing_wave(p) if p.wave_amp != 0.0 else (
                    np.full(p.shape, p.rho0), [np.zeros(p.shape) for _ in range(3)])
            drho = np.asarray(rho, dtype=np.float64) - p.rho0
        self.drho = np.array(drho, dtype=np.float64)
        self.g = [np.array(a, dtype=np.float64) for a in g]
        self.parts = Particles(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0),
                               np.zeros(0), np.zeros((0, 3)))
        self.step_index = 0
        self.acc = Accumulators(sf=np.zeros((0, 3)), sl=np.zeros((0, 3)))
        self.last = {}

    @property
    def rho(self):
        return self.p.rho0 + self.drho

    # ------------------------------------------------------------------ setup
    def velocities(self, drho=None, g=None):
        """v^a = g^a / rho^a with the face density rho0 + (drho_i + drho_{i+a}) / 2."""
        drho = self.drho if drho is None else drho
        g = self.g if g is None else g
        return [g[a] / (self.p.rho0 + 0.5 * (drho + fluid.up(drho, a))) for a in range(3)]

    def add_particles(self, q, m_e, kappa_ratio, k_spring=None, u=None):
        """Append particles; u defaults to J v at q (no-slip, Eq. (noslip))."""
        q = np.mod(np.atleast_2d(np.asarray(q, dtype=np.float64)), self.p.lengths)
        n = q.shape[0]
        if u is None:
            _, faces = peskin.all_stencils(q, self.p.h, self.p.shape)
            v = self.velocities()
            u = np.stack([faces[a].interp(v[a]) for a in range(3)], axis=1)
        u = np.atleast_2d(np.asarray(u, dtype=np.float64)).reshape(n, 3)
        ks = np.zeros(n) if k_spring is None else np.broadcast_to(np.asarray(k_spring, float), (n,))
        pp = self.parts
        self.parts = Particles(np.vstack([pp.q, q]), np.vstack([pp.u, u]),
                               np.concatenate([pp.m_e, np.broadcast_to(np.asarray(m_e, float), (n,))]),
                               np.concatenate([pp.eps, epsilon_from_kappa_ratio(
                                   np.broadcast_to(np.asarray(kappa_ratio, float), (n,)), self.p.c)]),
                               np.concatenate([pp.k_s, ks]), np.vstack([pp.q_eq, q]))
        self.acc.sf = np.vstack([self.acc.sf, np.zeros((n, 3))])
        self.acc.sl = np.vstack([self.acc.sl, np.zeros((n, 3))])

    # ------------------------------------------------------------ diagnostics
    def total_momentum(self):
        """m_e u + h^3 sum g (the conserved total of Eq. (eq:totmom))."""
        pm = np.sum(self.parts.m_e[:, None] * self.parts.u, axis=0)
        return np.array([self.p.h ** 3 * np.sum(self.g[a]) for a in range(3)]) + pm

    def spring_force(self, q):
        d = q - self.parts.q_eq
        L = self.p.lengths
        d = d - L * np.round(d / L)
        return -self.parts.k_s[:, None] * d

    # ------------------------------------------------------------------ step
    def step(self, weight=0.0):
        p, fp, pt = self.p, self.p.fluid(), self.parts
        h, dt, shape = p.h, p.dt, p.shape
        vol = peskin.kernel_volume(h)
        t_n = self.step_index * dt
        rho_n, g_n = self.drho, self.g
        v_n = self.velocities(rho_n, g_n)
        npart = pt.n

        # substep 1: half-step position with J at q^n
        if npart:
            _, faces_n = peskin.all_stencils(pt.q, h, shape)
            jv_n = np.stack([faces_n[a].interp(v_n[a]) for a in range(3)], axis=1)
            q_half = np.mod(pt.q + 0.5 * dt * jv_n, p.lengths)
            # substep 2: external force at q^{n+1/2}
            force = self.spring_force(q_half)
            centre, faces = peskin.all_stencils(q_half, h, shape)
            jv_n_half = np.stack([faces[a].interp(v_n[a]) for a in range(3)], axis=1)
            face_force = [faces[a].spread(force[:, a], shape, h) for a in range(3)]
        else:
            force = np.zeros((0, 3))
            face_force = None

        # substep 3: SSP-RK3 for the fluid with the particle frozen
        normals = None
        if p.kT > 0.0:
            z = philox.stress_normals(p.seed, p.box, self.step_index, int(np.prod(shape)))
            w_a, w_b = z[0:6].reshape((6,) + shape), z[6:12].reshape((6,) + shape)
        rho_s, g_s = rho_n, g_n
        for s in range(3):
            extra = external_pressure(p, t_n + fluid.RK3_TIME[s] * dt)
            if npart:
                pp = particle_pressure(centre, rho_s, pt.eps, p)
                extra = pp if extra is None else extra + pp
            if p.kT > 0.0:
                normals = w_a + fluid.RK3_BETA[s] * w_b
            drho, dg = fluid.rates(rho_s, g_s, fp, extra, normals, face_force)
            rho_next = fluid.rk3_combine(s, rho_n, rho_s, dt * drho)
            g_next = [fluid.rk3_combine(s, g_n[a], g_s[a], dt * dg[a]) for a in range(3)]
            rho_s, g_s = rho_next, g_next
        rho_new, g_tilde = rho_s, g_s

        if npart:
            # substep 4: impulse from the unperturbed velocity
            v_tilde = self.velocities(rho_new, g_tilde)
            jv_tilde = np.stack([faces[a].interp(v_tilde[a]) for a in range(3)], axis=1)
            m_f = vol * (p.rho0 + centre.interp(rho_new))
            me = pt.m_e[:, None]
            mf = m_f[:, None]
            dgp = me * mf / (me + mf) * (jv_tilde - pt.u)
            # substep 5
            u_new = pt.u + mf / (me + mf) * (jv_tilde - pt.u)
            # substep 6
            if p.momentum_form == "g":
                g_new = [g_tilde[a] - faces[a].spread(dgp[:, a], shape, h) for a in range(3)]
            else:
                rf = [p.rho0 + 0.5 * (rho_new + fluid.up(rho_new, a)) for a in range(3)]
                g_new = [rf[a] * (v_tilde[a] - faces[a].spread(vol / m_f * dgp[:, a], shape, h))
                         for a in range(3)]
            v_new = self.velocities(rho_new, g_new)
            # substep 7
            jv_new = np.stack([faces[a].interp(v_new[a]) for a in range(3)], axis=1)
            q_new = np.mod(pt.q + 0.5 * dt * (jv_new + jv_n_half), p.lengths)
            lam = dgp / dt - force
            self.last = dict(q_half=q_half, force=force, g_tilde=g_tilde, jv_tilde=jv_tilde,
                             m_f=m_f, dg=dgp, jv_new=jv_new, lam=lam)
            pt.q, pt.u = q_new, u_new
        else:
            g_new = g_tilde
            lam = np.zeros((0, 3))
            self.last = dict(g_tilde=g_tilde)

        self.drho, self.g = rho_new, g_new
        self.step_index += 1
        if weight != 0.0:
            self.acc.sw += weight
            self.acc.sa2 += weight * mode_amplitude(p, self.drho) ** 2
            self.acc.sf += weight * force
            self.acc.sl += weight * lam
        self.lam = lam

    def run(self, nsteps, weights=None):
        for i in range(nsteps):
            self.step(0.0 if weights is None else float(weights[i]))

    def time_average(self):
        """(<F_spring>_w, <lambda>_w, <A^2>_w)."""
        sw = self.acc.sw
        return self.acc.sf / sw, self.acc.sl / sw, self.acc.sa2 / sw
