"""Compressible fluctuating hydrodynamics on the periodic staggered grid.

Equations (Sec. 4.2): d_t rho + div g = 0 (Eq. (eq:consvDens)) and
d_t g + div(g v) = -div P (Eq. (eq:consvMom)) with P = pi I - sigma (Eq. (totp)),
a Newtonian stress whose divergence is eta lap v + (zeta + eta/3) grad div v, and
the Landau-Lifshitz stochastic stress
    Sigma = sqrt(2 eta kT) W~ + (sqrt(zeta kT / 3) - sqrt(2 eta kT) / 3) Tr(W~) I.

The paper defers the spatial discretisation to other work (App. A.1-A.2), so
the following is this project's reading, written in conservative (flux) form:

* rho at centres, g^alpha on alpha-faces; face density rho^alpha = average of
  the two adjacent centres; v^alpha = g^alpha / rho^alpha.
* The momentum flux T = g v + pi I - sigma - Sigma has its diagonal at cell
  centres and its off-diagonal on cell edges (the (alpha, beta) edge owned by
  cell i sits at r_i + h/2 (e_alpha + e_beta)).
* Advective parts are products of two-point averages; the viscous stress is
  sigma = eta (grad v + grad v^T) + (zeta - 2 eta / 3)(div v) I with centred
  differences, which makes div sigma equal to the paper's Laplacian form
  exactly on the staggered grid.
* W~ = (W + W^T) / sqrt(2): the text's (W + W^T)/2 would give half the
  Landau-Lifshitz covariance and half the equipartition velocity variance.
  With it, at a centre Sigma_aa = sqrt(2) S N_aa + sqrt(2)(B - S/3)(N_xx+N_yy+N_zz)
  and on an edge Sigma_ab = S N_ab, with S = sqrt(2 eta kT / (h^3 dt)),
  B = sqrt(zeta kT / (3 h^3 dt)) and N unit normals.
"""
from dataclasses import dataclass

import numpy as np

# array axis of each spatial direction (arrays are [z, y, x])
AXIS = (2, 1, 0)
EDGES = ((0, 1), (0, 2), (1, 2))      # (alpha, beta) pairs: xy, xz, yz


def up(a, d):
    """Field value at i + e_d (periodic)."""
    return np.roll(a, -1, axis=AXIS[d])


def dn(a, d):
    """Field value at i - e_d (periodic)."""
    return np.roll(a, 1, axis=AXIS[d])


@dataclass
class FluidParams:
    h: float = 1.0
    rho0: float = 1.0
    c: float = 4.0
    eta: float = 0.5
    zeta: float = 0.0
    kT: float = 0.0
    dt: float = 0.025


def noise_amplitudes(p):
    """(S, B) prefactors of the discrete stochastic stress."""
    vol_dt = p.h ** 3 * p.dt
    return np.sqrt(2.0 * p.eta * p.kT / vol_dt), np.sqrt(p.zeta * p.kT / (3.0 * vol_dt))


def rates(drho, g, p, pressure_extra=None, normals=None, face_force=None):
    """Time derivatives (d rho/dt, [d g^x/dt, d g^y/dt, d g^z/dt]).

    drho           : density excess rho - rho0 at centres (the constant p0 + c^2 rho0
                     of the equation of state p = p0 + c^2 rho, Sec. 3, has no gradient,
                     so the state is carried as rho - rho0 to avoid cancellation)
    g              : list of the three face momentum arrays
    pressure_extra : pressure added to c^2 rho at centres (particle term S Omega
                     plus the external drive), or None
    normals        : (6, ...) unit normals of this stage, rows xx, yy, zz, xy,
                     xz, yz (already combined as W_A + beta W_B), or None
    face_force     : list of three face arrays added to d g/dt (S F), or None
    """
    h = p.h
    # mass, Eq. (eq:consvDens)
    drho_dt = -sum(g[a] - dn(g[a], a) for a in range(3)) / h

    rho_face = [p.rho0 + 0.5 * (drho + up(drho, a)) for a in range(3)]
    v = [g[a] / rho_face[a] for a in range(3)]
    dv = [(v[a] - dn(v[a], a)) / h for a in range(3)]
    div_v = dv[0] + dv[1] + dv[2]

    pi = p.c ** 2 * drho
    if pressure_extra is not None:
        pi = pi + pressure_extra

    if normals is not None and p.kT > 0.0:
        s_amp, b_amp = noise_amplitudes(p)
        trace = normals[0] + normals[1] + normals[2]
        sig_cc = [np.sqrt(2.0) * s_amp * normals[a] + np.sqrt(2.0) * (b_amp - s_amp / 3.0) * trace
                  for a in range(3)]
        sig_e = [s_amp * normals[3 + e] for e in range(3)]
    else:
        sig_cc = [0.0, 0.0, 0.0]
        sig_e = [0.0, 0.0, 0.0]

    # diagonal of the momentum flux at centres
    t_cc = []
    for a in range(3):
        adv = 0.25 * (dn(g[a], a) + g[a]) * (dn(v[a], a) + v[a])
        visc = 2.0 * p.eta * dv[a] + (p.zeta - 2.0 * p.eta / 3.0) * div_v
        t_cc.append(adv + pi - visc - sig_cc[a])

    # off-diagonal fluxes on edges: flux[a][b] carries a-momentum along b
    flux = [[None] * 3 for _ in range(3)]
    for e, (a, b) in enumerate(EDGES):
        visc = p.eta * ((up(v[a], b) - v[a]) / h + (up(v[b], a) - v[b]) / h)
        flux[a][b] = 0.25 * (g[a] + up(g[a], b)) * (v[b] + up(v[b], a)) - visc - sig_e[e]
        flux[b][a] = 0.25 * (g[b] + up(g[b], a)) * (v[a] + up(v[a], b)) - visc - sig_e[e]

    # momentum, Eq. (eq:consvMom): minus the divergence of T over the face's control volume
    dg = []
    for a in range(3):
        div_t = up(t_cc[a], a) - t_cc[a]
        for b in range(3):
            if b != a:
                div_t = div_t + flux[a][b] - dn(flux[a][b], b)
        rate = -div_t / h
        if face_force is not None:
            rate = rate + face_force[a]
        dg.append(rate)
    return drho_dt, dg


# SSP-RK3 stage weights (App. A.2): U_{s+1} = a_s U^n + b_s (U_s + dU(U_s))
RK3_A = (0.0, 0.75, 1.0 / 3.0)
RK3_B = (1.0, 0.25, 2.0 / 3.0)
# noise combination W_s = W_A + beta_s W_B (App. A.2)
RK3_BETA = (-np.sqrt(3.0), np.sqrt(3.0), 0.0)
# time of each stage's flux evaluation, in units of dt after t^n
RK3_TIME = (0.0, 1.0, 0.5)


def rk3_combine(stage, u_n, u_s, du):
    """a_s U^n + b_s (U_s + dU) for one array."""
    a, b = RK3_A[stage], RK3_B[stage]
    if stage == 0:
        return u_s + du
    return a * u_n + b * (u_s + du)
