"""Closed forms the oracle is pinned against.

These are the paper's analytic results, restated:

* Eq. (eq:acousticForce2): primary radiation force of a standing wave
  F_1 = c_f^2 Delta rho^2 V k / (4 rho0) (f_1 + 3/2 f_2) sin(2 k z), with the
  monopole and dipole coefficients of Eqs. (f1), (f2).
* Eqs. (part_svel), (ke): c_p^2 = c_f^2 + epsilon, kappa_e = -epsilon kappa_f / c_p^2.
* Eq. (eq:densityVariance): Var[J rho] = rho0 kT / (c_p^2 V).
* App. A.1 / Table I: the forcing frequency of the driven mode equals the
  dispersion relation of the centred staggered operators,
  omega = (2 c / h) sin(k h / 2) (0.0784137 for h = 10, N = 32, c = 4).
"""
import numpy as np


def f1(kappa_ratio):
    """Monopole coefficient f_1 = 1 - kappa_p/kappa_f = -kappa_e/kappa_f (Eq. (f1))."""
    return 1.0 - np.asarray(kappa_ratio, dtype=np.float64)


def f2(m_e, rho0, vol):
    """Dipole coefficient f_2 = 2 m_e / (2 m_e + 3 rho0 V) (Eq. (f2))."""
    m_e = np.asarray(m_e, dtype=np.float64)
    return 2.0 * m_e / (2.0 * m_e + 3.0 * rho0 * vol)


def gorkov_force(c, drho, vol, k, rho0, kappa_ratio, m_e, z):
    """Primary radiation force on a particle at z in the wave cos(k z) (Eq. (eq:acousticForce2))."""
    return (c ** 2 * drho ** 2 * vol * k / (4.0 * rho0)
            * (f1(kappa_ratio) + 1.5 * f2(m_e, rho0, vol)) * np.sin(2.0 * k * z))


def particle_sound_speed(c, eps):
    """c_p = sqrt(c_f^2 + epsilon) (Eq. (part_svel))."""
    return np.sqrt(c ** 2 + np.asarray(eps, dtype=np.float64))


def excess_compressibility_ratio(c, eps):
    """kappa_e / kappa_f = -epsilon / c_p^2 (Eq. (ke))."""
    eps = np.asarray(eps, dtype=np.float64)
    return -eps / (c ** 2 + eps)


def kernel_density_variance(rho0, kT, c_p, vol):
    """Var[J rho] = rho0 kT / (c_p^2 V) (Eq. (eq:densityVariance))."""
    return rho0 * kT / (c_p ** 2 * vol)


def discrete_sound_frequency(c, h, n, nlambda=1):
    """omega of mode k = 2 pi nlambda / (n h) under centred staggered differences."""
    k = 2.0 * np.pi * nlambda / (n * h)
    return (2.0 * c / h) * np.sin(0.5 * k * h)


def resonant_amplitude(pressure_amp, gamma, omega):
    """Steady density amplitude of a mode driven at resonance by P sin(omega t).

    From delta rho'' + 2 Gamma k^2 delta rho' + c^2 k^2 delta rho = -k^2 p(t) at
    omega = c k (the resonance case of the paper's linear response, Sec. 6).
    """
    return pressure_amp / (2.0 * gamma * omega)
