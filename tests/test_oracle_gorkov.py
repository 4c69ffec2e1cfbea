"""The whole method, on the oracle, against the primary radiation force of a
standing wave: Eq. (eq:acousticForce2) with the monopole and dipole
coefficients f_1, f_2 of Eqs. (f1), (f2).

The force is read as the paper does (Sec. 6): two mirrored particles tethered
by springs, the radiation force minus the windowed time average of the spring
force, Gor'kov evaluated at the measured mode amplitude <A^2>_w.  The run is
in the regime of Table I (cells of h = 10, c_f = 4, eta = 0.5,
dt = 0.1 h / c_f, so the viscous length is about a quarter of the particle
radius) on a 16^3 box to keep the oracle's cost down: the dipolar case
m_e = m_f (rho_p = 2 rho0), c_p = c_f (f_1 = 0, f_2 = 0.4), for which the
paper reports agreement within 1.5 % at 32^3.  Here it comes out within
1.5 % too; the test allows 5 %.

Outside that regime Gor'kov's inviscid force is not the method's limit: in the
h = 1 box of the single-particle configuration the viscous length is about
the particle radius, and the converged oracle force is 0.57 of Gor'kov (see
tests/golden/config1_force.json and the GPU test that checks the library
against it).
"""
import numpy as np
import pytest

from oracle import ic as oic
from oracle import theory
from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.slow


def test_dipolar_force_paper_regime_on_the_oracle():
    n, h, nsteps, skip = 16, 10.0, 24000, 8000
    mass_ratio, kappa_ratio, k_s = 2.0, 1.0, 1.0
    gp, _, _ = W.single_particle_config(n=n, k_spring=k_s, mirror=True, mass_ratio=mass_ratio,
                                        kappa_ratio=kappa_ratio)
    gp.update(h=h, dt=0.1 * h / gp["c"], zeta=1.0)
    L = n * h
    q = np.array([[L / 8, L / 2, L / 2], [7 * L / 8, L / 2, L / 2]])
    vol = 8.0 * h ** 3
    m_e = (mass_ratio - 1.0) * vol
    p = oic.GridParams(**{k: v for k, v in gp.items() if k in oic.GridParams.__dataclass_fields__})
    rho, g = W.velocity_phase_wave_fields(gp)
    sim = oic.Simulation(p, rho, g)
    sim.add_particles(q, m_e, kappa_ratio, k_s)
    sim.run(nsteps, W.blackman_harris(nsteps, skip))
    f, _, a2 = sim.time_average()
    fg = theory.gorkov_force(p.c, np.sqrt(2.0 * a2), vol, 2.0 * np.pi / L, p.rho0, kappa_ratio, m_e, L / 8)
    r1, r2 = -f[0, 0] / fg, f[1, 0] / fg
    assert abs(np.sqrt(2.0 * a2) - 1e-3) < 2e-5          # the drive holds the mode at A = 1e-3
    assert r1 == pytest.approx(r2, rel=1e-6)             # mirror symmetry
    assert r1 == pytest.approx(1.0, abs=0.05), r1
