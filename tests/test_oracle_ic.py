"""Pins of the oracle's IC step (Secs. 3-4, App. A.2)."""
import numpy as np
import pytest

from oracle import ic, peskin, theory


def make_sim(n=10, kT=0.0, seed=3, form="g", forcing="none", wave_amp=0.0, nparts=4, m_e=4.0,
             kappa=0.5, k_spring=0.0, rng_seed=0):
    p = ic.GridParams(nx=n, ny=n + 1, nz=n + 2, kT=kT, seed=seed, momentum_form=form,
                      forcing=forcing, wave_amp=wave_amp, zeta=0.3)
    rng = np.random.default_rng(rng_seed)
    rho = 1.0 + 2e-3 * rng.uniform(-1, 1, p.shape)
    g = [2e-3 * rng.uniform(-1, 1, p.shape) for _ in range(3)]
    s = ic.Simulation(p, rho, g)
    q = rng.uniform(0, 1, (nparts, 3)) * p.lengths
    s.add_particles(q, m_e, kappa, k_spring)
    return s


def test_particle_pressure_average_is_epsilon_times_density_excess():
    """J[S Omega] = epsilon (J rho - rho0) for one particle, since J S = 1/V (Eqs. (kvol), (omega), (jdp))."""
    p = ic.GridParams(nx=9, ny=9, nz=9, h=0.8)
    rng = np.random.default_rng(2)
    rho = 1.0 + 1e-2 * rng.normal(size=p.shape)
    for q in rng.uniform(0, 9 * 0.8, (5, 3)):
        centre = peskin.Stencils(q[None], p.h, p.shape, peskin.CENTRE)
        eps = np.array([7.5])
        pp = ic.particle_pressure(centre, rho - p.rho0, eps, p)
        assert centre.interp(pp)[0] == pytest.approx(eps[0] * (centre.interp(rho)[0] - 1.0), rel=1e-12)
        # uniform density excess: J[c^2 drho + S Omega] = (c^2 + epsilon) drho (Eq. (jdp))
        d = 3e-3
        pp_u = ic.particle_pressure(centre, np.full(p.shape, d), eps, p)
        assert centre.interp(p.c ** 2 * d + pp_u)[0] == pytest.approx((p.c ** 2 + eps[0]) * d, rel=1e-12)


def test_sound_speed_and_compressibility_maps():
    """c_p = 2 c_f gives kappa_e = -3/4 kappa_f (Sec. 6.1); kappa_p/kappa_f = 0.5 gives epsilon = c_f^2."""
    c = 4.0
    eps = ic.epsilon_from_kappa_ratio(0.25, c)           # kappa_p/kappa_f = (c_f/c_p)^2 = 1/4
    assert theory.particle_sound_speed(c, eps) == pytest.approx(2 * c)
    assert theory.excess_compressibility_ratio(c, eps) == pytest.approx(-0.75)
    assert ic.epsilon_from_kappa_ratio(0.5, c) == pytest.approx(c ** 2)
    assert theory.f1(0.5) == pytest.approx(0.5)
    assert theory.f2(4.0, 1.0, 8.0) == pytest.approx(0.25)


@pytest.mark.parametrize("kT", [0.0, 1e-3])
def test_total_momentum_conserved_with_overlapping_particles(kT):
    """With F = 0, m_e u + h^3 sum g is a constant of motion (Eq. (eq:totmom)), to rounding."""
    s = make_sim(kT=kT, nparts=6)
    # force two overlapping kernels
    s.parts.q[1] = s.parts.q[0] + np.array([1.1, -0.6, 0.9])
    p0 = s.total_momentum()
    for _ in range(15):
        s.step()
    assert np.allclose(s.total_momentum(), p0, rtol=0, atol=1e-15)
    assert np.max(np.abs(s.parts.u)) > 1e-5


def test_spring_momentum_balance():
    """Total momentum changes by exactly dt sum_p F^{n+1/2} per step (substeps 3-6)."""
    s = make_sim(nparts=3, k_spring=0.7)
    s.parts.q_eq = s.parts.q + 0.3                    # loaded springs
    for _ in range(5):
        p0 = s.total_momentum()
        s.step()
        f = s.last["force"].sum(axis=0)
        assert np.allclose(s.total_momentum() - p0, s.p.dt * f, rtol=0, atol=1e-16)
        assert np.max(np.abs(f)) > 0.05


def test_neutrally_buoyant_particle_leaves_fluid_untouched():
    """m_e = 0: dg = 0, so g^{n+1} = g~^{n+1} and u^{n+1} = J v~^{n+1} (App. A.2 substep 6 remark)."""
    s = make_sim(nparts=3, m_e=0.0, kT=1e-3)
    s.step()
    for a in range(3):
        assert np.array_equal(s.g[a], s.last["g_tilde"][a])
    assert np.array_equal(s.parts.u, s.last["jv_tilde"])


def test_v_form_enforces_no_slip_exactly():
    """Paper's velocity form of substep 6: u^{n+1} = J^{n+1/2} v^{n+1} (App. A.2)."""
    s = make_sim(nparts=1, form="v", m_e=5.0, kT=1e-3)
    for _ in range(3):
        s.step()
        c, faces = peskin.all_stencils(s.last["q_half"], s.p.h, s.p.shape)
        v = s.velocities()
        jv = np.stack([faces[a].interp(v[a]) for a in range(3)], axis=1)
        assert np.allclose(jv, s.parts.u, rtol=0, atol=1e-16)


def test_g_form_no_slip_holds_to_density_order():
    """g form: u^{n+1} = J v^{n+1} up to O(delta rho / rho0) of the impulse."""
    s = make_sim(nparts=1, m_e=5.0)
    s.step()
    c, faces = peskin.all_stencils(s.last["q_half"], s.p.h, s.p.shape)
    v = s.velocities()
    jv = np.stack([faces[a].interp(v[a]) for a in range(3)], axis=1)
    dmax = np.max(np.abs(s.drho))
    err = np.abs(jv - s.parts.u)
    assert np.all(err <= 4 * dmax * np.abs(s.last["dg"]) / s.last["m_f"][:, None] + 1e-17)


def test_impulse_formulas():
    """Substeps 4-5: dg = m_e m_f/(m_e+m_f)(Jv~ - u^n) and u^{n+1} - u^n = dg / m_e."""
    s = make_sim(nparts=4, m_e=3.0, kT=1e-3)
    u0 = s.parts.u.copy()
    s.step()
    assert np.allclose(s.parts.u - u0, s.last["dg"] / 3.0, rtol=1e-12, atol=1e-18)
    lam = s.last["lam"]
    assert np.allclose(lam, s.last["dg"] / s.p.dt - s.last["force"], rtol=1e-14, atol=1e-18)


def test_particles_are_advected_with_a_uniform_flow():
    """A uniform flow v0 moves a neutrally buoyant particle by v0 dt per step (substeps 1, 7)."""
    p = ic.GridParams(nx=8, ny=8, nz=8, eta=0.5)
    v0 = np.array([0.01, -0.02, 0.005])
    g = [np.full(p.shape, v0[a]) for a in range(3)]
    s = ic.Simulation(p, np.full(p.shape, 1.0), g)
    s.add_particles([[3.3, 4.1, 2.7]], 0.0, 1.0)
    q0 = s.parts.q.copy()
    for _ in range(4):
        s.step()
    assert np.allclose(s.parts.q, q0 + 4 * p.dt * v0, atol=1e-14)
    assert np.allclose(s.parts.u, v0[None], atol=1e-15)
