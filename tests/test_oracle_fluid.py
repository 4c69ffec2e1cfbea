"""Pins of the oracle's fluid solver (Sec. 4.2, App. A.2, Table I)."""
import os

import numpy as np
import pytest
from scipy.optimize import curve_fit

from oracle import fluid, ic, theory

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table1():
    vals = {}
    with open(os.path.join(GOLDEN, "table1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def run_trace(p, nsteps, rho=None, g=None, probe=None):
    s = ic.Simulation(p, rho, g)
    out = np.empty(nsteps + 1)
    probe = probe or (lambda sim: ic.mode_amplitude(p, sim.drho))
    out[0] = probe(s)
    for i in range(nsteps):
        s.step()
        out[i + 1] = probe(s)
    return s, out


def test_mass_and_momentum_conserved_with_noise():
    p = ic.GridParams(nx=6, ny=5, nz=7, kT=1e-2, zeta=0.3, seed=4)
    rng = np.random.default_rng(1)
    rho = 1.0 + 1e-2 * rng.uniform(-1, 1, p.shape)
    g = [1e-2 * rng.uniform(-1, 1, p.shape) for _ in range(3)]
    s = ic.Simulation(p, rho, g)
    m0, p0 = s.drho.sum(), s.total_momentum()
    s.run(20)
    assert abs(s.drho.sum() - m0) < 1e-13
    assert np.allclose(s.total_momentum(), p0, atol=1e-14)
    assert np.max(np.abs(s.g[0] - g[0])) > 1e-4          # something happened


def test_sound_frequency_matches_table1():
    """Inviscid standing wave oscillates at Table I's omega = 0.0784137."""
    t1 = table1()
    h, n, c = t1["h"], int(t1["cells"]), t1["c_f"]
    dt = 0.1 * h / c
    p = ic.GridParams(nx=n, ny=4, nz=4, h=h, c=c, eta=0.0, zeta=0.0, dt=dt, wave_amp=1e-7)
    period = 2 * np.pi / 0.0784
    nsteps = int(0.8 * period / dt)
    _, a = run_trace(p, nsteps)
    t = dt * np.arange(nsteps + 1)
    # first zero crossing of A0 cos(omega t): linear interpolation is exact to O(dt^3) there
    i = np.nonzero(np.sign(a[1:]) != np.sign(a[:-1]))[0]
    crossings = [t[j] + dt * a[j] / (a[j] - a[j + 1]) for j in i]
    omega = (np.pi / 2) / crossings[0]
    assert omega == pytest.approx(t1["omega_fig4"], abs=6e-8)
    assert omega == pytest.approx(theory.discrete_sound_frequency(c, h, n), rel=1e-6)
    assert abs(omega - 2 * np.pi * c / (n * h)) > 1e-4      # not the continuum value


def test_shear_mode_decays_at_eta_k2():
    """A transverse mode g_y = B cos(k x) decays at (eta/rho0) k~^2 with k~ = (2/h) sin(kh/2)."""
    p = ic.GridParams(nx=16, ny=4, nz=4, h=1.0, eta=0.7, zeta=0.4, c=4.0)
    k = 2 * np.pi / 16
    x = np.arange(16) * p.h
    rho = np.full(p.shape, 1.0)
    g = [np.zeros(p.shape), np.broadcast_to(1e-6 * np.cos(k * x), p.shape).copy(), np.zeros(p.shape)]
    probe = lambda sim: 2 * np.mean(sim.g[1] * np.cos(k * ic.axis_coordinate(p, 0)))
    nsteps = 400
    _, b = run_trace(p, nsteps, rho, g, probe)
    rate = -np.log(b[-1] / b[0]) / (nsteps * p.dt)
    kd2 = (2 / p.h * np.sin(k * p.h / 2)) ** 2
    assert rate == pytest.approx(p.eta / p.rho0 * kd2, rel=1e-5)


@pytest.mark.parametrize("eta,zeta", [(0.5, 0.0), (0.2, 0.9)])
def test_sound_mode_decays_at_gamma_k2(eta, zeta):
    """A sound mode decays at Gamma k~^2 with Gamma = (4 eta/3 + zeta) / (2 rho0) (Sec. 6)."""
    p = ic.GridParams(nx=16, ny=4, nz=4, eta=eta, zeta=zeta, wave_amp=1e-7)
    nsteps = 1200
    _, a = run_trace(p, nsteps)
    t = p.dt * np.arange(nsteps + 1)
    model = lambda t, a0, b0, gam, om: np.exp(-gam * t) * (a0 * np.cos(om * t) + b0 * np.sin(om * t))
    _, kd, omega, gamma = ic.wave_numbers(p)
    popt, _ = curve_fit(model, t, a / 1e-7, p0=[1.0, 0.0, gamma * kd ** 2, omega], xtol=1e-14, ftol=1e-14)
    assert popt[2] == pytest.approx(gamma * kd ** 2, rel=2e-4)
    assert popt[3] == pytest.approx(np.sqrt(omega ** 2 - (gamma * kd ** 2) ** 2), rel=1e-5)


@pytest.mark.parametrize("forcing", ["mode", "plane"])
def test_driven_mode_holds_amplitude(forcing):
    """The resonant drive keeps the k mode at the target amplitude A (linear response, Sec. 6)."""
    A = 1e-6
    p = ic.GridParams(nx=16, ny=4, nz=4, eta=0.5, zeta=0.5, wave_amp=A, forcing=forcing)
    _, kd, omega, gamma = ic.wave_numbers(p)
    period = 2 * np.pi / omega
    nsteps = int(6 * period / p.dt)
    _, a = run_trace(p, nsteps)
    last = a[-int(period / p.dt) - 2:]
    tol = 2e-3 if forcing == "mode" else 2e-2          # the plane also excites other modes
    assert np.max(np.abs(last)) == pytest.approx(A, rel=tol)


def test_equipartition_and_density_variance():
    """Thermal fluid: <v^2> = kT / (rho0 h^3) per face, <drho^2> = rho0 kT / (c^2 h^3).

    The initial sample is the Gibbs state; after the short-wavelength modes have
    relaxed several times, a noise normalisation off by a factor would show.
    """
    p = ic.GridParams(nx=8, ny=8, nz=8, h=1.0, kT=1e-4, eta=0.5, zeta=0.5, seed=21)
    rho, g = ic.thermal_state(p, seed=99)
    s = ic.Simulation(p, rho, g)
    s.run(100)
    v2, r2 = [], []
    for i in range(500):
        s.step()
        if i % 2 == 0:
            v = s.velocities()
            v2.append(np.mean([np.mean(v[a] ** 2) for a in range(3)]))
            r2.append(np.mean(s.drho ** 2))
    expect_v = p.kT / (p.rho0 * p.h ** 3)
    expect_r = p.rho0 * p.kT / (p.c ** 2 * p.h ** 3)
    # <v^2> per face, and the total of N^3 - 1 nonzero density modes
    assert np.mean(v2) == pytest.approx(expect_v * (1 - 1 / 512), rel=0.04)
    assert np.mean(r2) == pytest.approx(expect_r * (1 - 1 / 512), rel=0.04)


def test_thermal_state_statistics():
    p = ic.GridParams(nx=16, ny=16, nz=16, kT=2e-3, c=3.0)
    rho, g = ic.thermal_state(p, seed=5)
    assert abs(np.mean(rho) - p.rho0) < 1e-15
    assert np.mean((rho - p.rho0) ** 2) == pytest.approx(p.rho0 * p.kT / p.c ** 2, rel=0.05)
    for a in range(3):
        assert abs(np.mean(g[a])) < 1e-16
        assert np.mean(g[a] ** 2) == pytest.approx(p.rho0 * p.kT, rel=0.05)


# ---- the advective flux against the continuum term of Eq. (eq:consvMom) ----
def _smooth_flow(x, y, z):
    """A smooth periodic flow on [0, 2 pi)^3 (trigonometric polynomials, so
    rho v_a v_b is band-limited well below the grids' Nyquist wavenumber)."""
    rho = 1.0 + 0.3 * np.sin(x) * np.cos(2 * y) + 0.2 * np.cos(z + 0.3) + 0.1 * np.sin(x + y + z)
    v = (0.4 * np.sin(y + 0.4) + 0.3 * np.cos(z) + 0.2 * np.sin(x),
         0.5 * np.cos(x) * np.sin(z + 0.2) + 0.1 * np.cos(y),
         0.3 * np.sin(x + y) + 0.2 * np.cos(2 * x - z))
    return rho, v


def _advection_error(n):
    """max |discrete - continuum| / max |continuum| of the advective momentum
    tendency -d_b (rho v_a v_b) at the a-faces of an n^3 grid."""
    h = 2 * np.pi / n
    idx = np.arange(n) * h
    k = 2 * np.pi * np.fft.fftfreq(n, d=h)

    def points(shift):   # coordinates [z][y][x] of the cells shifted by shift * h/2
        z, y, x = np.meshgrid(idx + 0.5 * h * shift[2], idx + 0.5 * h * shift[1], idx + 0.5 * h * shift[0],
                              indexing="ij")
        return x, y, z

    rho_c, _ = _smooth_flow(*points((0, 0, 0)))
    g, exact = [], []
    for a in range(3):
        shift = tuple(1 if b == a else 0 for b in range(3))
        rho_f, v_f = _smooth_flow(*points(shift))
        g.append(rho_f * v_f[a])
        # continuum: -sum_b d_b (rho v_a v_b) at the a-faces, by exact spectral derivatives
        t = np.zeros_like(rho_f)
        for b in range(3):
            ax = fluid.AXIS[b]
            kk = k.reshape([-1 if i == ax else 1 for i in range(3)])
            t -= np.real(np.fft.ifft(1j * kk * np.fft.fft(rho_f * v_f[a] * v_f[b], axis=ax), axis=ax))
        exact.append(t)
    p = fluid.FluidParams(h=h, rho0=1.0, c=1.0, eta=0.0, zeta=0.0, kT=0.0)
    drho = rho_c - 1.0
    _, dg = fluid.rates(drho, g, p)
    _, dg0 = fluid.rates(drho, [np.zeros_like(drho)] * 3, p)   # the pressure gradient alone
    scale = max(np.max(np.abs(e)) for e in exact)
    return max(np.max(np.abs((dg[a] - dg0[a]) - exact[a])) for a in range(3)) / scale


def test_advective_flux_converges_to_the_continuum_at_second_order():
    """The advective part of the discrete momentum rate (the products of
    two-point averages on the staggered grid, a reading of the discretisation
    the paper defers) tends to the paper's continuum -div(g v) of
    Eq. (eq:consvMom) with the error falling 4x per halving of h.  A wrong
    average, index, operand or sign in any of the nine flux components leaves
    an O(1) or O(h) error instead."""
    e16, e32, e64 = (_advection_error(n) for n in (16, 32, 64))
    assert e64 < 1e-2
    assert 3.6 < e16 / e32 < 4.4 and 3.8 < e32 / e64 < 4.2, (e16, e32, e64)


def _viscous_and_mass_errors(n, eta=0.7, zeta=0.4):
    """Relative errors, on an n^3 grid, of the discrete viscous momentum rate
    against eta lap v + (zeta + eta/3) grad div v (Sec. 4.2) at the faces, and
    of the mass rate against -div g at the centres (uniform density, so that
    v = g / rho0 exactly and the pressure has no gradient)."""
    h = 2 * np.pi / n
    idx = np.arange(n) * h
    k = 2 * np.pi * np.fft.fftfreq(n, d=h)
    kk = [k.reshape([-1 if i == fluid.AXIS[b] else 1 for i in range(3)]) for b in range(3)]

    def points(shift):
        z, y, x = np.meshgrid(idx + 0.5 * h * shift[2], idx + 0.5 * h * shift[1], idx + 0.5 * h * shift[0],
                              indexing="ij")
        return x, y, z

    def d(f, b):   # exact spectral derivative along axis b
        return np.real(np.fft.ifft(1j * kk[b] * np.fft.fft(f, axis=fluid.AXIS[b]), axis=fluid.AXIS[b]))

    rho0 = 1.3
    g, exact_g = [], []
    for a in range(3):
        shift = tuple(1 if b == a else 0 for b in range(3))
        x, y, z = points(shift)
        _, v = _smooth_flow(x, y, z)
        g.append(rho0 * v[a])
        # eta lap v_a + (zeta + eta/3) d_a div v, every term by spectral derivatives on the a-face grid
        lap = sum(d(d(v[a], b), b) for b in range(3))
        grad_div = sum(d(d(v[b], b), a) for b in range(3))
        exact_g.append(eta * lap + (zeta + eta / 3.0) * grad_div)
    # -div g at the centres: each g_a is sampled on its face grid, so differentiate there and shift to the centres
    xc, yc, zc = points((0, 0, 0))
    _, vc = _smooth_flow(xc, yc, zc)
    exact_rho = -sum(rho0 * d(vc[a], a) for a in range(3))
    zero = np.zeros((n, n, n))
    visc = fluid.FluidParams(h=h, rho0=rho0, c=1.0, eta=eta, zeta=zeta, kT=0.0)
    invisc = fluid.FluidParams(h=h, rho0=rho0, c=1.0, eta=0.0, zeta=0.0, kT=0.0)
    drho_dt, dg = fluid.rates(zero, g, visc)
    _, dg0 = fluid.rates(zero, g, invisc)
    sg = max(np.max(np.abs(e)) for e in exact_g)
    err_g = max(np.max(np.abs((dg[a] - dg0[a]) - exact_g[a])) for a in range(3)) / sg
    err_rho = np.max(np.abs(drho_dt - exact_rho)) / np.max(np.abs(exact_rho))
    return err_g, err_rho


def test_viscous_and_mass_rates_converge_to_the_continuum_at_second_order():
    """The viscous part of the discrete momentum rate tends to the paper's
    eta lap v + (zeta + eta/3) grad div v, with its cross terms, and the
    discrete mass rate to -div g (Eq. (eq:consvDens)), both with the error
    falling 4x per halving of h on a general smooth flow (beyond the single
    Fourier modes whose decay rates pin the same operators exactly)."""
    (g16, r16), (g32, r32), (g64, r64) = (_viscous_and_mass_errors(n) for n in (16, 32, 64))
    assert g64 < 1e-2 and r64 < 1e-2, (g64, r64)
    assert 3.6 < g16 / g32 < 4.4 and 3.8 < g32 / g64 < 4.2, (g16, g32, g64)
    assert 3.6 < r16 / r32 < 4.4 and 3.8 < r32 / r64 < 4.2, (r16, r32, r64)


def _rk3_mode_error(dt, T=4.0, amp=1e-9):
    """Relative error at time T of the oracle's step against the exact
    solution of the semi-discrete linear dynamics in the invariant subspace of
    one x-mode: delta rho in span{cos k x_i, sin k x_i}, g_x in span{cos k
    x_(i+1/2), sin k x_(i+1/2)} (k = 2 pi / 16).  The 4 x 4 generator comes
    from central differences of the rates, its exponential from scipy."""
    from scipy.linalg import expm

    n = 16
    p = ic.GridParams(nx=n, ny=6, nz=6, h=1.0, rho0=1.0, c=4.0, eta=0.5, zeta=0.3, kT=0.0, dt=dt)
    shape = p.shape
    kx = 2 * np.pi / n
    xc = np.broadcast_to(np.arange(n, dtype=float), shape)
    xf = xc + 0.5
    basis = [np.cos(kx * xc), np.sin(kx * xc), np.cos(kx * xf), np.sin(kx * xf)]   # drho, drho, g_x, g_x
    zero = np.zeros(shape)

    def fields(y):
        return y[0] * basis[0] + y[1] * basis[1], [y[2] * basis[2] + y[3] * basis[3], zero, zero]

    def coords(drho, gx):   # orthogonal projection onto the basis
        return np.array([np.sum(drho * basis[0]), np.sum(drho * basis[1]), np.sum(gx * basis[2]),
                         np.sum(gx * basis[3])]) / (0.5 * basis[0].size)

    fp, eps = p.fluid(), 1e-6
    M = np.zeros((4, 4))
    for j in range(4):
        e = np.zeros(4)
        e[j] = eps
        rp, gp = fluid.rates(*fields(e), fp)
        rm, gm = fluid.rates(*fields(-e), fp)
        M[:, j] = coords((rp - rm) / (2 * eps), (gp[0] - gm[0]) / (2 * eps))
    y0 = amp * np.array([1.0, 0.3, 0.5, -0.2])
    exact = expm(M * T) @ y0
    drho, g = fields(y0)
    sim = ic.Simulation(p, g=g, drho=drho)
    for _ in range(int(round(T / dt))):
        sim.step()
    return np.linalg.norm(coords(sim.drho, sim.g[0]) - exact) / np.linalg.norm(exact)


def test_ssp_rk3_is_third_order_in_time():
    """The three stages with the weights (1, 0), (3/4, 1/4), (1/3, 2/3) of
    App. A.2 integrate the semi-discrete equations to third order: on a
    damped sound mode (viscous and bulk terms included) the error at a fixed
    time falls 8x per halving of dt.  A wrong stage weight or stage input
    lowers the order."""
    e1, e2, e3 = (_rk3_mode_error(dt) for dt in (0.05, 0.025, 0.0125))
    assert 7.0 < e1 / e2 < 9.0 and 7.0 < e2 / e3 < 9.0, (e1, e2, e3)
