"""The paper's validation sweeps on the GPU, against its closed forms.

* Primary radiation force in the Table I regime (h = 10, 32^3 cells, c_f = 4,
  eta = 0.5), a mirrored pair of tethered particles (Sec. 6), the force read
  as minus the windowed average of the spring force and compared with
  Gor'kov (Eq. (eq:acousticForce2)) at the measured <A^2>; a tether acts at
  the drive frequency as an excess mass -k_s / omega^2, which enters f2.
  Swept as in Fig. 3 (particle sound speed c_p / c_f at rho_p = rho0: the
  monopolar term f1 of Eq. (f1); the paper finds it ~10 % below the
  infinite-box value at L = 32) and Fig. 4 (density ratio rho_p / rho0 at
  c_p = c_f: the dipolar term f2 of Eq. (f2), within ~1.5 % in the paper).
  The sweeps use the mode drive (a body pressure on the driven mode alone);
  the paper's own layout -- a drive on one grid plane (Eq. (pext)), wave along
  z, particles at (1/2, 1/2, 3/8) L and (0, 0, -3/8) L -- is checked at two
  points.
* Thermal compressibility (Sec. 4.4, Eq. (eq:densityVariance)): J rho of
  neutrally buoyant particles is Gaussian with variance rho0 kT / (c_p^2 V)
  for c_p from c_f / 2 to 2 c_f, and its error grows with the CFL number
  alpha = c_p dt / h (Fig. 7): at c_p = 4 c_f halving dt cuts it several-fold.
"""
import numpy as np
import pytest

from oracle import theory
from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def pair_force_ratio(mass_ratio, kappa_ratio, k_s, zeta, drive="mode", nsteps=24000, skip=8000,
                     paper_layout=False):
    """Measured / Gor'kov force on the pair (both particles).  drive="plane":
    the paper's setup of Sec. 6 (wave along z, paper_protocol_config);
    drive="mode": the wave along x, the pair at L/8 and 7L/8 on one line, or
    with paper_layout at the paper's places (3L/8 and 5L/8 along the wave,
    transverse (L/2, L/2) and (0, 0))."""
    from paper_1307_0702_gb300 import Grid

    h = 10.0
    if drive == "plane":
        gp, parts = W.paper_protocol_config(mass_ratio, kappa_ratio, k_s, zeta, h=h)
        ax = 2
    else:
        gp, parts, _ = W.single_particle_config(n=32, k_spring=k_s, mirror=True, mass_ratio=mass_ratio,
                                                kappa_ratio=kappa_ratio)
        gp.update(h=h, dt=0.1 * h / gp["c"], zeta=zeta, precision="fp32")
        L = 32 * h
        parts["q"] = np.array([[L / 8, L / 2, L / 2], [7 * L / 8, L / 2, L / 2]])
        if paper_layout:
            parts["q"] = np.array([[3 * L / 8, L / 2, L / 2], [5 * L / 8, 0.0, 0.0]])
        parts["m_e"] = np.full(2, (mass_ratio - 1.0) * 8 * h ** 3)
        ax = 0
    rho, g = W.velocity_phase_wave_fields(gp)
    w = W.blackman_harris(nsteps, skip)
    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
        grid.step(nsteps, w)
        f, _, a2 = grid.time_average()
    L = 32 * h
    k = 2 * np.pi / L
    omega = theory.discrete_sound_frequency(gp["c"], h, 32)
    m_eff = parts["m_e"][0] - k_s / omega ** 2
    fg = [theory.gorkov_force(gp["c"], np.sqrt(2 * a2), 8 * h ** 3, k, gp["rho0"], kappa_ratio, m_eff,
                              parts["q"][j, ax]) for j in range(2)]
    return np.array([-f[j, ax] / fg[j] for j in range(2)]), np.array([-f[j, ax] for j in range(2)])


def test_fig3_monopolar_force_over_particle_sound_speed():
    ratios, forces = [], []
    for cp_over_cf in (1.5, 2.0, 4.0):
        r, f = pair_force_ratio(1.0, 1.0 / cp_over_cf ** 2, k_s=0.5, zeta=0.5)
        assert r[0] == pytest.approx(r[1], rel=2e-3)          # the mirror particle
        ratios.append(r[0])
        forces.append(abs(f[0]))
    assert forces[0] < forces[1] < forces[2]                  # f1 = 1 - (c_f / c_p)^2 grows with c_p
    for r in ratios:
        assert 0.85 <= r <= 1.0, ratios                       # the paper's finite-size deficit at L = 32


def test_fig4_dipolar_force_over_density_ratio():
    ratios = []
    for rho_ratio in (0.5, 2.0, 5.0):
        # long runs: the heaviest tethered particle rings at sqrt(k_s / m_p) for ~10^4 steps
        r, _ = pair_force_ratio(rho_ratio, 1.0, k_s=1.0, zeta=1.0, nsteps=64000, skip=16000)
        assert r[0] == pytest.approx(r[1], rel=2e-3)
        ratios.append(r[0])
    # the viscous layer (delta = sqrt(2 nu / omega) ~ 0.4 R_H here) raises the dipolar
    # force of dense particles above the inviscid Gor'kov value (the paper: ~2 %)
    for r in ratios:
        assert 0.97 <= r <= 1.07, ratios


def test_paper_layout_with_plane_drive():
    """Sec. 6 as written: one-plane drive (Eq. (pext)), wave along z, particles
    at (1/2, 1/2, 3/8) L and (0, 0, -3/8) L.

    The drive does not change the force: a drive on one plane forces every
    Fourier mode of the wave axis alike, each harmonic answers off resonance
    in phase with the drive, a quadrature away from the resonant mode, and the
    cross terms average out.  The mode drive with the particles at the same
    places gives the same ratios (measured after 24000 steps: dipole 1.1005
    vs 1.1001, monopole 0.9127 vs 0.9130).

    The layout does.  After 24000 steps the tethered particle's first-order
    ringing (period ~3200 steps, lightly damped) still leaks into the window,
    with the sign of the wave at the particle: the dipole reads 1.034 at
    L/8 and 1.072 at 3L/8 on one line, and both settle at 1.051 after 128000
    steps.  The paper's transverse offset of the mirror particle adds ~1 % to
    the settled dipole (1.061).  The monopole of a pair on one line, 8 cells
    apart along the wave, drifts (0.89, 0.86, 0.84 at 24k, 64k, 128k steps);
    with the paper's offset it stays at 0.913."""
    for args in [(1.0, 0.25, 0.5, 0.5), (2.0, 1.0, 1.0, 1.0)]:
        r_plane, _ = pair_force_ratio(*args[:2], k_s=args[2], zeta=args[3], drive="plane")
        r_mode, _ = pair_force_ratio(*args[:2], k_s=args[2], zeta=args[3], drive="mode", paper_layout=True)
        assert r_plane[0] == pytest.approx(r_plane[1], rel=2e-3)
        assert r_plane[0] == pytest.approx(r_mode[0], rel=3e-3), (args, r_plane, r_mode)
    assert r_plane[0] == pytest.approx(1.100, abs=0.01)          # the dipole, unsettled
    r_long, _ = pair_force_ratio(2.0, 1.0, k_s=1.0, zeta=1.0, drive="plane", nsteps=128000, skip=32000)
    assert r_long[0] == pytest.approx(1.061, abs=0.008), r_long  # settled: Fig. 4's 1.05 plus the layout's 1 %


def test_plane_drive_harmonics():
    """The plane drive's spectrum along the wave axis (no particles, 4
    periods after 8000 steps): the resonant mode at the set amplitude 1e-3
    rho0 (rms 7.07e-4); modes 3-16 at ~0.83 % of it each, the flat spectrum
    of a forcing on one plane answered off resonance; mode 2 at ~1.8 %, that
    plus the advective second harmonic (1.3 % under the mode drive too)."""
    from paper_1307_0702_gb300 import Grid

    gp, _ = W.paper_protocol_config(2.0, 1.0, 1.0, 1.0, h=10.0)
    omega = theory.discrete_sound_frequency(gp["c"], gp["h"], 32)
    per = int(round(2 * np.pi / omega / gp["dt"]))
    rho, g = W.velocity_phase_wave_fields(gp)
    prof = []
    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.step(8000)
        for _ in range(per):
            grid.step(4)
            prof.append((grid.get_state()[0] - gp["rho0"]).mean(axis=(1, 2)))
    amp = np.sqrt(np.mean(np.abs(np.fft.rfft(np.array(prof), axis=1) / 16) ** 2, axis=0))
    assert amp[1] == pytest.approx(1e-3 / np.sqrt(2), rel=5e-3)
    assert amp[2] < 0.025 * amp[1], amp / amp[1]
    assert np.all(amp[3:] < 0.012 * amp[1]), amp / amp[1]
    assert np.all(amp[3:] > 0.006 * amp[1]), amp / amp[1]       # the harmonics are there


def density_samples(cp_over_cf, dt_factor=1.0, n=48, warm=400, samples=300, every=8):
    from paper_1307_0702_gb300 import Grid

    gp = W.grid_params(n, kT=1e-3, wave_amp=0.0, forcing="none", zeta=0.5, seed=21, precision="fp32")
    gp["dt"] *= dt_factor
    rng = np.random.default_rng(9)
    pts = np.stack(np.meshgrid(*[np.arange(0, n, 4.0)] * 3, indexing="ij"), -1).reshape(-1, 3)
    q = pts + rng.uniform(0, 1, pts.shape)    # lattice of spacing 4h: kernels do not overlap
    out = []
    with Grid(gp) as grid:
        grid.set_state(np.full((n, n, n), 1.0))
        grid.init_thermal(6)
        grid.add_particles(q, 0.0, 1.0 / cp_over_cf ** 2)
        grid.step(int(warm / dt_factor))
        for _ in range(samples):
            grid.step(int(every / dt_factor))
            out.append(grid.particle_density())
    s = np.array(out).ravel() - 1.0
    var = theory.kernel_density_variance(1.0, gp["kT"], gp["c"] * cp_over_cf, 8.0)
    return s, var


@pytest.mark.parametrize("cp_over_cf", [0.5, 1.0, 2.0])
def test_density_pdf_over_particle_sound_speed(cp_over_cf):
    s, var = density_samples(cp_over_cf)
    assert abs(np.mean(s)) < 0.05 * np.sqrt(var)
    assert np.var(s) == pytest.approx(var, rel=0.04)
    z = s / np.sqrt(np.var(s))
    assert abs(np.mean(z ** 3)) < 0.05                        # Gaussian: no skew
    assert np.mean(z ** 4) == pytest.approx(3.0, abs=0.1)     # and kurtosis 3


def test_density_pdf_at_large_particle_sound_speed():
    """The upper end of the paper's range, c_p up to 40 (5 and 10 c_f), dt cut
    so that the CFL number alpha = c_p dt / h is 0.2: J rho stays Gaussian.
    Its variance is within 4 % of rho0 kT / (c_p^2 V) at 5 c_f; at 10 c_f it is
    5 % low at alpha = 0.2 (measured) and converges as alpha falls to 0.1."""
    for cp_over_cf in (5.0, 10.0):
        s, var = density_samples(cp_over_cf, 0.2 / (0.1 * cp_over_cf))
        z = s / np.sqrt(np.var(s))
        assert abs(np.mean(z ** 3)) < 0.05
        assert np.mean(z ** 4) == pytest.approx(3.0, abs=0.1)
        if cp_over_cf == 5.0:
            assert np.var(s) == pytest.approx(var, rel=0.04)
        else:
            e2 = abs(np.var(s) / var - 1.0)
            s1, _ = density_samples(cp_over_cf, 0.1 / (0.1 * cp_over_cf))
            e1 = abs(np.var(s1) / var - 1.0)
            assert e2 < 0.07 and e1 < 0.6 * e2, (e1, e2)


def test_density_variance_converges_with_cfl_number():
    """c_p = 4 c_f: alpha = 0.4 at dt = 0.1 h / c_f, 0.2 at half of it."""
    s1, var = density_samples(4.0, 1.0)
    s2, _ = density_samples(4.0, 0.5)
    e1, e2 = abs(np.var(s1) / var - 1.0), abs(np.var(s2) / var - 1.0)
    assert e2 < 0.04
    assert e1 > 2.0 * e2, (e1, e2)


def test_ensemble_averaged_force_in_a_thermal_bath():
    """Thirty-two fluctuating boxes (Philox box ids 0..31) of the Table I
    dipolar case and one deterministic box, advanced as one batch: thermal
    noise scatters the per-box time-averaged forces, and their ensemble mean
    (Sec. 6) agrees with the deterministic force within its statistical error;
    the deterministic force is Gor'kov's within the dipolar tolerance above."""
    from paper_1307_0702_gb300 import Batch, Grid

    nsteps, skip, k_s, h = 24000, 8000, 1.0, 10.0
    w = W.blackman_harris(nsteps, skip)
    L = 32 * h
    q = np.array([[L / 8, L / 2, L / 2], [7 * L / 8, L / 2, L / 2]])
    grids = []
    for b in range(33):
        gp, _, _ = W.single_particle_config(n=32, k_spring=k_s, mirror=True, mass_ratio=2.0, kappa_ratio=1.0)
        gp.update(h=h, dt=0.1 * h / gp["c"], zeta=1.0, precision="fp32", kT=1e-7 if b else 0.0, seed=77, box=b)
        rho, g = W.velocity_phase_wave_fields(gp)
        grid = Grid(gp)
        grid.set_state(rho, g)
        grid.add_particles(q, (2.0 - 1.0) * 8 * h ** 3, 1.0, k_s)
        grids.append(grid)
    with Batch(grids) as batch:
        batch.step(nsteps, w)
    forces, a2s = [], []
    for grid in grids:
        f, _, a2 = grid.time_average()
        forces.append(-f[0, 0])
        a2s.append(a2)
        grid.close()
    f_det, thermal = forces[0], np.array(forces[1:])
    mean, sem = thermal.mean(), thermal.std(ddof=1) / np.sqrt(len(thermal))
    assert np.std(thermal) > 0 and sem < 0.1 * abs(f_det)      # independent, resolvable fluctuations
    assert abs(mean - f_det) < 4 * sem, (mean, f_det, sem)
    k = 2 * np.pi / L
    omega = theory.discrete_sound_frequency(4.0, h, 32)
    fg = theory.gorkov_force(4.0, np.sqrt(2 * a2s[0]), 8 * h ** 3, k, 1.0, 1.0, 8 * h ** 3 - k_s / omega ** 2, L / 8)
    assert 0.97 <= f_det / fg <= 1.07
