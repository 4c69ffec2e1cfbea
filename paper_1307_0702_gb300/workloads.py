"""Seeded synthetic workloads (inputs only; no arithmetic of the method).

Each recipe returns plain host data: a dict of grid parameters, the initial
density and momentum fields, and the particle arrays.  The same arrays feed
the CUDA library and the CPU oracle in the tests and the benchmark.  The
paper uses no dataset: these stand in for its Table I runs and for the
standing-wave, thermal and many-particle workloads of the benchmark.

Units: h = 1, rho0 = 1, c = 4, eta = 0.5, dt = 0.1 h / c unless stated.
Volume of one particle kernel V = 8 h^3 (excess mass m_e is given in units of
rho0 V through ``mass_ratio`` = m_p / (rho0 V) = 1 + m_e / (rho0 V)).
"""
import numpy as np

KERNEL_VOLUME_CELLS = 8.0   # V / h^3 of the 3-point kernel


def grid_params(n, *, h=1.0, rho0=1.0, c=4.0, eta=0.5, zeta=0.0, kT=0.0, dt=None,
                seed=0, forcing="mode", wave_axis=0, wave_amp=1e-3, wave_nlambda=1,
                precision="fp64", plane_index=0, wave_phase=0.0):
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), h=float(h), rho0=float(rho0), c=float(c),
                eta=float(eta), zeta=float(zeta), kT=float(kT),
                dt=float(0.1 * h / c if dt is None else dt), seed=int(seed),
                forcing=forcing, wave_axis=int(wave_axis), wave_amp=float(wave_amp),
                wave_nlambda=int(wave_nlambda), precision=precision, plane_index=int(plane_index),
                wave_phase=float(wave_phase))


def standing_wave_fields(gp):
    """rho = rho0 + A cos(k x) along the wave axis, g = 0 (fields shaped [z, y, x])."""
    shape = (gp["nz"], gp["ny"], gp["nx"])
    n_ax = (gp["nx"], gp["ny"], gp["nz"])[gp["wave_axis"]]
    x = np.arange(n_ax) * gp["h"]
    k = 2.0 * np.pi * gp["wave_nlambda"] / (n_ax * gp["h"])
    prof = gp["wave_amp"] * np.cos(k * (x - gp["plane_index"] * gp["h"]))
    bshape = [1, 1, 1]
    bshape[2 - gp["wave_axis"]] = n_ax
    rho = gp["rho0"] + np.broadcast_to(prof.reshape(bshape), shape)
    return np.ascontiguousarray(rho), [np.zeros(shape) for _ in range(3)]


def velocity_phase_wave_fields(gp):
    """The same standing wave a quarter period later: rho = rho0 and
    g = c A sin(k x) on the faces normal to the wave axis (drive phase pi/2).
    A particle started at rest in this state oscillates about its start."""
    shape = (gp["nz"], gp["ny"], gp["nx"])
    ax = gp["wave_axis"]
    n_ax = (gp["nx"], gp["ny"], gp["nz"])[ax]
    k = 2.0 * np.pi * gp["wave_nlambda"] / (n_ax * gp["h"])
    xf = (np.arange(n_ax) + 0.5 - gp["plane_index"]) * gp["h"]
    prof = gp["c"] * gp["wave_amp"] * np.sin(k * xf)
    bshape = [1, 1, 1]
    bshape[2 - ax] = n_ax
    g = [np.zeros(shape) for _ in range(3)]
    g[ax] = np.ascontiguousarray(np.broadcast_to(prof.reshape(bshape), shape))
    return np.full(shape, gp["rho0"]), g


def random_fields(gp, seed, amp_rho=1e-3, amp_g=1e-3):
    """Smooth-free random fields for parity tests: rho0 + amp * U(-1,1), g = amp * U(-1,1)."""
    rng = np.random.default_rng(seed)
    shape = (gp["nz"], gp["ny"], gp["nx"])
    rho = gp["rho0"] + amp_rho * rng.uniform(-1, 1, shape)
    g = [amp_g * rng.uniform(-1, 1, shape) for _ in range(3)]
    return rho, g


def place_uniform(n_particles, lengths, seed, min_sep=0.0):
    """Uniform positions in the periodic box, rejection-sampled for a minimum
    separation (periodic Euclidean distance)."""
    rng = np.random.default_rng(seed)
    L = np.asarray(lengths, dtype=np.float64)
    if min_sep <= 0.0:
        return rng.uniform(0.0, 1.0, (n_particles, 3)) * L
    out = np.empty((n_particles, 3))
    count = 0
    # uniform cell list with cells of side >= min_sep for the rejection test
    ncell = np.maximum(1, np.floor(L / min_sep).astype(int))
    csize = L / ncell
    buckets = {}
    tries = 0
    while count < n_particles:
        tries += 1
        if tries > 200 * n_particles + 10000:
            raise RuntimeError("could not place particles with the requested separation")
        x = rng.uniform(0.0, 1.0, 3) * L
        c = np.floor(x / csize).astype(int) % ncell
        ok = True
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    key = tuple((c + np.array([dx, dy, dz])) % ncell)
                    for j in buckets.get(key, ()):
                        d = out[j] - x
                        d -= L * np.round(d / L)
                        if d @ d < min_sep * min_sep:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[count] = x
            buckets.setdefault(tuple(c), []).append(count)
            count += 1
    return out


def single_particle_config(n=32, steps=2000, k_spring=1.0, mirror=False, mass_ratio=1.5,
                           kappa_ratio=0.5):
    """Deterministic standing wave with a tethered particle (kT = 0, FP64).

    32^3 grid, wave along x with density amplitude 1e-3 rho0 and wavelength L;
    one particle at (L/8, L/2, L/2) (sin 2kx = 1) with m_p = 1.5 rho0 V and
    kappa_p = 0.5 kappa_f, tethered by a spring; seed 0.  ``mirror`` adds its
    mirror image at (7L/8, L/2, L/2), whose spring force is opposite, so the
    springs inject no net momentum (the paper's two-particle layout, Sec. 6).
    The drive phase is pi/2 so that ``velocity_phase_wave_fields`` is the
    matching initial state.
    """
    gp = grid_params(n, wave_amp=1e-3, seed=0, wave_phase=0.5 * np.pi)
    L = n * gp["h"]
    q = [[L / 8.0, L / 2.0, L / 2.0]] + ([[7.0 * L / 8.0, L / 2.0, L / 2.0]] if mirror else [])
    npart = len(q)
    vol = KERNEL_VOLUME_CELLS * gp["h"] ** 3
    parts = dict(q=np.array(q), m_e=np.full(npart, (mass_ratio - 1.0) * gp["rho0"] * vol),
                 kappa_ratio=np.full(npart, kappa_ratio), k_spring=np.full(npart, k_spring))
    return gp, parts, steps


def paper_protocol_config(mass_ratio, kappa_ratio, k_spring, zeta, n=32, h=10.0, precision="fp32"):
    """The force protocol of Sec. 6 in the Table I regime.

    32^3 cells of h = 10, c_f = 4, eta = 0.5, dt = 0.1 h / c_f; the paper's
    drive (Eq. (pext)): a pressure on the grid plane z = 0 (``forcing='plane'``)
    holding the standing wave along z at density amplitude 1e-3 rho0 (phase
    pi/2, so that ``velocity_phase_wave_fields`` is the matching start); two
    tethered particles at (L/2, L/2, 3L/8) and (0, 0, -3L/8), whose radiation
    forces are equal and opposite.
    """
    gp = grid_params(n, h=h, zeta=zeta, wave_amp=1e-3, forcing="plane", wave_axis=2, plane_index=0,
                     seed=0, precision=precision, wave_phase=0.5 * np.pi)
    L = n * h
    q = np.array([[L / 2.0, L / 2.0, 3.0 * L / 8.0], [0.0, 0.0, 5.0 * L / 8.0]])
    vol = KERNEL_VOLUME_CELLS * h ** 3
    parts = dict(q=q, m_e=np.full(2, (mass_ratio - 1.0) * gp["rho0"] * vol),
                 kappa_ratio=np.full(2, float(kappa_ratio)), k_spring=np.full(2, float(k_spring)))
    return gp, parts


def many_particle_config(n, n_particles, *, kT=1e-3, wave_amp=5e-3, wave_nlambda=1, seed=1,
                         min_sep=0.0, mass_range=(0.5, 2.0), kappa_range=(0.0, 2.0),
                         kappa_min=0.04, fixed_contrast=None, k_spring=0.0, precision="fp64",
                         place_seed=None):
    """Fluctuating box with many particles.

    Particle mass ratio m_p/(rho0 V) ~ U(mass_range) and kappa_p/kappa_f ~
    U(kappa_range) clamped below at ``kappa_min`` (a vanishing kappa_p makes
    the particle sound speed, hence the CFL number, unbounded); or, with
    ``fixed_contrast=(mass_ratio, kappa_ratio)``, the same contrast for all.
    """
    gp = grid_params(n, kT=kT, wave_amp=wave_amp, wave_nlambda=wave_nlambda, seed=seed,
                     precision=precision)
    L = np.array([gp["nx"], gp["ny"], gp["nz"]], dtype=np.float64) * gp["h"]
    rng = np.random.default_rng(seed + 1000)
    q = place_uniform(n_particles, L, seed if place_seed is None else place_seed, min_sep)
    vol = KERNEL_VOLUME_CELLS * gp["h"] ** 3
    if fixed_contrast is None:
        mass_ratio = rng.uniform(*mass_range, n_particles)
        kappa = np.maximum(rng.uniform(*kappa_range, n_particles), kappa_min)
    else:
        mass_ratio = np.full(n_particles, fixed_contrast[0])
        kappa = np.full(n_particles, fixed_contrast[1])
    parts = dict(q=q, m_e=(mass_ratio - 1.0) * gp["rho0"] * vol, kappa_ratio=kappa,
                 k_spring=np.full(n_particles, float(k_spring)))
    return gp, parts


def large_box_config(n=128, n_particles=10000):
    """128^3 FP32 box, 1e4 free particles (min separation 2h, host RNG seed 3),
    contrasts of the single-particle case (m_p = 1.5 rho0 V, kappa_p = 0.5
    kappa_f), kT = 1e-3, two wavelengths along x, A = 1e-3."""
    return many_particle_config(n, n_particles, kT=1e-3, wave_amp=1e-3, wave_nlambda=2, seed=3,
                                min_sep=2.0, fixed_contrast=(1.5, 0.5), k_spring=0.0,
                                precision="fp32", place_seed=3)


def line_config(n=64, n_particles=16, wave_amp=1e-3, precision="fp64", offset=0.0, k_spring=1.0):
    """Deterministic box for the differentiable rollout: n^3, n_particles
    tethered particles evenly spaced on a line along x at y = z = n/2 (every
    n / n_particles cells from x = 2, all coordinates shifted by ``offset``),
    m_e = 4 (m_p = 1.5 rho0 V) and kappa_p/kappa_f = 0.5, at rest in the
    standing-wave eigenmode rho0 + A cos(k x) with the mode drive, kT = 0.
    Returns (grid params, rho, g, particles)."""
    gp = grid_params(n, kT=0.0, wave_amp=wave_amp, forcing="mode", precision=precision)
    rho, g = standing_wave_fields(gp)
    sp = n / n_particles
    q = np.stack([2.0 + sp * np.arange(n_particles), np.full(n_particles, n / 2.0),
                  np.full(n_particles, n / 2.0)], axis=1) + offset
    parts = dict(q=q, m_e=np.full(n_particles, 4.0), kappa_ratio=np.full(n_particles, 0.5),
                 k_spring=np.full(n_particles, float(k_spring)), u=np.zeros((n_particles, 3)))
    return gp, rho, g, parts


def ensemble_config(n_boxes=256, sizes=(16, 24, 32, 48), max_particles=200, seed=0):
    """Heterogeneous ensemble: box edges uniform over ``sizes``, 1..max_particles
    particles per box (uniform count, min separation 2h), contrasts of the
    single-particle case (m_p = 1.5 rho0 V, kappa_p = 0.5 kappa_f), kT = 1e-3,
    FP32, Philox seed = box index.  Returns [(grid params, particles)]."""
    rng = np.random.default_rng(seed)
    edges = rng.choice(np.asarray(sizes), n_boxes)
    counts = rng.integers(1, max_particles + 1, n_boxes)
    out = []
    for b in range(n_boxes):
        gp, parts = many_particle_config(int(edges[b]), int(counts[b]), kT=1e-3, wave_amp=1e-3, seed=b,
                                         min_sep=2.0, fixed_contrast=(1.5, 0.5), precision="fp32",
                                         place_seed=10000 + b)
        out.append((gp, parts))
    return out


def blackman_harris(nsteps, skip=0):
    """Averaging weights: zero for the first ``skip`` steps, then a 4-term
    Blackman-Harris window normalised to sum 1."""
    w = np.zeros(nsteps)
    m = nsteps - skip
    if m <= 0:
        return w
    t = np.arange(m) / max(m - 1, 1)
    a = (0.35875, 0.48829, 0.14128, 0.01168)
    win = a[0] - a[1] * np.cos(2 * np.pi * t) + a[2] * np.cos(4 * np.pi * t) - a[3] * np.cos(6 * np.pi * t)
    w[skip:] = win / win.sum()
    return w
