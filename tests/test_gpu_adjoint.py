"""GPU adjoint of the deterministic IC step (through the C ABI) against the
oracle's FP64 adjoint and against central finite differences of the GPU's own
forward rollout.

Objective: Phi = sum_p d_p . <F_p>_w, the weighted time average of the tether
forces (Sec. 6).  Gradients with respect to m_e, kappa_p/kappa_f, the drive
amplitude A and the initial state.  FP64 agrees with the oracle to 1e-9
normwise (the adjoint spreads with atomic adds, so its rounding order is not
the oracle's); FP32 to 2e-3; finite differences (step 1e-6) to 1e-5.
"""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import ic as oic
from paper_1307_0702_gb300 import workloads as W
from pairs import oracle_params, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 2e-3}


def case(prec, shape=(12, 10, 9), forcing="mode", nsteps=10, seed=3, amp=2e-3, u_amp=1e-3, wave_amp=3e-3):
    gp = W.grid_params(shape, kT=0.0, wave_amp=wave_amp, forcing=forcing, zeta=0.3, precision=prec, plane_index=2,
                       wave_phase=0.4)
    rng = np.random.default_rng(seed)
    L = np.array(shape, dtype=float)
    q = rng.uniform(0.1, 0.9, (4, 3)) * L
    q[1] = (q[0] + np.array([1.2, -0.7, 0.5])) % L         # overlapping kernels
    q[2, 0] = L[0] - 0.3                                   # near the periodic seam
    parts = dict(q=q, m_e=rng.uniform(0.5, 6.0, 4), kappa_ratio=rng.uniform(0.3, 1.5, 4),
                 k_spring=rng.uniform(0.2, 0.8, 4), u=u_amp * rng.normal(size=(4, 3)))
    rho, g = W.random_fields(gp, seed=seed, amp_rho=amp, amp_g=amp)
    weights = np.linspace(0.5, 1.5, nsteps)
    direction = rng.normal(size=(4, 3))
    return gp, rho, g, parts, weights, direction


def gpu_gradient(gp, rho, g, parts, weights, direction, K, tapes=True):
    from paper_1307_0702_gb300 import Grid
    from paper_1307_0702_gb300.adjoint import Rollout

    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"], parts["u"])
        roll = Rollout(grid, parts["kappa_ratio"], checkpoint_every=K, tapes=tapes)
        phi = roll.forward(weights, direction)
        return phi, roll.backward()


def oracle_gradient(gp, rho, g, parts, weights, direction, K=None):
    p = oracle_params(gp)
    op = oadj.make_parts(parts["q"], parts["u"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"], p.c)
    drho = np.asarray(rho, dtype=np.float64) - p.rho0
    return oadj.rollout_gradient(p, drho, g, op, weights, direction, checkpoint_every=K)


def compare(gr, orc):
    errs = {k: rel_err(gr[k], orc[k]) for k in ("m_e", "kappa_ratio", "eps")}
    errs["A"] = abs(gr["A"] - orc["A"]) / abs(orc["A"])
    st = orc["state"]
    errs["rho"] = rel_err(gr["rho"], st["drho"])
    for a in range(3):
        errs[f"g{a}"] = rel_err(gr["g"][a], st["g"][a])
    errs["q"] = rel_err(gr["q"], st["q"])
    errs["u"] = rel_err(gr["u"], st["u"])
    return errs


@pytest.mark.parametrize("prec,forcing", [("fp64", "mode"), ("fp64", "plane"), ("fp32", "mode")])
def test_rollout_gradient_matches_the_oracle_adjoint(prec, forcing):
    gp, rho, g, parts, weights, direction = case(prec, forcing=forcing)
    phi, gr = gpu_gradient(gp, rho, g, parts, weights, direction, K=4)
    ophi, orc = oracle_gradient(gp, rho, g, parts, weights, direction)
    assert abs(phi - ophi) <= (1e-11 if prec == "fp64" else 1e-4) * abs(ophi)
    errs = compare(gr, orc)
    bad = {k: v for k, v in errs.items() if not v <= TOL[prec]}
    assert not bad, errs


def test_checkpoint_interval_changes_the_gradient_only_by_rounding():
    gp, rho, g, parts, weights, direction = case("fp64", nsteps=9)
    ref = gpu_gradient(gp, rho, g, parts, weights, direction, K=9)[1]
    for K in (1, 4):
        got = gpu_gradient(gp, rho, g, parts, weights, direction, K=K)[1]
        for k in ("m_e", "kappa_ratio"):
            assert rel_err(got[k], ref[k]) < 1e-12
        assert abs(got["A"] - ref["A"]) < 1e-12 * abs(ref["A"])
        assert rel_err(got["rho"], ref["rho"]) < 1e-12


def gpu_phi(gp, rho, g, parts, weights, direction):
    from paper_1307_0702_gb300 import Grid

    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"], parts["u"])
        grid.step(len(weights), weights)
        f_avg = grid.time_average()[0]
    return float(np.sum(direction * f_avg))


def test_gpu_gradient_against_central_differences_of_the_gpu_forward():
    """Central differences of the GPU forward, step 1e-6: the gradient of each
    parameter family (m_e and kappa_p/kappa_f of all particles) within 1e-5
    of them normwise.  The rounding of Phi (~1e-13 relative after 64 FP64
    steps) divided by the step leaves ~2e-9 of noise in each difference, so
    a small component of a family is only resolved relative to the family's
    largest; step 1e-4 (truncation ~1e-8) checks every component to 1e-6."""
    gp, rho, g, parts, weights, direction = case("fp64", nsteps=64, amp=3e-2, u_amp=2e-2, wave_amp=5e-2)
    phi, gr = gpu_gradient(gp, rho, g, parts, weights, direction, K=5)

    def fd(key, j, e):
        pp = {k: np.array(v, copy=True) for k, v in parts.items()}
        pm = {k: np.array(v, copy=True) for k, v in parts.items()}
        pp[key][j] += e
        pm[key][j] -= e
        return (gpu_phi(gp, rho, g, pp, weights, direction) - gpu_phi(gp, rho, g, pm, weights, direction)) / (2 * e)

    for key in ("m_e", "kappa_ratio"):
        d6 = np.array([fd(key, j, 1e-6) for j in range(4)])
        assert np.max(np.abs(gr[key] - d6)) <= 1e-5 * np.max(np.abs(d6)), (key, gr[key], d6)
        d4 = np.array([fd(key, j, 1e-4) for j in range(4)])
        assert np.allclose(gr[key], d4, rtol=1e-6, atol=0), (key, gr[key], d4)
    # the drive amplitude (initial state held fixed)
    e = 1e-6
    fa = (gpu_phi({**gp, "wave_amp": gp["wave_amp"] * (1 + e)}, rho, g, parts, weights, direction) -
          gpu_phi({**gp, "wave_amp": gp["wave_amp"] * (1 - e)}, rho, g, parts, weights, direction)) / (
              2 * e * gp["wave_amp"])
    assert gr["A"] == pytest.approx(fa, rel=1e-5)


def test_autograd_function_with_the_standing_wave_start():
    """torch.autograd through time_averaged_force: the initial density
    rho0 + A cos(k x) is built in torch, so dPhi/dA collects the drive and the
    initial state; checked against central differences of the GPU forward."""
    import torch

    from paper_1307_0702_gb300.adjoint import time_averaged_force

    gp = W.grid_params((16, 8, 8), kT=0.0, wave_amp=5e-2, forcing="mode", precision="fp64")
    n = 3
    q = np.array([[2.0, 4.0, 4.0], [6.5, 4.2, 3.9], [12.0, 3.5, 4.5]])
    weights = np.ones(64)
    k = 2 * np.pi / 16.0
    cosk = torch.as_tensor(np.cos(k * np.arange(16.0)), dtype=torch.float64).reshape(1, 1, 16)

    def phi(m_e, kappa, A):
        rho = 1.0 + A * cosk.expand(8, 8, 16)
        return time_averaged_force(gp, q, m_e, kappa, np.full(n, 1.0), A, rho, weights=weights, checkpoint_every=7)

    m_e = torch.tensor([4.0, 1.0, 2.5], dtype=torch.float64, requires_grad=True)
    kappa = torch.tensor([0.5, 0.8, 1.3], dtype=torch.float64, requires_grad=True)
    A = torch.tensor(5e-2, dtype=torch.float64, requires_grad=True)
    out = phi(m_e, kappa, A)
    dm, dk, dA = torch.autograd.grad(out, (m_e, kappa, A))
    e = 1e-6
    with torch.no_grad():
        fd_A = (phi(m_e, kappa, A * (1 + e)) - phi(m_e, kappa, A * (1 - e))) / (2 * e * A)
        d = torch.tensor([e, 0.0, 0.0], dtype=torch.float64)
        fd_m = (phi(m_e + d, kappa, A) - phi(m_e - d, kappa, A)) / (2 * e)
        fd_k = (phi(m_e, kappa + d, A) - phi(m_e, kappa - d, A)) / (2 * e)
    assert float(dA) == pytest.approx(float(fd_A), rel=1e-5)
    assert float(dm[0]) == pytest.approx(float(fd_m), rel=1e-5)
    assert float(dk[0]) == pytest.approx(float(fd_k), rel=1e-5)


def test_adjoint_calls_are_refused_in_the_wrong_state():
    from paper_1307_0702_gb300 import Grid, ICError

    gp = W.grid_params(8, kT=1e-3, precision="fp64")
    with Grid(gp) as grid:
        with pytest.raises(ICError):
            grid.adjoint_enable()            # thermal box
    gp = W.grid_params(8, kT=0.0, precision="fp64")
    with Grid(gp) as grid:
        grid.add_particles([[2.0, 3.0, 4.0]], 1.0, 0.5, 0.3)
        with pytest.raises(ICError):
            grid.step_record()               # not enabled
        grid.adjoint_enable()
        with pytest.raises(ICError):
            grid.adjoint_step(1.0)           # nothing recorded
        grid.step_record()
        grid.step(1)
        with pytest.raises(ICError):
            grid.adjoint_step(1.0)           # the state moved on
        grid.add_particles([[5.0, 5.0, 5.0]], 1.0, 0.5, 0.3)
        with pytest.raises(ICError):
            grid.step_record()               # particles added after enabling
        snap = grid.new_snapshot()
        grid.snapshot_save(snap)
        with Grid(W.grid_params(9, kT=0.0, precision="fp64")) as other:
            with pytest.raises(ICError):
                other.snapshot_load(snap)    # another grid


def test_snapshot_round_trip_reproduces_the_steps():
    from paper_1307_0702_gb300 import Grid

    gp, rho, g, parts, weights, direction = case("fp32", nsteps=4)
    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"], parts["u"])
        grid.step(3)
        snap = grid.new_snapshot()
        grid.snapshot_save(snap)
        grid.step(5)
        a = grid.get_state(), grid.forces()
        grid.snapshot_load(snap)
        assert grid.stats()[2] == 3
        grid.step(5)
        b = grid.get_state(), grid.forces()
    assert np.array_equal(a[0][0], b[0][0]) and all(np.array_equal(a[0][1][i], b[0][1][i]) for i in range(3))
    assert all(np.array_equal(x, y) for x, y in zip(a[1], b[1]))


# ---------------------------------------------------------------- the 64^3 rollout
def line_case(prec, A=1e-3, nsteps=1000, offset=0.0):
    """64^3, 16 tethered particles on a line along x (workloads.line_config),
    1000 steps of unit weight."""
    gp, rho, g, parts = W.line_config(64, 16, wave_amp=A, precision=prec, offset=offset)
    return gp, rho, g, parts, np.ones(nsteps)


def test_line_of_particles_amplitude_homogeneity():
    """With 16 particles spaced evenly over one wavelength, the objective
    Phi = sum_p sin(2 k x_p) <F_x,p> is even in A: A -> -A is the shift by
    half a wavelength, which maps the line onto itself and leaves every
    sin(2 k x_p) unchanged.  So Phi = a_2 A^2 + a_4 A^4 + ..., the radiation
    force being quadratic in the amplitude at leading order
    (Eq. (eq:acousticForce2)), and the adjoint's A dPhi/dA / Phi = 2 + 2 (a_4/a_2) A^2 + ...:
    within 1e-4 of 2 at A = 1e-3, and its excess over 2 grows as A^2 (the
    exponent between A = 2.5e-4 and 1e-3 within 0.1 of 2; the next term
    moves it by a few hundredths).  The line sits a quarter cell off the
    grid points: a particle oscillating about a point where the 3-point
    function's second derivative jumps (|r| = 1/2, App. A.1) adds a term in
    |A|^3 to Phi, which is even but not analytic in A."""
    import torch

    from paper_1307_0702_gb300.adjoint import time_averaged_force

    def log_slope(amp):
        gp, rho, g, parts, weights = line_case("fp64", A=amp, offset=0.25)
        k = 2 * np.pi / 64.0
        direction = np.zeros((16, 3))
        direction[:, 0] = np.sin(2 * k * parts["q"][:, 0])
        cosk = torch.as_tensor(np.cos(k * np.arange(64.0)), dtype=torch.float64).reshape(1, 1, 64)
        A = torch.tensor(amp, dtype=torch.float64, requires_grad=True)
        rho_t = 1.0 + A * cosk.expand(64, 64, 64)
        phi = time_averaged_force(gp, parts["q"], torch.tensor(parts["m_e"]), torch.tensor(parts["kappa_ratio"]),
                                  parts["k_spring"], A, rho_t, weights=weights, direction=direction,
                                  checkpoint_every=50)
        (dA,) = torch.autograd.grad(phi, (A,))
        phi = float(phi.detach())
        assert abs(phi) > 0
        return amp * float(dA) / phi

    small, large = log_slope(2.5e-4), log_slope(1e-3)
    assert large == pytest.approx(2.0, abs=1e-4), (small, large)
    exponent = np.log((large - 2.0) / (small - 2.0)) / np.log(4.0)
    assert exponent == pytest.approx(2.0, abs=0.1), (small, large)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_line_of_particles_gradient(prec):
    """The 64^3 rollout of 1000 steps with a checkpoint every 50 steps:
    gradients of sum_p <F_x,p> with respect to each particle's m_e and
    kappa_p/kappa_f.  FP64 against central differences of the GPU forward
    within 1e-5 normwise (A = 1e-2 and step 1e-3: the rounding of Phi over
    1000 steps puts ~3e-9 of noise into a difference of step 1e-5, while
    step 1e-3 is limited by truncation at ~1e-7); FP32 within 1e-3 of FP64.
    The line and the wave are symmetric under x -> -x, which makes the summed
    x force vanish for every A, so its A-gradient is zero."""
    gp, rho, g, parts, weights = line_case(prec, A=1e-2)
    direction = np.tile([1.0, 0.0, 0.0], (16, 1))
    phi, gr = gpu_gradient(gp, rho, g, parts, weights, direction, K=50)
    if prec == "fp64":
        e = 1e-3
        for key in ("m_e", "kappa_ratio"):
            fd = []
            for j in (0, 5):
                pp = {kk: np.array(v, copy=True) for kk, v in parts.items()}
                pm = {kk: np.array(v, copy=True) for kk, v in parts.items()}
                pp[key][j] += e
                pm[key][j] -= e
                fd.append((gpu_phi(gp, rho, g, pp, weights, direction) -
                           gpu_phi(gp, rho, g, pm, weights, direction)) / (2 * e))
            got = gr[key][[0, 5]]
            assert np.max(np.abs(got - fd)) <= 1e-5 * np.max(np.abs(fd)), (key, got, fd)
        assert abs(gr["A"]) < 1e-12
    else:
        _, ref = gpu_gradient({**gp, "precision": "fp64"}, rho, g, parts, weights, direction, K=50)
        for key in ("m_e", "kappa_ratio"):
            assert rel_err(gr[key], ref[key]) < 1e-3, (key, rel_err(gr[key], ref[key]))


def test_dipolar_force_gradient_follows_f2():
    """The closed form of the dipolar force, Eq. (eq:acousticForce2) with f_2
    of Eq. (f2): at c_p = c_f (f_1 = 0) the radiation force is proportional
    to f_2(m), m = m_e - k_s / omega^2 (the tether's excess mass at the drive
    frequency), so d ln F / d m_e = f_2'(m) / f_2(m) = 3 rho0 V / (m (2 m +
    3 rho0 V)), whatever the amplitude prefactor.  The adjoint of the 64 000
    step Table I run of Fig. 4 (rho_p = 2 rho0, mirrored tethered pair, mode
    drive, Blackman-Harris window after 16 000 steps; FP32) gives it within
    3 % (measured 0.8 %), and central differences of its own forward (both
    masses moved by 1 %) within 1 %: the FP32 forward's rounding leaves ~0.5 %
    of noise in such a difference.  (In FP64 the same adjoint matches central
    differences to 1e-6, and the FP32 adjoint is within 6e-4 of it.)"""
    from paper_1307_0702_gb300 import Grid
    from oracle import theory

    h, n = 10.0, 32
    gp, parts, _ = W.single_particle_config(n=n, k_spring=1.0, mirror=True, mass_ratio=2.0, kappa_ratio=1.0)
    gp.update(h=h, dt=0.1 * h / gp["c"], zeta=1.0, precision="fp32", wave_amp=1e-3)
    L = n * h
    parts["q"] = np.array([[L / 8, L / 2, L / 2], [7 * L / 8, L / 2, L / 2]])
    vol = 8 * h ** 3
    parts["m_e"] = np.full(2, 1.0 * vol)
    parts["u"] = None
    rho, g = W.velocity_phase_wave_fields(gp)
    weights = W.blackman_harris(64000, 16000)
    # Phi = F_0 - F_1 = 2 F_0: the radiation force is minus the averaged spring force
    direction = np.array([[-1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    phi, gr = gpu_gradient(gp, rho, g, parts, weights, direction, K=100)
    dphi = float(gr["m_e"][0] + gr["m_e"][1])          # both masses together
    omega = theory.discrete_sound_frequency(gp["c"], h, n)
    m = parts["m_e"][0] - 1.0 / omega ** 2
    closed = 3.0 * gp["rho0"] * vol / (m * (2.0 * m + 3.0 * gp["rho0"] * vol))

    def phi_of(scale):
        with Grid(gp) as grid:
            grid.set_state(rho, g)
            grid.add_particles(parts["q"], parts["m_e"] * scale, parts["kappa_ratio"], parts["k_spring"])
            grid.step(len(weights), weights)
            f = grid.time_average()[0]
        return float(np.sum(direction * f))

    d = 0.01
    fd = (phi_of(1 + d) - phi_of(1 - d)) / (2 * d * parts["m_e"][0])
    info = dict(phi=phi, adjoint=dphi, fd=fd, log_slope=dphi / phi, closed=closed)
    assert phi > 0, info                                    # pushed towards the pressure node
    assert dphi == pytest.approx(fd, rel=1e-2), info
    assert dphi / phi == pytest.approx(closed, rel=0.03), info


@pytest.mark.parametrize("case_id", range(8))
def test_adjoint_random_configurations(case_id):
    """Seeded random cases against the oracle's adjoint: edges 6-20, both
    precisions, every drive (or none) along any axis, 1-6 particles anywhere
    (overlapping, on the seam), tethered or free, random objective directions
    and checkpoint intervals."""
    rng = np.random.default_rng(500 + case_id)
    shape = tuple(int(x) for x in rng.integers(6, 21, 3))
    prec = ["fp64", "fp32"][case_id % 2]
    forcing = ["none", "mode", "plane"][int(rng.integers(3))]
    axis = int(rng.integers(3))
    gp = W.grid_params(shape, kT=0.0, wave_amp=float(rng.uniform(1e-3, 5e-3)), forcing=forcing, wave_axis=axis,
                       plane_index=int(rng.integers(shape[axis])), zeta=float(rng.uniform(0.0, 1.0)),
                       precision=prec, wave_phase=float(rng.uniform(0, 6.3)))
    npart = int(rng.integers(1, 7))
    L = np.array(shape, dtype=float)
    q = rng.uniform(0.0, 1.0, (npart, 3)) * L
    if npart > 1:
        q[1] = (q[0] + rng.uniform(-1.0, 1.0, 3)) % L
    if npart > 2:
        q[2, 1] = L[1] - 0.05
    parts = dict(q=q, m_e=rng.uniform(-2.0, 8.0, npart), kappa_ratio=rng.uniform(0.3, 2.0, npart),
                 k_spring=np.where(rng.uniform(size=npart) < 0.7, rng.uniform(0.1, 1.0, npart), 0.0),
                 u=2e-3 * rng.normal(size=(npart, 3)))
    parts["k_spring"][0] = 0.5                               # at least one tether: a non-zero objective
    rho, g = W.random_fields(gp, seed=case_id, amp_rho=3e-3, amp_g=3e-3)
    nsteps = int(rng.integers(3, 9))
    weights = rng.uniform(0.2, 1.0, nsteps)
    direction = rng.normal(size=(npart, 3))
    K = int(rng.integers(1, nsteps + 1))
    phi, gr = gpu_gradient(gp, rho, g, parts, weights, direction, K=K)
    ophi, orc = oracle_gradient(gp, rho, g, parts, weights, direction)
    assert abs(phi - ophi) <= (1e-11 if prec == "fp64" else 1e-4) * abs(ophi)
    errs = compare(gr, orc) if forcing != "none" else {k: v for k, v in compare(gr, {**orc, "A": 1.0}).items()
                                                        if k != "A"}
    bad = {k: v for k, v in errs.items() if not v <= TOL[prec]}
    assert not bad, (shape, prec, forcing, npart, nsteps, K, errs)
    if forcing == "none":
        assert gr["A"] == 0.0


def test_rollout_without_particles():
    """No particles: the objective and every gradient vanish, and the calls
    run (nothing to spread or gather)."""
    from paper_1307_0702_gb300 import Grid
    from paper_1307_0702_gb300.adjoint import Rollout

    gp = W.grid_params((10, 8, 9), kT=0.0, wave_amp=2e-3, forcing="mode", precision="fp64")
    rho, g = W.random_fields(gp, seed=1)
    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.adjoint_enable()
        grid.adjoint_reset()
        snap = grid.new_snapshot()
        grid.snapshot_save(snap)
        grid.step(2)
        grid.snapshot_load(snap)
        grid.step_record()
        grid.adjoint_step(1.0)
        out = grid.adjoint_read()
    assert out["A"] == 0.0
    assert not np.any(out["rho"]) and not any(np.any(x) for x in out["g"])
    assert out["m_e"].shape == (0,)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_tapes_and_recomputed_steps_give_the_same_gradient(prec):
    """Reversing recorded tapes (two forward passes per step) and recording
    each step again before reversing it (three) differentiate the same
    steps: the gradients agree to the rounding of the atomic spreads."""
    gp, rho, g, parts, weights, direction = case(prec, nsteps=11)
    phi_t, gt = gpu_gradient(gp, rho, g, parts, weights, direction, K=4, tapes=True)
    phi_r, gr = gpu_gradient(gp, rho, g, parts, weights, direction, K=4, tapes=False)
    assert phi_t == phi_r
    tol = 1e-12 if prec == "fp64" else 1e-5
    for key in ("m_e", "kappa_ratio", "rho", "q", "u"):
        assert rel_err(gt[key], gr[key]) < tol, key
    assert abs(gt["A"] - gr["A"]) <= tol * abs(gr["A"])


@pytest.mark.parametrize("tapes", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_reverse_step_graphs_equal_direct_launches(prec, tapes, monkeypatch):
    """The reverse step launched as one CUDA graph per tape -- its per-step
    drive derivative and weight rewritten before each launch -- against the
    same kernels launched one by one: the same gradient to the rounding of
    the atomic spreads.  Eleven steps with checkpoints every 4 reuse every
    graph with other steps and weights."""
    gp, rho, g, parts, weights, direction = case(prec, nsteps=11)
    phi_g, gg = gpu_gradient(gp, rho, g, parts, weights, direction, K=4, tapes=tapes)
    monkeypatch.setenv("IC_NO_GRAPH", "1")
    phi_d, gd = gpu_gradient(gp, rho, g, parts, weights, direction, K=4, tapes=tapes)
    assert phi_g == phi_d
    tol = 1e-12 if prec == "fp64" else 1e-5
    for key in ("m_e", "kappa_ratio", "rho", "q", "u"):
        assert rel_err(gg[key], gd[key]) < tol, key
    for a in range(3):
        assert rel_err(gg["g"][a], gd["g"][a]) < tol, a
    assert abs(gg["A"] - gd["A"]) <= tol * abs(gd["A"])


def test_tape_of_another_grid_is_refused():
    from paper_1307_0702_gb300 import Grid, ICError

    gp = W.grid_params(8, kT=0.0, precision="fp64")
    with Grid(gp) as a, Grid(W.grid_params(9, kT=0.0, precision="fp64")) as b:
        for grid in (a, b):
            grid.add_particles([[2.0, 3.0, 4.0]], 1.0, 0.5, 0.3)
            grid.adjoint_enable()
        tape = a.new_tape()
        a.step_record_tape(tape)
        a.adjoint_step_tape(tape, 1.0)
        with pytest.raises(ICError):
            b.adjoint_step_tape(tape, 1.0)
