"""Pins of the oracle's adjoint of the deterministic IC step.

Every transpose is checked against a derivative taken independently of it:
complex-step (exact to rounding) for the fluid rates and the velocity map,
central finite differences of the forward oracle for the kernel weights, one
whole step and whole rollouts.  The gradient of the time-averaged tether
force is checked against central differences with step 1e-6 (relative
agreement 1e-5 or better).
"""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import fluid, ic, peskin


def small_params(n=(7, 6, 8), forcing="mode", A=2e-3, zeta=0.3, **kw):
    return ic.GridParams(nx=n[0], ny=n[1], nz=n[2], forcing=forcing, wave_amp=A, zeta=zeta, **kw)


def random_state(p, seed, amp=2e-3):
    rng = np.random.default_rng(seed)
    return amp * rng.uniform(-1, 1, p.shape), [amp * rng.uniform(-1, 1, p.shape) for _ in range(3)]


def test_phi_prime_is_the_derivative_of_phi_and_continuous():
    r = np.linspace(-1.6, 1.6, 3201)
    r = r[np.min(np.abs(np.abs(r)[:, None] - np.array([0.0, 0.5, 1.5])[None]), axis=1) > 1e-4]
    e = 1e-6
    fd = (peskin.phi(r + e) - peskin.phi(r - e)) / (2 * e)
    assert np.max(np.abs(adj.phi_prime(r) - fd)) < 1e-7
    # C^1 at the branch points: -sign(r) at |r| = 1/2, 0 at |r| = 3/2 and beyond
    for x, want in ((0.5, -1.0), (-0.5, 1.0), (1.5, 0.0), (-1.5, 0.0), (2.0, 0.0)):
        for d in (-1e-12, 1e-12):
            assert adj.phi_prime(np.array([x + d]))[0] == pytest.approx(want, abs=1e-5)


def test_weight_derivatives_match_finite_differences():
    rng = np.random.default_rng(1)
    shape, h = (9, 8, 7), 0.9
    q = rng.uniform(0, 1, (5, 3)) * np.array([7, 8, 9]) * h
    for off in (peskin.CENTRE,) + peskin.FACE:
        st = adj.StencilsD(q, h, shape, off)
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = 1e-6
            wp = peskin.Stencils(q + e, h, shape, off)
            wm = peskin.Stencils(q - e, h, shape, off)
            assert np.array_equal(wp.flat, st.flat) and np.array_equal(wm.flat, st.flat)
            fd = (wp.w - wm.w) / 2e-6
            assert np.max(np.abs(st.dw[:, :, ax] - fd)) < 1e-8


def test_interp_transpose_and_spread_are_adjoint():
    """<J f, lam> = <f, J^T lam> and S = J^T / h^3 (Eq. (adj))."""
    rng = np.random.default_rng(2)
    shape, h = (6, 7, 8), 1.3
    q = rng.uniform(0, 1, (4, 3)) * np.array([8, 7, 6]) * h
    st = adj.StencilsD(q, h, shape, peskin.FACE[1])
    f = rng.normal(size=shape)
    lam = rng.normal(size=4)
    assert np.dot(st.interp(f), lam) == pytest.approx(np.sum(f * st.interp_T(lam, shape)), rel=1e-13)
    assert np.allclose(st.spread(lam, shape, h), st.interp_T(lam, shape) / h ** 3, rtol=1e-14, atol=0)


def complex_step(fun, x, dx, e=1e-30):
    return np.imag(fun(x + 1j * e * dx)) / e


def test_rates_transpose_against_complex_step():
    p = small_params(eta=0.7, zeta=0.4)
    fp = p.fluid()
    drho, g = random_state(p, 3, amp=5e-2)
    rng = np.random.default_rng(4)
    pe = 1e-2 * rng.normal(size=p.shape)
    d_rho, d_g, d_pe = rng.normal(size=p.shape), [rng.normal(size=p.shape) for _ in range(3)], rng.normal(size=p.shape)
    lam_rho, lam_g = rng.normal(size=p.shape), [rng.normal(size=p.shape) for _ in range(3)]

    def pack(r, gg, e):
        return np.concatenate([r.ravel()] + [x.ravel() for x in gg] + [e.ravel()])

    n = drho.size

    def rates_flat(x):
        r, gg, e = x[:n].reshape(p.shape), [x[(1 + a) * n:(2 + a) * n].reshape(p.shape) for a in range(3)], \
            x[4 * n:].reshape(p.shape)
        dr, dg = fluid.rates(r, gg, fp, e)
        return np.concatenate([dr.ravel()] + [x.ravel() for x in dg])

    jvp = complex_step(rates_flat, pack(drho, g, pe), pack(d_rho, d_g, d_pe))
    lhs = np.dot(np.concatenate([lam_rho.ravel()] + [x.ravel() for x in lam_g]), jvp)
    rb, gb, pb = adj.rates_vjp(drho, g, fp, lam_rho, lam_g)
    rhs = np.dot(pack(rb, gb, pb), pack(d_rho, d_g, d_pe))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_velocity_map_transpose_against_complex_step():
    p = small_params()
    drho, g = random_state(p, 5, amp=0.1)
    rng = np.random.default_rng(6)
    d_rho, d_g = rng.normal(size=p.shape), [rng.normal(size=p.shape) for _ in range(3)]
    vb = [rng.normal(size=p.shape) for _ in range(3)]
    e = 1e-30
    vc = adj.velocities(p, drho + 1j * e * d_rho, [g[a] + 1j * e * d_g[a] for a in range(3)])
    lhs = sum(np.sum(vb[a] * np.imag(vc[a]) / e) for a in range(3))
    rb, gb = adj.velocities_vjp(p, drho, g, vb)
    rhs = np.sum(rb * d_rho) + sum(np.sum(gb[a] * d_g[a]) for a in range(3))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def make_case(p, npart=3, seed=7, tethered=True):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.1, 0.9, (npart, 3)) * p.lengths
    if npart > 1:
        q[1] = q[0] + np.array([1.2, -0.7, 0.5])       # overlapping kernels
    u = 1e-3 * rng.normal(size=(npart, 3))
    parts = adj.make_parts(q, u, rng.uniform(0.5, 6.0, npart), rng.uniform(0.3, 1.5, npart),
                           rng.uniform(0.2, 0.8, npart) if tethered else 0.0, p.c)
    parts["q_eq"] = parts["q_eq"] + 0.05 * rng.normal(size=(npart, 3))
    return parts


def test_record_step_is_the_oracle_step():
    p = small_params(forcing="plane", plane_index=2)
    drho, g = random_state(p, 8)
    parts = make_case(p)
    sim = ic.Simulation(p, drho=drho, g=g)
    sim.add_particles(parts["q"], parts["m_e"], 1.0, parts["k_s"], u=parts["u"])
    sim.parts.eps[:] = parts["eps"]
    sim.parts.q_eq[:] = parts["q_eq"]
    for n in range(3):
        T, new = adj.record_step(p, parts, drho, g, n)
        sim.step()
        assert np.array_equal(new["drho"], sim.drho)
        assert all(np.array_equal(new["g"][a], sim.g[a]) for a in range(3))
        assert np.array_equal(new["q"], sim.parts.q) and np.array_equal(new["u"], sim.parts.u)
        assert np.array_equal(T["force"], sim.last["force"])
        drho, g = new["drho"], new["g"]
        parts = {**parts, "q": new["q"], "u": new["u"]}


@pytest.mark.parametrize("forcing", ["mode", "plane"])
def test_one_step_transpose_against_central_differences(forcing):
    """<bar_out, d step> = <bar_in, d state> + grad . d params for random directions."""
    p = small_params(forcing=forcing, plane_index=3, A=3e-3)
    drho, g = random_state(p, 9)
    parts = make_case(p, npart=3)
    rng = np.random.default_rng(10)
    npart = 3
    bar = dict(drho=rng.normal(size=p.shape), g=[rng.normal(size=p.shape) for _ in range(3)],
               q=rng.normal(size=(npart, 3)), u=rng.normal(size=(npart, 3)))
    direction = rng.normal(size=(npart, 3))
    weight = 0.7
    dx = dict(drho=rng.normal(size=p.shape) * 1e-3, g=[rng.normal(size=p.shape) * 1e-3 for _ in range(3)],
              q=rng.normal(size=(npart, 3)), u=rng.normal(size=(npart, 3)) * 1e-3)
    dth = dict(m_e=rng.normal(size=npart), eps=rng.normal(size=npart), A=1e-3 * rng.normal())

    def f(t):
        pp = ic.GridParams(**{**p.__dict__, "wave_amp": p.wave_amp + t * dth["A"]})
        pa = {**parts, "q": parts["q"] + t * dx["q"], "u": parts["u"] + t * dx["u"],
              "m_e": parts["m_e"] + t * dth["m_e"], "eps": parts["eps"] + t * dth["eps"]}
        T, new = adj.record_step(pp, pa, drho + t * dx["drho"], [g[a] + t * dx["g"][a] for a in range(3)], 4)
        val = np.sum(new["drho"] * bar["drho"]) + sum(np.sum(new["g"][a] * bar["g"][a]) for a in range(3))
        val += np.sum(new["q"] * bar["q"]) + np.sum(new["u"] * bar["u"])
        return val + weight * np.sum(direction * T["force"])

    e = 1e-6
    fd = (f(e) - f(-e)) / (2 * e)
    T, _ = adj.record_step(p, parts, drho, g, 4)
    out, gr = adj.adjoint_step(p, parts, T, bar, weight, direction)
    an = np.sum(out["drho"] * dx["drho"]) + sum(np.sum(out["g"][a] * dx["g"][a]) for a in range(3))
    an += np.sum(out["q"] * dx["q"]) + np.sum(out["u"] * dx["u"])
    an += np.dot(gr["m_e"], dth["m_e"]) + np.dot(gr["eps"], dth["eps"]) + gr["A"] * dth["A"]
    assert an == pytest.approx(fd, rel=1e-7)


def rollout_case(forcing="mode", n=(8, 6, 7), nsteps=24):
    p = small_params(n=n, forcing=forcing, A=3e-3, plane_index=1)
    drho, g = ic.standing_wave(p)
    drho = drho - p.rho0
    parts = make_case(p, npart=3, seed=11)
    parts["u"] = np.zeros_like(parts["u"])
    weights = np.linspace(0.5, 1.5, nsteps)
    direction = np.zeros((3, 3))
    direction[:, 0] = 1.0                  # the x force summed over particles
    return p, drho, g, parts, weights, direction


def phi_of(p, parts, weights, direction, A=None, m_e=None, kappa=None):
    pp = ic.GridParams(**{**p.__dict__, "wave_amp": p.wave_amp if A is None else A})
    drho, g = ic.standing_wave(pp)
    pa = dict(parts)
    if m_e is not None:
        pa["m_e"] = m_e
    if kappa is not None:
        pa["eps"] = ic.epsilon_from_kappa_ratio(kappa, p.c)
    return adj.rollout(pp, drho - pp.rho0, g, pa, weights, direction)[0]


@pytest.mark.parametrize("forcing", ["mode", "plane"])
def test_rollout_gradient_against_central_differences(forcing):
    """Gradient of the time-averaged x force w.r.t. m_e, kappa_p/kappa_f and A (initial
    standing wave and drive both scale with A), central differences with step 1e-6."""
    p, drho, g, parts, weights, direction = rollout_case(forcing)
    phi, gr = adj.rollout_gradient(p, drho, g, parts, weights, direction, checkpoint_every=5)
    assert phi == pytest.approx(phi_of(p, parts, weights, direction), rel=1e-14)
    k, kd, omega, gamma = ic.wave_numbers(p)
    cosk = np.cos(k * ic.axis_coordinate(p, p.wave_axis))
    dA = gr["A"] + np.sum(gr["state"]["drho"] * cosk)        # initial rho0 + A cos(kx)
    e = 1e-6
    kappa = p.c ** 2 / (parts["eps"] + p.c ** 2)
    fd_A = (phi_of(p, parts, weights, direction, A=p.wave_amp * (1 + e)) -
            phi_of(p, parts, weights, direction, A=p.wave_amp * (1 - e))) / (2 * e * p.wave_amp)
    scale = abs(phi) / p.wave_amp
    assert abs(dA - fd_A) < 1e-6 * scale
    for j in range(3):
        de = np.zeros(3)
        de[j] = e
        fd_m = (phi_of(p, parts, weights, direction, m_e=parts["m_e"] + de) -
                phi_of(p, parts, weights, direction, m_e=parts["m_e"] - de)) / (2 * e)
        fd_k = (phi_of(p, parts, weights, direction, kappa=kappa + de) -
                phi_of(p, parts, weights, direction, kappa=kappa - de)) / (2 * e)
        assert gr["m_e"][j] == pytest.approx(fd_m, rel=1e-5, abs=1e-9 * abs(phi))
        assert gr["kappa_ratio"][j] == pytest.approx(fd_k, rel=1e-5, abs=1e-9 * abs(phi))
    assert np.max(np.abs(gr["m_e"])) > 0 and np.max(np.abs(gr["kappa_ratio"])) > 0


def test_checkpoint_interval_does_not_change_the_gradient():
    p, drho, g, parts, weights, direction = rollout_case(nsteps=12)
    ref = adj.rollout_gradient(p, drho, g, parts, weights, direction)
    for K in (1, 5, 12):
        got = adj.rollout_gradient(p, drho, g, parts, weights, direction, checkpoint_every=K)
        assert got[0] == ref[0]
        for key in ("m_e", "kappa_ratio", "A"):
            assert np.array_equal(got[1][key], ref[1][key])
        assert np.array_equal(got[1]["state"]["drho"], ref[1]["state"]["drho"])


def test_untethered_particles_feel_no_objective_and_fluid_only_gradient_is_drive_only():
    """k_s = 0: F = 0 for every step, so Phi and all gradients vanish."""
    p, drho, g, parts, weights, direction = rollout_case(nsteps=6)
    parts["k_s"] = np.zeros(3)
    phi, gr = adj.rollout_gradient(p, drho, g, parts, weights, direction)
    assert phi == 0.0
    assert np.all(gr["m_e"] == 0) and np.all(gr["kappa_ratio"] == 0) and gr["A"] == 0.0
