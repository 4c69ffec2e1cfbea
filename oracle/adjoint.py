"""Reverse-mode derivative (adjoint) of the deterministic IC step (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

What is differentiated.  The observable of Sec. 6 is the time-averaged force
on the particles, read from their tethers, whose closed form is
Eq. (eq:acousticForce2) with the contrast factors f_1 (Eq. (f1), through the
excess compressibility) and f_2 (Eq. (f2), through the excess mass).  Here the
objective is the discrete quantity the method computes,

    Phi = sum_n w_n sum_p d_p . F_p^{n+1/2} / sum_n w_n,
    F_p^{n+1/2} = -k_p (q_p^{n+1/2} - q_p^eq)      (substep 2 of App. A.2),

for a rollout of deterministic (kT = 0) steps of ``ic.Simulation.step`` in its
default momentum form, and its gradient is taken with respect to every
particle's excess mass m_e, its compressibility ratio kappa_p/kappa_f
(epsilon_pf = c^2 (kappa_f/kappa_p - 1), Eqs. (part_svel), (ke)), the drive
amplitude A of the standing wave, and the initial state (delta rho, g, q, u).

How.  Each function below is the transpose of one line group of the forward
step, taken in reverse order: the interpolation J and the spreading S swap
roles (they are adjoint, Eq. (adj)), np.roll by +1 becomes np.roll by -1, and
products give the usual two terms.  Positions enter through the kernel
weights, whose derivative is that of the 3-point function (App. A.1); the
periodic wrap of positions and of the tether displacement has derivative 1.
Nothing here is blocked or fused; the forward intermediates are recomputed
from the state at the start of each step (``record_step``).
"""
import numpy as np

from . import fluid, peskin
from .fluid import dn, up
from .ic import epsilon_from_kappa_ratio, external_pressure


def phi_prime(r):
    """d phi / d r of the 3-point Roma-Peskin function (App. A.1).

    Inner branch (|r| <= 1/2): phi = (1 + sqrt(1 - 3 r^2)) / 3, so
    phi' = -r / sqrt(1 - 3 r^2).  Outer branch (1/2 < |r| <= 3/2):
    phi = (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6, so
    phi' = -sign(r) (1 + (1 - |r|) / sqrt(1 - 3 (1 - |r|)^2)) / 2.
    Both branches give -sign(r) at |r| = 1/2 and 0 at |r| = 3/2 (phi is C^1).
    """
    r = np.asarray(r, dtype=np.float64)
    a = np.abs(r)
    out = np.zeros_like(r)
    inner = a <= 0.5
    outer = (a > 0.5) & (a <= 1.5)
    out[inner] = -r[inner] / np.sqrt(1.0 - 3.0 * r[inner] ** 2)
    b = 1.0 - a[outer]
    out[outer] = -np.sign(r[outer]) * 0.5 * (1.0 + b / np.sqrt(1.0 - 3.0 * b ** 2))
    return out


class StencilsD(peskin.Stencils):
    """Stencils with the derivative of each weight with respect to q.

    dw (np, 27, 3): d w_i / d q_alpha = -(1/h) phi'(x_i/h - s_alpha) times the
    other two 1D weights.
    """

    def __init__(self, q, h, shape, offset):
        super().__init__(q, h, shape, offset)
        q = np.atleast_2d(np.asarray(q, dtype=np.float64))
        one = []
        for ax in range(3):
            s = q[:, ax] / h - offset[ax]
            i0 = np.floor(s + 0.5).astype(np.int64)
            rel = i0[:, None] + np.arange(-1, 2) - s[:, None]
            one.append((peskin.phi(rel), -phi_prime(rel) / h))
        (wx, dwx), (wy, dwy), (wz, dwz) = one
        npart = q.shape[0]

        def prod(fx, fy, fz):
            return (fz[:, :, None, None] * fy[:, None, :, None] * fx[:, None, None, :]).reshape(npart, 27)

        self.dw = np.stack([prod(dwx, wy, wz), prod(wx, dwy, wz), prod(wx, wy, dwz)], axis=2)

    def interp_grad(self, field):
        """d (J f)_p / d q_p for every particle: (np, 3)."""
        return np.sum(self.dw * field.reshape(-1)[self.flat][:, :, None], axis=1)

    def interp_T(self, values, shape):
        """Transpose of J: point i receives w_i values_p (no 1/h^3)."""
        out = np.zeros(int(np.prod(shape)))
        np.add.at(out, self.flat.reshape(-1), (self.w * np.asarray(values, dtype=np.float64)[:, None]).reshape(-1))
        return out.reshape(shape)


def all_stencils_d(q, h, shape):
    return (StencilsD(q, h, shape, peskin.CENTRE),
            tuple(StencilsD(q, h, shape, peskin.FACE[a]) for a in range(3)))


# ------------------------------------------------------------------ fluid part
def velocities(p, drho, g):
    return [g[a] / (p.rho0 + 0.5 * (drho + up(drho, a))) for a in range(3)]


def velocities_vjp(p, drho, g, v_bar):
    """Transpose of v^a = g^a / (rho0 + (drho_i + drho_{i+a}) / 2): (drho_bar, g_bar)."""
    drho_bar = np.zeros_like(drho)
    g_bar = []
    for a in range(3):
        rf = p.rho0 + 0.5 * (drho + up(drho, a))
        g_bar.append(v_bar[a] / rf)
        rf_bar = -v_bar[a] * (g[a] / rf) / rf
        drho_bar += 0.5 * (rf_bar + dn(rf_bar, a))
    return drho_bar, g_bar


def rates_vjp(drho, g, p, lam_rho, lam_g):
    """Transpose of ``fluid.rates`` (deterministic) applied to (lam_rho, lam_g).

    Returns (drho_bar, g_bar, pi_bar): the adjoints of the density excess, the
    face momenta and the extra centre pressure (particle pressure plus drive).
    The face force enters the rates additively, so its adjoint is lam_g itself.
    """
    h, eta = p.h, p.eta
    lam2 = p.zeta - 2.0 * eta / 3.0
    rho_face = [p.rho0 + 0.5 * (drho + up(drho, a)) for a in range(3)]
    v = [g[a] / rho_face[a] for a in range(3)]

    g_bar = [np.zeros_like(drho) for _ in range(3)]
    v_bar = [np.zeros_like(drho) for _ in range(3)]
    pi_bar = np.zeros_like(drho)
    dv_bar = [np.zeros_like(drho) for _ in range(3)]
    divv_bar = np.zeros_like(drho)

    # dg_a = -(up(t_cc_a, a) - t_cc_a + sum_b (flux_ab - dn(flux_ab, b))) / h
    t_bar = [(lam_g[a] - dn(lam_g[a], a)) / h for a in range(3)]
    f_bar = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            if b != a:
                f_bar[a][b] = (up(lam_g[a], b) - lam_g[a]) / h

    # off-diagonal fluxes on edges
    for a, b in fluid.EDGES:
        # flux_ab = 1/4 (g_a + up(g_a, b)) (v_b + up(v_b, a)) - visc
        A = g[a] + up(g[a], b)
        B = v[b] + up(v[b], a)
        A_bar = 0.25 * f_bar[a][b] * B
        B_bar = 0.25 * f_bar[a][b] * A
        g_bar[a] += A_bar + dn(A_bar, b)
        v_bar[b] += B_bar + dn(B_bar, a)
        # flux_ba = 1/4 (g_b + up(g_b, a)) (v_a + up(v_a, b)) - visc
        A = g[b] + up(g[b], a)
        B = v[a] + up(v[a], b)
        A_bar = 0.25 * f_bar[b][a] * B
        B_bar = 0.25 * f_bar[b][a] * A
        g_bar[b] += A_bar + dn(A_bar, a)
        v_bar[a] += B_bar + dn(B_bar, b)
        # visc = eta ((up(v_a, b) - v_a) / h + (up(v_b, a) - v_b) / h), in both fluxes with sign -1
        visc_bar = -(f_bar[a][b] + f_bar[b][a])
        v_bar[a] += eta * (dn(visc_bar, b) - visc_bar) / h
        v_bar[b] += eta * (dn(visc_bar, a) - visc_bar) / h

    # diagonal at centres: 1/4 (dn(g_a, a) + g_a)(dn(v_a, a) + v_a) + pi - 2 eta dv_a - lam2 div v
    for a in range(3):
        C = dn(g[a], a) + g[a]
        D = dn(v[a], a) + v[a]
        C_bar = 0.25 * t_bar[a] * D
        D_bar = 0.25 * t_bar[a] * C
        g_bar[a] += C_bar + up(C_bar, a)
        v_bar[a] += D_bar + up(D_bar, a)
        pi_bar += t_bar[a]
        dv_bar[a] += -2.0 * eta * t_bar[a]
        divv_bar += -lam2 * t_bar[a]
    for a in range(3):
        dv = dv_bar[a] + divv_bar
        # dv_a = (v_a - dn(v_a, a)) / h
        v_bar[a] += (dv - up(dv, a)) / h

    # pi = c^2 drho + extra
    drho_bar = p.c ** 2 * pi_bar
    # v_a = g_a / rho_face_a
    d2, g2 = velocities_vjp(p, drho, g, v_bar)
    drho_bar = drho_bar + d2
    for a in range(3):
        g_bar[a] += g2[a]
        # drho_dt = -sum_a (g_a - dn(g_a, a)) / h
        g_bar[a] += -(lam_rho - up(lam_rho, a)) / h
    return drho_bar, g_bar, pi_bar


# ------------------------------------------------------------------ one step
def drive_per_amplitude(p, t):
    """d p_ext / d A at time t (the drive is linear in A), or None."""
    if p.forcing == "none":
        return None
    q = p.__class__(**{**p.__dict__, "wave_amp": 1.0})
    return external_pressure(q, t)


def record_step(p, parts, drho, g, step_index):
    """The deterministic IC step of ``ic.Simulation.step`` (momentum form 'g'),
    keeping the intermediates the reverse sweep needs.

    parts: dict q, u, m_e, eps, k_s, q_eq (arrays).  Returns (tape, new state
    dict drho, g, q, u).  The arithmetic is that of ``ic.Simulation.step``,
    statement for statement, so the new state is identical to it.
    """
    if p.kT != 0.0 or p.momentum_form != "g":
        raise ValueError("the adjoint covers the deterministic step in the 'g' momentum form")
    h, dt, shape = p.h, p.dt, p.shape
    vol = peskin.kernel_volume(h)
    t_n = step_index * dt
    L = p.lengths
    q, u = parts["q"], parts["u"]
    npart = q.shape[0]
    v_n = velocities(p, drho, g)
    T = dict(drho_n=drho, g_n=g, v_n=v_n, q_n=q, u_n=u, t_n=t_n)
    if npart:
        cen_n, faces_n = all_stencils_d(q, h, shape)
        jv_n = np.stack([faces_n[a].interp(v_n[a]) for a in range(3)], axis=1)
        q_half = np.mod(q + 0.5 * dt * jv_n, L)
        d = q_half - parts["q_eq"]
        d = d - L * np.round(d / L)
        force = -parts["k_s"][:, None] * d
        centre, faces = all_stencils_d(q_half, h, shape)
        jv_nh = np.stack([faces[a].interp(v_n[a]) for a in range(3)], axis=1)
        face_force = [faces[a].spread(force[:, a], shape, h) for a in range(3)]
        T.update(faces_n=faces_n, q_half=q_half, force=force, centre=centre, faces=faces)
    else:
        face_force = None
    rho_s, g_s = drho, g
    stages = []
    for s in range(3):
        extra = external_pressure(p, t_n + fluid.RK3_TIME[s] * dt)
        omega = None
        if npart:
            omega = parts["eps"] * vol * centre.interp(rho_s)
            pp = centre.spread(omega, shape, h)
            extra = pp if extra is None else extra + pp
        stages.append(dict(drho=rho_s, g=g_s, omega=omega))
        drho_dt, dg = fluid.rates(rho_s, g_s, p.fluid(), extra, None, face_force)
        rho_next = fluid.rk3_combine(s, drho, rho_s, dt * drho_dt)
        g_next = [fluid.rk3_combine(s, g[a], g_s[a], dt * dg[a]) for a in range(3)]
        rho_s, g_s = rho_next, g_next
    T["stages"] = stages
    rho_new, g_tilde = rho_s, g_s
    if npart:
        v_tilde = velocities(p, rho_new, g_tilde)
        jv_tilde = np.stack([faces[a].interp(v_tilde[a]) for a in range(3)], axis=1)
        m_f = vol * (p.rho0 + centre.interp(rho_new))
        me = parts["m_e"][:, None]
        mf = m_f[:, None]
        dgp = me * mf / (me + mf) * (jv_tilde - u)
        u_new = u + mf / (me + mf) * (jv_tilde - u)
        g_new = [g_tilde[a] - faces[a].spread(dgp[:, a], shape, h) for a in range(3)]
        v_new = velocities(p, rho_new, g_new)
        jv_new = np.stack([faces[a].interp(v_new[a]) for a in range(3)], axis=1)
        q_new = np.mod(q + 0.5 * dt * (jv_new + jv_nh), L)
        T.update(g_tilde=g_tilde, v_tilde=v_tilde, jv_tilde=jv_tilde, m_f=m_f, dgp=dgp, g_new=g_new,
                 v_new=v_new)
    else:
        g_new, q_new, u_new = g_tilde, q, u
    T["drho_new"] = rho_new
    return T, dict(drho=rho_new, g=g_new, q=q_new, u=u_new)


def adjoint_step(p, parts, T, bar, weight, direction):
    """Reverse sweep of one recorded step.

    bar: adjoints of the step's outputs, dict drho, g (list of 3), q, u.
    weight, direction: this step's term weight * sum_p direction_p . F_p of the
    objective.  Returns (adjoints of the step's inputs, dict of gradient
    contributions m_e (np), eps (np), A (scalar)).
    """
    h, dt, shape = p.h, p.dt, p.shape
    vol = peskin.kernel_volume(h)
    h3 = h ** 3
    npart = T["q_n"].shape[0]
    drho_bar = bar["drho"].copy()
    g_bar = [x.copy() for x in bar["g"]]
    grad = dict(m_e=np.zeros(npart), eps=np.zeros(npart), A=0.0)
    if npart:
        faces, centre = T["faces"], T["centre"]
        me, mf = parts["m_e"], T["m_f"]
        q_bar = bar["q"].copy()                 # d q^{n+1} / d q^n = 1
        qh_bar = np.zeros((npart, 3))
        # substep 7: q^{n+1} = q^n + dt/2 (J^{n+1/2} v^{n+1} + J^{n+1/2} v^n)
        jv_new_bar = 0.5 * dt * bar["q"]
        jv_nh_bar = 0.5 * dt * bar["q"]
        v_bar = [faces[a].interp_T(jv_new_bar[:, a], shape) for a in range(3)]
        qh_bar += sum(jv_new_bar[:, [a]] * faces[a].interp_grad(T["v_new"][a]) for a in range(3))
        d2, g2 = velocities_vjp(p, T["drho_new"], T["g_new"], v_bar)
        drho_bar += d2
        for a in range(3):
            g_bar[a] += g2[a]
        # substep 6: g^{n+1} = g~ - S dg
        dgp_bar = np.stack([-faces[a].interp(g_bar[a]) / h3 for a in range(3)], axis=1)
        qh_bar += sum(-T["dgp"][:, [a]] / h3 * faces[a].interp_grad(g_bar[a]) for a in range(3))
        # substeps 4-5: dg = mu (J v~ - u), u^{n+1} = u + r (J v~ - u), r = m_f / (m_e + m_f), mu = m_e r
        dvel = T["jv_tilde"] - T["u_n"]
        tot = me + mf
        r = (mf / tot)[:, None]
        mu = (me * mf / tot)[:, None]
        jvt_bar = r * bar["u"] + mu * dgp_bar
        u_bar = (1.0 - r) * bar["u"] - mu * dgp_bar
        su = np.sum(bar["u"] * dvel, axis=1)
        sg = np.sum(dgp_bar * dvel, axis=1)
        mf_bar = me / tot ** 2 * su + me ** 2 / tot ** 2 * sg
        grad["m_e"] += -mf / tot ** 2 * su + mf ** 2 / tot ** 2 * sg
        # m_f = V (rho0 + J_c rho^{n+1})
        drho_bar += vol * centre.interp_T(mf_bar, shape)
        qh_bar += vol * mf_bar[:, None] * centre.interp_grad(T["drho_new"])
        # J v~ at q^{n+1/2}
        v_bar = [faces[a].interp_T(jvt_bar[:, a], shape) for a in range(3)]
        qh_bar += sum(jvt_bar[:, [a]] * faces[a].interp_grad(T["v_tilde"][a]) for a in range(3))
        d2, g2 = velocities_vjp(p, T["drho_new"], T["g_tilde"], v_bar)
        drho_bar += d2
        for a in range(3):
            g_bar[a] += g2[a]
        force_bar = np.zeros((npart, 3))
    else:
        u_bar = bar["u"].copy() if "u" in bar else np.zeros((0, 3))
        q_bar = bar["q"].copy() if "q" in bar else np.zeros((0, 3))

    # substep 3: SSP-RK3 stages in reverse; (drho_bar, g_bar) is the adjoint of U_{s+1}
    acc_rho = np.zeros(shape)
    acc_g = [np.zeros(shape) for _ in range(3)]
    for s in (2, 1, 0):
        st = T["stages"][s]
        a_s, b_s = fluid.RK3_A[s], fluid.RK3_B[s]
        lam_rho = b_s * dt * drho_bar
        lam_g = [b_s * dt * x for x in g_bar]
        r_rho, r_g, pi_bar = rates_vjp(st["drho"], st["g"], p, lam_rho, lam_g)
        new_rho = b_s * drho_bar + r_rho
        new_g = [b_s * g_bar[a] + r_g[a] for a in range(3)]
        dpa = drive_per_amplitude(p, T["t_n"] + fluid.RK3_TIME[s] * dt)
        if dpa is not None:
            grad["A"] += float(np.sum(pi_bar * dpa))
        if npart:
            # pi += S_c Omega, Omega = eps V J_c rho_s
            omega_bar = centre.interp(pi_bar) / h3
            qh_bar += st["omega"][:, None] / h3 * centre.interp_grad(pi_bar)
            jr = centre.interp(st["drho"])
            grad["eps"] += vol * jr * omega_bar
            new_rho += centre.interp_T(parts["eps"] * vol * omega_bar, shape)
            qh_bar += (parts["eps"] * vol * omega_bar)[:, None] * centre.interp_grad(st["drho"])
            # face force S F enters every stage's rates
            for a in range(3):
                force_bar[:, a] += faces[a].interp(lam_g[a]) / h3
            qh_bar += sum(T["force"][:, [a]] / h3 * faces[a].interp_grad(lam_g[a]) for a in range(3))
        if s > 0:
            acc_rho += a_s * drho_bar
            for a in range(3):
                acc_g[a] += a_s * g_bar[a]
        drho_bar, g_bar = new_rho, new_g
    drho_bar = drho_bar + acc_rho
    g_bar = [g_bar[a] + acc_g[a] for a in range(3)]

    if npart:
        faces_n = T["faces_n"]
        # substep 2: F = -k_s (q^{n+1/2} - q_eq), plus the objective's own term
        force_bar += weight * direction
        qh_bar += -parts["k_s"][:, None] * force_bar
        # J^{n+1/2} v^n (substep 7's second term)
        v_bar = [faces[a].interp_T(jv_nh_bar[:, a], shape) for a in range(3)]
        qh_bar += sum(jv_nh_bar[:, [a]] * faces[a].interp_grad(T["v_n"][a]) for a in range(3))
        # substep 1: q^{n+1/2} = q^n + dt/2 J^n v^n
        q_bar += qh_bar
        jv_n_bar = 0.5 * dt * qh_bar
        for a in range(3):
            v_bar[a] = v_bar[a] + faces_n[a].interp_T(jv_n_bar[:, a], shape)
        q_bar += sum(jv_n_bar[:, [a]] * faces_n[a].interp_grad(T["v_n"][a]) for a in range(3))
        d2, g2 = velocities_vjp(p, T["drho_n"], T["g_n"], v_bar)
        drho_bar += d2
        for a in range(3):
            g_bar[a] += g2[a]
    return dict(drho=drho_bar, g=g_bar, q=q_bar, u=u_bar), grad


# ------------------------------------------------------------------ rollout
def make_parts(q, u, m_e, kappa_ratio, k_s, c, q_eq=None):
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    n = q.shape[0]
    return dict(q=q, u=np.atleast_2d(np.asarray(u, dtype=np.float64)).reshape(n, 3),
                m_e=np.broadcast_to(np.asarray(m_e, float), (n,)).copy(),
                eps=epsilon_from_kappa_ratio(np.broadcast_to(np.asarray(kappa_ratio, float), (n,)), c),
                k_s=np.broadcast_to(np.asarray(k_s, float), (n,)).copy(),
                q_eq=q.copy() if q_eq is None else np.atleast_2d(np.asarray(q_eq, float)))


def rollout(p, drho, g, parts, weights, direction, step0=0):
    """Objective Phi of ``nsteps = len(weights)`` deterministic steps."""
    parts = dict(parts)
    sf = 0.0
    for n, w in enumerate(weights):
        T, new = record_step(p, parts, drho, g, step0 + n)
        if parts["q"].shape[0]:
            sf += w * float(np.sum(direction * T["force"]))
        drho, g = new["drho"], new["g"]
        parts["q"], parts["u"] = new["q"], new["u"]
    return sf / float(np.sum(weights)), dict(drho=drho, g=g, q=parts["q"], u=parts["u"])


def rollout_gradient(p, drho, g, parts, weights, direction, checkpoint_every=None, step0=0):
    """(Phi, gradients) of a rollout by the reverse sweep with checkpointing.

    States are kept every ``checkpoint_every`` steps (all steps if None); the
    steps in between are recomputed forward before their reverse sweep.
    Gradients: m_e, kappa_ratio (per particle), A (drive only), and the
    adjoint of the initial state drho, g, q, u.
    """
    weights = np.asarray(weights, dtype=np.float64)
    nsteps = len(weights)
    W = float(np.sum(weights))
    K = nsteps if checkpoint_every is None else int(checkpoint_every)
    parts = {k: np.array(v, dtype=np.float64) for k, v in parts.items()}
    # forward sweep keeping the checkpoints
    ckpt = {}
    cur = dict(drho=drho, g=g, q=parts["q"], u=parts["u"])
    phi = 0.0
    for n in range(nsteps):
        if n % K == 0:
            ckpt[n] = cur
        pn = {**parts, "q": cur["q"], "u": cur["u"]}
        T, cur = record_step(p, pn, cur["drho"], cur["g"], step0 + n)
        if pn["q"].shape[0]:
            phi += weights[n] * float(np.sum(direction * T["force"]))
    phi /= W
    # reverse sweep, segment by segment
    npart = parts["q"].shape[0]
    bar = dict(drho=np.zeros(p.shape), g=[np.zeros(p.shape) for _ in range(3)], q=np.zeros((npart, 3)),
               u=np.zeros((npart, 3)))
    grad = dict(m_e=np.zeros(npart), eps=np.zeros(npart), A=0.0)
    for start in sorted(ckpt, reverse=True):
        stop = min(start + K, nsteps)
        states = [ckpt[start]]
        for n in range(start, stop - 1):
            s = states[-1]
            _, nxt = record_step(p, {**parts, "q": s["q"], "u": s["u"]}, s["drho"], s["g"], step0 + n)
            states.append(nxt)
        for n in range(stop - 1, start - 1, -1):
            s = states[n - start]
            pn = {**parts, "q": s["q"], "u": s["u"]}
            T, _ = record_step(p, pn, s["drho"], s["g"], step0 + n)
            bar, gr = adjoint_step(p, pn, T, bar, weights[n] / W, direction)
            for k in grad:
                grad[k] = grad[k] + gr[k]
    kappa = p.c ** 2 / (parts["eps"] + p.c ** 2)          # kappa_p / kappa_f from epsilon
    grad["kappa_ratio"] = grad["eps"] * (-p.c ** 2 / kappa ** 2)
    grad["state"] = bar
    return phi, grad
