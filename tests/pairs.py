"""Run the same seeded input through libic (GPU) and the CPU oracle."""
import numpy as np

from oracle import ic as oic

ORACLE_KEYS = {f for f in oic.GridParams.__dataclass_fields__}


def oracle_params(gp, **over):
    d = {k: v for k, v in gp.items() if k in ORACLE_KEYS}
    d.update(over)
    return oic.GridParams(**d)


def run_gpu(gp, rho, g, parts=None, nsteps=1, weights=None, thermal_seed=None, chunks=None, tile=None,
            stage_copy=None):
    from paper_1307_0702_gb300 import Grid

    out = {}
    with Grid(gp) as grid:
        if tile is not None:
            grid.set_tile(*tile)
        if stage_copy is not None:
            grid.set_stage_copy(stage_copy)
        out["stage_copy"] = grid.stage_copy()
        out["tile"] = grid.tile()
        grid.set_state(rho, g)
        if thermal_seed is not None:
            grid.init_thermal(thermal_seed, add=True)
        if parts is not None:
            grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts.get("k_spring"), parts.get("u"))
        for lo, hi in (chunks or [(0, nsteps)]):
            grid.step(hi - lo, None if weights is None else weights[lo:hi])
        out["rho"], out["g"] = grid.get_state()
        if parts is not None:
            out["lam"], out["u"], out["q"] = grid.forces()
            if weights is not None:
                out["f_avg"], out["lam_avg"], out["a2"] = grid.time_average()
        out["p_total"], out["mode"], out["step"] = grid.stats()
    return out


def run_oracle(gp, rho, g, parts=None, nsteps=1, weights=None, thermal_seed=None, **over):
    p = oracle_params(gp, **over)
    drho = np.asarray(rho, dtype=np.float64) - p.rho0
    if thermal_seed is not None:
        th_drho, th_g = oic.thermal_fluctuation(p, thermal_seed)
        drho = drho + th_drho
        g = [g[a] + th_g[a] for a in range(3)]
    sim = oic.Simulation(p, g=g, drho=drho)
    if parts is not None:
        sim.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts.get("k_spring"), parts.get("u"))
    sim.run(nsteps, weights)
    return sim


def rel_err(a, b, ref=0.0):
    """max |a - b| / max |b - ref| (normwise, per field)."""
    scale = np.max(np.abs(np.asarray(b) - ref))
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / (scale if scale > 0 else 1.0)


def compare(out, sim, gp, q0=None):
    """Relative errors of every output against the oracle simulation."""
    errs = {"rho": rel_err(out["rho"], sim.rho, gp["rho0"])}
    for a in range(3):
        errs[f"g{a}"] = rel_err(out["g"][a], sim.g[a])
    if "u" in out:
        errs["u"] = rel_err(out["u"], sim.parts.u)
        errs["lam"] = rel_err(out["lam"], sim.lam)
        L = sim.p.lengths
        dq = out["q"] - sim.parts.q
        dq -= L * np.round(dq / L)
        disp = sim.parts.q - (q0 if q0 is not None else sim.parts.q_eq)
        disp -= L * np.round(disp / L)
        errs["q"] = np.max(np.abs(dq)) / max(np.max(np.abs(disp)), 1e-300)
    if "f_avg" in out:
        fo, lo, a2o = sim.time_average()
        errs["f_avg"] = rel_err(out["f_avg"], fo)
        errs["lam_avg"] = rel_err(out["lam_avg"], lo)
        errs["a2"] = abs(out["a2"] - a2o) / abs(a2o)
    return errs
