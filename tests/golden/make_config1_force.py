"""Writes config1_force.json: the oracle's time-averaged tether force on the
single particle of the deterministic 32^3 standing-wave box (h = 1, FP64,
kT = 0; the particle at (L/8, L/2, L/2), m_p = 1.5 rho0 V, kappa_p = 0.5
kappa_f, spring k_s = 1; the mode drive holding density amplitude 1e-3 from
the velocity-phase start), averaged with a Blackman-Harris window over steps
3000..8000 (the period averages of the spring force have settled by step
3000).

    python tests/golden/make_config1_force.py

Calls only the oracle (oracle/ic.py) and the input generators; takes a few
minutes.  The GPU tests compare the library's FP64 and FP32 runs with it."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ic as oic  # noqa: E402
from oracle import theory  # noqa: E402
from paper_1307_0702_gb300 import workloads as W  # noqa: E402

NSTEPS, SKIP = 8000, 3000


def main():
    gp, parts, _ = W.single_particle_config()
    p = oic.GridParams(**{k: v for k, v in gp.items() if k in oic.GridParams.__dataclass_fields__})
    rho, g = W.velocity_phase_wave_fields(gp)
    sim = oic.Simulation(p, rho, g)
    sim.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
    w = W.blackman_harris(NSTEPS, SKIP)
    sim.run(NSTEPS, w)
    f, lam, a2 = sim.time_average()
    L = p.nx * p.h
    fg = theory.gorkov_force(p.c, np.sqrt(2.0 * a2), 8.0 * p.h ** 3, 2.0 * np.pi / L, p.rho0,
                             parts["kappa_ratio"][0], parts["m_e"][0], L / 8.0)
    out = {"nsteps": NSTEPS, "skip": SKIP, "f_spring": f[0].tolist(), "lambda": lam[0].tolist(), "a2": a2,
           "gorkov": fg, "ratio": -f[0, 0] / fg,
           "note": "oracle FP64, deterministic 32^3 box, single tethered particle; written by make_config1_force.py"}
    with open(os.path.join(HERE, "config1_force.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
