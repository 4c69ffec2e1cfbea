"""Static structure factors of the library's thermal fluid (Sec. 4.5), the
check tests/test_oracle_structure_factor.py makes on the oracle, here on the
GPU in both precisions: every Fourier mode of the density carries
rho0 kT / c^2, the longitudinal velocity kT / rho0 and the two transverse
components kT / rho0 each, flat in |k|.  A noise component or coefficient
wrong at some wavenumbers only (which a real-space variance averages away)
shows up in a shell.

Protocol: 16^3 with bulk viscosity, started at rest, 2000 relaxation steps,
then 640 snapshots 50 steps apart in 16 batches (each batch spans ~4 decay
times of the slowest shear mode); per |k| shell the mean of the batch means
within 3.5 standard errors of the closed form, the middle shells pooled
within 1 %."""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W
from test_oracle_structure_factor import shells, structure_factors

pytestmark = pytest.mark.gpu

N, RELAX, EVERY, SNAPSHOTS, BATCHES = 16, 2000, 50, 640, 16


def velocities(drho, g, rho0):
    """Face velocities g^a / (rho0 + (drho_i + drho_{i+a}) / 2)."""
    from oracle import fluid

    return [g[a] / (rho0 + 0.5 * (drho + fluid.up(drho, a))) for a in range(3)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_flat_structure_factors_on_the_gpu(prec):
    from oracle import ic as oic
    from paper_1307_0702_gb300 import Grid

    gp = W.grid_params(N, kT=1e-3, zeta=0.5, wave_amp=0.0, forcing="none", seed=13, precision=prec)
    p = oic.GridParams(nx=N, ny=N, nz=N, kT=gp["kT"], zeta=gp["zeta"], seed=gp["seed"])
    rho0 = np.full((N, N, N), gp["rho0"])
    zero = [np.zeros((N, N, N)) for _ in range(3)]
    S = []
    with Grid(gp) as grid:
        grid.set_state(rho0, zero)
        grid.step(RELAX)
        for _ in range(SNAPSHOTS):
            grid.step(EVERY)
            rho, g = grid.get_state()
            drho = rho - gp["rho0"]
            S.append(structure_factors(p, drho, velocities(drho, g, gp["rho0"])))
    S = np.array(S)
    expect = [gp["rho0"] * gp["kT"] / gp["c"] ** 2, gp["kT"] / gp["rho0"], 2.0 * gp["kT"] / gp["rho0"]]
    shell = shells(N)
    for f in range(3):
        pooled = []
        for j in range(1, shell.max() + 1):
            sel = shell == j
            per = S[:, f][:, sel].mean(axis=1) / expect[f]
            b = per.reshape(BATCHES, -1).mean(axis=1)
            mu, se = b.mean(), b.std(ddof=1) / np.sqrt(BATCHES)
            assert abs(mu - 1.0) <= 3.5 * se, (prec, f, j, mu, se)
            if 4 <= j <= 10:
                pooled.append(per)
        assert abs(np.mean(pooled) - 1.0) <= 0.01, (prec, f, np.mean(pooled))
