"""The whole-row FP32 stage kernel (tile variant "rows": a CTA per band of
whole x rows, bulk copies of the planes into shared memory, four cells per
thread).

Its per-cell arithmetic is the same sequence of rounded operations as the
wide-tile kernel's, so deterministic steps (kT = 0) give the same bits, for
every band height and run split the planner picks: one band of every row,
bands with ring rows and a ragged last band, short and long z runs, particles,
and every drive and wave axis.  With noise it stores the stress divergence of
W_2 and W_3 (3 words each) instead of their normals, which rounds differently:
those steps are checked against the oracle at the FP32 tolerance.
"""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W
from pairs import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

# (nx, ny, nz), forcing, wave axis, particles
CASES = [
    ((128, 20, 10), "mode", 0, 6),     # bands with ring rows, ragged last band
    ((40, 20, 18), "plane", 1, 5),     # one band of every row
    ((64, 30, 9), "mode", 2, 9),
    ((12, 30, 7), "plane", 0, 3),
    ((8, 6, 6), "none", 0, 2),         # the smallest box
    ((128, 64, 12), "mode", 0, 12),    # the benchmark's rows
]


def particles(shape, n, seed):
    if n == 0:
        return None
    rng = np.random.default_rng(seed)
    L = np.array(shape, dtype=float)
    q = rng.uniform(0.0, 1.0, (n, 3)) * L
    if n > 2:
        q[1] = (q[0] + rng.uniform(-1.0, 1.0, 3)) % L   # overlapping kernels
        q[2, 0] = L[0] - 0.05                            # on the periodic seam
    return dict(q=q, m_e=rng.uniform(-2.0, 8.0, n), kappa_ratio=rng.uniform(0.3, 2.0, n),
                k_spring=np.where(rng.uniform(size=n) < 0.5, rng.uniform(0.1, 1.0, n), 0.0))


def params(case, kT):
    shape, forcing, axis, _ = CASES[case]
    return W.grid_params(shape, kT=kT, wave_amp=2e-3, forcing=forcing, wave_axis=axis,
                         plane_index=min(3, shape[axis] - 1), zeta=0.3, seed=17 + case, precision="fp32",
                         wave_phase=0.4)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rows_equal_wide_tile_bit_for_bit(case):
    gp = params(case, 0.0)
    rho, g = W.random_fields(gp, seed=case)
    parts = particles(CASES[case][0], CASES[case][3], case)
    w = np.linspace(0.5, 1.0, 5)
    runs = [run_gpu(gp, rho, g, parts, nsteps=5, weights=w, tile=t) for t in ((0, 8), (0, 32), (32, 16))]
    assert all(r["tile"][0] == gp["nx"] for r in runs[:2]), [r["tile"] for r in runs]
    assert runs[2]["tile"][0] == 32
    keys = ["rho", "u", "q", "lam", "f_avg", "lam_avg"] if parts else ["rho"]
    for other in runs[1:]:
        for k in keys:
            assert np.array_equal(runs[0][k], other[k]), k
        for a in range(3):
            assert np.array_equal(runs[0]["g"][a], other["g"][a]), a
        assert np.array_equal(runs[0]["p_total"], other["p_total"])
        if parts:
            assert abs(runs[0]["a2"] - other["a2"]) <= 1e-5 * abs(other["a2"])


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rows_with_noise_against_oracle(case):
    gp = params(case, 1e-3)
    rho, g = W.random_fields(gp, seed=case)
    parts = particles(CASES[case][0], CASES[case][3], case)
    w = np.linspace(0.5, 1.0, 4)
    sim = run_oracle(gp, rho, g, parts, nsteps=4, weights=w, thermal_seed=3)
    out = run_gpu(gp, rho, g, parts, nsteps=4, weights=w, thermal_seed=3, tile=(0, 8))
    assert out["tile"][0] == gp["nx"]
    errs = compare(out, sim, gp, q0=None if parts is None else parts["q"])
    bad = {k: v for k, v in errs.items() if not v <= 1e-4}
    assert not bad, errs


def test_rows_noise_runs_split_anywhere():
    """With noise, the stored divergence does not depend on where the runs of
    z planes start and end (the stage-1 stresses of the plane below a run are
    drawn again by the CTA that starts there)."""
    gp = params(0, 1e-3)
    rho, g = W.random_fields(gp, seed=9)
    a = run_gpu(gp, rho, g, nsteps=3, thermal_seed=5, tile=(0, 8))
    b = run_gpu(gp, rho, g, nsteps=3, thermal_seed=5, tile=(0, 32))
    assert np.array_equal(a["rho"], b["rho"])
    for k in range(3):
        assert np.array_equal(a["g"][k], b["g"][k])
