"""GPU (libic through the C ABI) against the CPU oracle, element by element.

FP64: every field, particle quantity and weighted average within 1e-11
relative (normwise per field: max |gpu - oracle| / max |oracle - reference|),
with the same Philox streams on both sides.  FP32: within 1e-4 relative.
Sizes span several CTA tiles (32 x 13 cells for FP32, 32 x 6 for FP64, each
marching runs of z planes) and ragged tails.
"""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W
from pairs import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-4}


def particles(n, shape, seed, m_e=4.0, kappa=0.5, k_spring=0.7, overlap=True):
    rng = np.random.default_rng(seed)
    L = np.array(shape[::-1], dtype=float)
    q = rng.uniform(0, 1, (n, 3)) * L
    if overlap and n >= 2:
        q[1] = (q[0] + np.array([1.3, -0.8, 0.4])) % L          # overlapping kernels
    if n >= 3:
        q[2] = np.array([0.0, 0.5, L[2] - 1e-9])              # on the periodic seam
    if n >= 4:
        q[3] = np.array([2.5, 3.5, 1.5])                       # half-integer tie
    return dict(q=q, m_e=np.full(n, m_e) if np.isscalar(m_e) else m_e,
                kappa_ratio=np.full(n, kappa) if np.isscalar(kappa) else kappa,
                k_spring=np.full(n, k_spring))


def check(errs, tol):
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"errors above {tol}: {bad} (all: {errs})"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fluid_only_deterministic(prec):
    gp = W.grid_params((37, 19, 22), kT=0.0, wave_amp=0.0, forcing="none", zeta=0.3, precision=prec)
    rho, g = W.random_fields(gp, seed=3, amp_rho=1e-2, amp_g=1e-2)
    out = run_gpu(gp, rho, g, nsteps=6)
    sim = run_oracle(gp, rho, g, nsteps=6)
    check(compare(out, sim, gp), TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fluid_with_noise_and_mode_drive(prec):
    gp = W.grid_params((33, 17, 18), kT=1e-3, wave_amp=2e-3, forcing="mode", zeta=0.4, seed=11,
                       precision=prec, wave_phase=0.3)
    rho, g = W.random_fields(gp, seed=4)
    out = run_gpu(gp, rho, g, nsteps=5)
    sim = run_oracle(gp, rho, g, nsteps=5)
    check(compare(out, sim, gp), TOL[prec])


@pytest.mark.parametrize("axis", [1, 2])
def test_plane_drive_on_other_axes(axis):
    gp = W.grid_params((12, 14, 16), kT=1e-4, wave_amp=1e-3, forcing="plane", wave_axis=axis,
                       plane_index=3, seed=2)
    rho, g = W.standing_wave_fields(gp)
    out = run_gpu(gp, rho, g, nsteps=8)
    sim = run_oracle(gp, rho, g, nsteps=8)
    check(compare(out, sim, gp), TOL["fp64"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_particles_full_step(prec):
    gp = W.grid_params((20, 18, 16), kT=1e-3, wave_amp=1e-3, zeta=0.2, seed=5, precision=prec)
    rho, g = W.random_fields(gp, seed=6)
    parts = particles(7, (16, 18, 20), seed=1, m_e=np.array([4.0, 0.0, 8.0, -2.0, 4.0, 1.0, 3.0]),
                      kappa=np.array([0.5, 1.0, 0.25, 2.0, 0.5, 0.8, 1.5]))
    w = np.linspace(0.5, 1.5, 10)
    out = run_gpu(gp, rho, g, parts, nsteps=10, weights=w)
    sim = run_oracle(gp, rho, g, parts, nsteps=10, weights=w)
    errs = compare(out, sim, gp, q0=parts["q"])
    check(errs, TOL[prec])


def test_fp32_wide_tile_staging_modes():
    """FP32 on a box whose x edge admits the row staging of the wide tile
    (72 = two tiles + 8 cells, so rows cross the periodic seam at both ends;
    30 rows = two tiles + 4), with noise, the mode drive and particles on the
    seam: every staging mode against the oracle, and all alike bit for bit."""
    gp = W.grid_params((72, 30, 14), kT=1e-3, wave_amp=2e-3, forcing="mode", zeta=0.3, seed=13, precision="fp32")
    rho, g = W.random_fields(gp, seed=5)
    parts = particles(6, (14, 30, 72), seed=4)
    parts["q"][0, 0] = 0.2     # on the x seam
    parts["q"][1, 0] = 71.9
    w = np.linspace(0.5, 1.5, 4)
    sim = run_oracle(gp, rho, g, parts, nsteps=4, weights=w, thermal_seed=3)
    runs = []
    for mode in ("thread", "bulk", "rows16"):
        out = run_gpu(gp, rho, g, parts, nsteps=4, weights=w, thermal_seed=3, tile=(32, 16), stage_copy=mode)
        assert out["stage_copy"] == mode
        check(compare(out, sim, gp, q0=parts["q"]), TOL["fp32"])
        runs.append(out)
    for other in runs[1:]:
        assert np.array_equal(runs[0]["rho"], other["rho"])
        for k in range(3):
            assert np.array_equal(runs[0]["g"][k], other["g"][k])
        for k in ("u", "q", "lam", "f_avg", "lam_avg"):
            assert np.array_equal(runs[0][k], other[k]), k


def test_particles_deterministic_single():
    """The single-particle standing wave in FP64 for 200 steps."""
    gp, parts, _ = W.single_particle_config(n=32, k_spring=0.25, mirror=True)
    rho, g = W.velocity_phase_wave_fields(gp)
    w = np.ones(200)
    out = run_gpu(gp, rho, g, parts, nsteps=200, weights=w)
    sim = run_oracle(gp, rho, g, parts, nsteps=200, weights=w)
    check(compare(out, sim, gp, q0=parts["q"]), TOL["fp64"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_thermal_initial_state(prec):
    gp = W.grid_params((24, 20, 17), kT=2e-3, wave_amp=1e-3, precision=prec)
    rho, g = W.standing_wave_fields(gp)
    out = run_gpu(gp, rho, g, nsteps=0, thermal_seed=42)
    sim = run_oracle(gp, rho, g, nsteps=0, thermal_seed=42)
    check(compare(out, sim, gp), 1e-13 if prec == "fp64" else 1e-6)


def test_many_particles_fp64_crowded():
    """Dense, strongly overlapping particles with a thermal start."""
    gp, parts = W.many_particle_config((24, 24, 24), 150, kT=1e-3, wave_amp=5e-3, seed=1)
    rho, g = W.standing_wave_fields(gp)
    out = run_gpu(gp, rho, g, parts, nsteps=4, thermal_seed=9)
    sim = run_oracle(gp, rho, g, parts, nsteps=4, thermal_seed=9)
    check(compare(out, sim, gp, q0=parts["q"]), TOL["fp64"])


def test_chunked_steps_equal_one_call():
    """ic_step(a) then ic_step(b) equals ic_step(a+b) bit for bit (graph reuse, weights offsets)."""
    gp = W.grid_params(16, kT=1e-3, wave_amp=1e-3, seed=3)
    rho, g = W.random_fields(gp, seed=1)
    parts = particles(3, (16, 16, 16), seed=2)
    w = np.arange(1, 8, dtype=float)
    a = run_gpu(gp, rho, g, parts, nsteps=7, weights=w)
    b = run_gpu(gp, rho, g, parts, nsteps=7, weights=w, chunks=[(0, 2), (2, 3), (3, 7)])
    assert np.array_equal(a["rho"], b["rho"])
    for k in range(3):
        assert np.array_equal(a["g"][k], b["g"][k])
    for k in ("u", "q", "lam", "f_avg", "lam_avg"):
        assert np.array_equal(a[k], b[k]), k
    assert a["a2"] == b["a2"]


@pytest.mark.parametrize("case", range(10))
def test_random_configurations(case):
    """Seeded random cases over the whole parameter space: grid edges from the
    minimum 6 up to 40 cells, both precisions, deterministic and thermal,
    every drive and wave axis, 0-12 particles anywhere (overlapping, on the
    periodic seam), tethered or free, any tiling; three steps against the
    oracle."""
    rng = np.random.default_rng(1000 + case)
    shape = tuple(int(x) for x in rng.integers(6, 41, 3))
    prec = ["fp64", "fp32"][case % 2]
    forcing = ["none", "mode", "plane"][int(rng.integers(3))]
    axis = int(rng.integers(3))
    kT = [0.0, 1e-3][int(rng.integers(2))]
    gp = W.grid_params(shape, kT=kT, wave_amp=float(rng.uniform(5e-4, 3e-3)), forcing=forcing, wave_axis=axis,
                       plane_index=int(rng.integers((shape[axis]))), zeta=float(rng.uniform(0.0, 1.0)),
                       seed=int(rng.integers(2 ** 62)), precision=prec, wave_phase=float(rng.uniform(0, 6.3)))
    rho, g = W.random_fields(gp, seed=case)
    npart = int(rng.integers(0, 13))
    parts = None
    if npart:
        L = np.array(shape, dtype=float)
        q = rng.uniform(0.0, 1.0, (npart, 3)) * L
        if npart > 2:
            q[1] = (q[0] + rng.uniform(-1.0, 1.0, 3)) % L     # overlapping kernels
            q[2, 0] = L[0] - 0.05                              # on the periodic seam
        parts = dict(q=q, m_e=rng.uniform(-2.0, 8.0, npart), kappa_ratio=rng.uniform(0.3, 2.0, npart),
                     k_spring=np.where(rng.uniform(size=npart) < 0.5, rng.uniform(0.1, 1.0, npart), 0.0))
    tile = ([32, 16][int(rng.integers(2))], int(rng.integers(8, 33)))
    out = run_gpu(gp, rho, g, parts, nsteps=3, weights=np.ones(3), thermal_seed=7 if kT else None, tile=tile)
    sim = run_oracle(gp, rho, g, parts, nsteps=3, weights=np.ones(3), thermal_seed=7 if kT else None)
    errs = compare(out, sim, gp, q0=None if parts is None else parts["q"])
    bad = {k: v for k, v in errs.items() if not v <= TOL[prec]}
    assert not bad, (shape, prec, forcing, axis, kT, npart, tile, errs)
