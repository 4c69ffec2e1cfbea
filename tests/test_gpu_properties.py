"""Properties of the GPU path that hold at any size, and the full-size check.

* two runs of the same seeded input are bit-identical (no atomics, fixed
  reduction orders), and resuming from a checkpoint reproduces the
  uninterrupted run bit for bit;
* total momentum h^3 sum g + sum m_e u is conserved to rounding with F = 0,
  and changes by dt sum F with tethers;
* at the benchmark's size (128^3 FP32, 1e4 particles) one step matches the
  oracle on every cell and particle to FP32 accuracy.
"""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W
from pairs import compare, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def small_case(prec="fp64", kT=1e-3, n=20, npart=12, k_spring=0.0):
    gp, parts = W.many_particle_config(n, npart, kT=kT, wave_amp=2e-3, seed=4, precision=prec, k_spring=k_spring)
    rho, g = W.standing_wave_fields(gp)
    return gp, rho, g, parts


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bitwise_reproducible(prec):
    gp, rho, g, parts = small_case(prec)
    a = run_gpu(gp, rho, g, parts, nsteps=12, thermal_seed=3, weights=np.ones(12))
    b = run_gpu(gp, rho, g, parts, nsteps=12, thermal_seed=3, weights=np.ones(12))
    for k in ("rho", "u", "q", "lam", "f_avg"):
        assert np.array_equal(a[k], b[k]), k
    for c in range(3):
        assert np.array_equal(a["g"][c], b["g"][c])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_resume_bit_exact(prec):
    from paper_1307_0702_gb300 import Grid

    gp, rho, g, parts = small_case(prec, k_spring=0.5)
    w = np.linspace(0.1, 1.0, 16)
    with Grid(gp) as ref:
        ref.set_state(rho, g)
        ref.init_thermal(5)
        ref.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
        ref.step(16, w)
        r_rho, r_g = ref.get_state()
        r_f = ref.forces()
        r_avg = ref.time_average()
    with Grid(gp) as first:
        first.set_state(rho, g)
        first.init_thermal(5)
        first.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
        first.step(9, w[:9])
        blob = first.checkpoint()
    with Grid(gp) as second:
        second.restore(blob)
        second.step(7, w[9:])
        s_rho, s_g = second.get_state()
        s_f = second.forces()
        s_avg = second.time_average()
        assert second.stats()[2] == 16
    assert np.array_equal(r_rho, s_rho)
    for c in range(3):
        assert np.array_equal(r_g[c], s_g[c])
    for x, y in zip(r_f, s_f):
        assert np.array_equal(x, y)
    assert np.array_equal(r_avg[0], s_avg[0]) and np.array_equal(r_avg[1], s_avg[1]) and r_avg[2] == s_avg[2]


def test_momentum_conserved_fp64():
    from paper_1307_0702_gb300 import Grid

    gp, rho, g, parts = small_case("fp64", npart=30)
    gp["forcing"] = "none"
    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.init_thermal(1)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"])
        p0 = grid.stats()[0]
        grid.step(25)
        p1 = grid.stats()[0]
    assert np.max(np.abs(p1 - p0)) < 1e-13


def test_full_size_one_step_fp32_against_oracle():
    """Benchmark workload (128^3 FP32, 1e4 particles, thermal start): one step, every cell."""
    gp, parts = W.large_box_config()
    rho, g = W.standing_wave_fields(gp)
    out = run_gpu(gp, rho, g, parts, nsteps=1, thermal_seed=1000)
    sim = run_oracle(gp, rho, g, parts, nsteps=1, thermal_seed=1000)
    errs = compare(out, sim, gp, q0=parts["q"])
    bad = {k: v for k, v in errs.items() if not v <= 1e-4}
    assert not bad, errs


def test_long_run_of_the_benchmark_box():
    """20 000 steps of the benchmark box (128^3 FP32, 1e4 free particles,
    kT = 1e-3, mode drive): the particles diffuse past a quarter skin, so the
    neighbour lists are rebuilt on the way; no device error is raised, the
    state stays finite and the total momentum h^3 sum g + sum m_e u (the
    particles start with the local fluid velocity, so it is not zero) is
    conserved to rounding level by every term of the step."""
    from paper_1307_0702_gb300 import Grid

    gp, parts = W.large_box_config()
    rho, g = W.standing_wave_fields(gp)
    with Grid(gp) as grid:
        grid.set_state(rho, g)
        grid.init_thermal(1000)
        grid.add_particles(parts["q"], parts["m_e"], parts["kappa_ratio"], parts["k_spring"])
        q0 = grid.forces()[2].copy()
        p0 = grid.stats()[0]
        for _ in range(4):
            grid.step(5000)
            grid.sync()
        p, a, n = grid.stats()
        rho_n, g_n = grid.get_state()
        q1 = grid.forces()[2]
    assert n == 20000
    assert np.all(np.isfinite(rho_n)) and all(np.all(np.isfinite(x)) for x in g_n)
    scale = sum(np.sum(np.abs(x)) for x in g_n)
    assert np.all(np.abs(p - p0) < 1e-6 * scale), (p, p0, scale)
    L = 128.0
    d = q1 - q0
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) > 0.25          # some particles moved past a quarter skin (a rebuild)
    assert abs(a) < 2e-3                     # the driven mode stays at its amplitude scale
