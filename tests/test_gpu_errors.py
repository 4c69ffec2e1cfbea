"""Error paths and degenerate inputs through the C ABI, on the GPU.

Every case is detected on the host or by a device status flag that the host
reads after the step (no kernel faults, no waits): neighbour-list overflow
(the kernels never write past a list), a state driven non-finite by a CFL
number far above the SSP-RK3 limit, empty calls, invalid particles, foreign
or truncated checkpoints, and averages requested with zero weight.
"""
import numpy as np
import pytest

from paper_1307_0702_gb300 import _lib
from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def grid(n=16, **kw):
    from paper_1307_0702_gb300 import Grid

    gp = W.grid_params(n, **kw)
    g = Grid(gp)
    rho, gg = W.standing_wave_fields(gp)
    g.set_state(rho, gg)
    return g


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_neighbour_overflow_is_reported(prec):
    from paper_1307_0702_gb300 import ICError

    with grid(24, precision=prec) as g:
        rng = np.random.default_rng(1)
        q = 12.0 + rng.uniform(-2.0, 2.0, (80, 3))   # 80 particles within one cutoff box
        g.add_particles(q, 0.0, 1.0)
        g.step(1)
        with pytest.raises(ICError) as e:
            g.sync()
        assert e.value.status == _lib.IC_ERR_CAPACITY
        # the flag is cleared once reported
        g.sync()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_nonfinite_state_is_reported(prec):
    from paper_1307_0702_gb300 import ICError

    # c dt / h = 40: far beyond the SSP-RK3 stability limit of the sound waves
    with grid(16, precision=prec, dt=10.0, wave_amp=0.1) as g:
        g.step(60)
        with pytest.raises(ICError) as e:
            g.sync()
        assert e.value.status == _lib.IC_ERR_NONFINITE


def test_empty_calls_change_nothing():
    with grid(16, precision="fp64", kT=1e-3) as g:
        before = g.get_state()
        g.step(0)
        assert g.add_particles(np.zeros((0, 3)), np.zeros(0), np.ones(0)) == 0
        g.sync()
        after = g.get_state()
        assert np.array_equal(before[0], after[0])
        assert all(np.array_equal(a, b) for a, b in zip(before[1], after[1]))
        assert g.stats()[2] == 0


def test_invalid_particles_rejected():
    from paper_1307_0702_gb300 import ICError

    with grid(16, precision="fp32") as g:
        with pytest.raises(ICError) as e:
            g.add_particles(np.array([[1.0, 2.0, np.nan]]), 0.0, 1.0)
        assert e.value.status == _lib.IC_ERR_ARG
        with pytest.raises(ICError) as e:
            g.add_particles(np.array([[1.0, 2.0, 3.0]]), 0.0, 0.0)     # kappa_p / kappa_f must be > 0
        assert e.value.status == _lib.IC_ERR_ARG
        assert g.n_particles == 0


def test_foreign_and_truncated_checkpoints_rejected():
    from paper_1307_0702_gb300 import ICError

    with grid(16, precision="fp32") as a, grid(18, precision="fp32") as b, grid(16, precision="fp64") as c:
        a.add_particles(np.array([[4.0, 5.0, 6.0]]), 1.0, 0.5)
        blob = a.checkpoint()
        for other in (b, c):
            with pytest.raises(ICError) as e:
                other.restore(blob)
            assert e.value.status == _lib.IC_ERR_ARG
        with pytest.raises(ICError) as e:
            a.restore(blob[: len(blob) // 2])
        assert e.value.status == _lib.IC_ERR_ARG
        with pytest.raises(ICError):
            a.restore(b"not a checkpoint" * 8)


def test_average_without_weight_is_an_error():
    from paper_1307_0702_gb300 import ICError

    with grid(16, precision="fp32") as g:
        g.add_particles(np.array([[4.0, 5.0, 6.0]]), 1.0, 0.5, 0.3)
        g.step(3)                                  # no weights given
        with pytest.raises(ICError) as e:
            g.time_average()
        assert e.value.status == _lib.IC_ERR_STATE
        g.step(2, np.ones(2))
        f, lam, a2 = g.time_average()
        assert np.all(np.isfinite(f)) and a2 > 0
