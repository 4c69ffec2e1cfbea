"""The bounded waits of the stage kernels' bulk staging, made to run out: with
IC_STAGE_STALL_TEST=1 each CTA's mbarriers expect one arrival that no thread
makes, so every wait gives up after about a second, the CTA flags the status
word and leaves (no copy is left in flight: the rows all land).  The next
status read returns IC_ERR_TIMEOUT, and the same context then steps exactly
as a fresh one.  Covered: the wide tile's two row-staging modes and the
whole-row kernel's plane rings."""
import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["bulk", "rows16", "whole_rows"])
def test_row_staging_wait_runs_out_and_reports(mode, monkeypatch):
    from paper_1307_0702_gb300 import Grid, ICError

    # 40 x 13 x 6: one wide-tile column pair, two CTAs, so the run-outs take seconds
    gp = W.grid_params((40, 13, 6), kT=0.0, wave_amp=0.0, forcing="none", precision="fp32")
    rho, g = W.random_fields(gp, seed=1)
    monkeypatch.setenv("IC_STAGE_STALL_TEST", "1")
    def setup(grid):
        if mode == "whole_rows":
            grid.set_tile(0, 8)              # (also drops step graphs captured before)
            assert grid.tile()[0] == gp["nx"]
        else:
            grid.set_tile(32, 8)
            grid.set_stage_copy(mode)         # (also drops step graphs captured before)
            assert grid.stage_copy() == mode

    with Grid(gp) as grid:
        setup(grid)
        grid.set_state(rho, g)
        grid.step(1)
        with pytest.raises(ICError) as e:
            grid.sync()
        assert e.value.status == -5          # IC_ERR_TIMEOUT
        monkeypatch.delenv("IC_STAGE_STALL_TEST")
        setup(grid)                           # drops the step graphs captured with the stall
        grid.set_state(rho, g)
        grid.step(2)
        grid.sync()
        after = grid.get_state()
    with Grid(gp) as fresh:
        setup(fresh)
        fresh.set_state(rho, g)
        fresh.step(2)
        ref = fresh.get_state()
    assert np.array_equal(after[0], ref[0])
    for a, b in zip(after[1], ref[1]):
        assert np.array_equal(a, b)
