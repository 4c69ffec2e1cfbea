"""The host schedule of the checkpointed reverse sweep (paper_1307_0702_gb300.
adjoint.Rollout) against a fake grid that only counts steps: every step of
the rollout is reversed exactly once, last first, from the state it was
recorded in, with its weight w_n / sum(w); with step tapes and without,
for several checkpoint intervals and rollout lengths."""
import numpy as np
import pytest

from paper_1307_0702_gb300.adjoint import Rollout


class FakeGrid:
    """Stands in for ``Grid``: the state is the step counter alone."""

    def __init__(self):
        self.params = {"kT": 0.0, "c": 4.0}
        self.step_n = 0
        self.recorded = None          # step recorded by step_record
        self.reversed = []            # (step, weight) of every reversed step
        self.forward_steps = 0
        self.sums = 0.0

    # state
    def adjoint_enable(self):
        pass

    def adjoint_reset(self, direction=None):
        self.reversed = []

    def new_snapshot(self):
        return {"step": None}

    def snapshot_save(self, buf):
        buf["step"] = self.step_n

    def snapshot_load(self, buf):
        assert buf["step"] is not None
        self.step_n = buf["step"]

    def step(self, n=1, weights=None):
        if weights is not None:
            self.sums += float(np.sum(weights))
        self.step_n += n
        self.forward_steps += n

    def time_average(self, reset=False):
        if self.sums == 0.0:
            raise RuntimeError("no sums")
        out = (np.zeros((1, 3)), None, None)
        if reset:
            self.sums = 0.0
        return out

    def objective(self, direction=None, reset=False):
        if self.sums == 0.0:
            raise RuntimeError("no sums")
        if reset:
            self.sums = 0.0
        return 0.0

    # one step recorded, then reversed
    def step_record(self):
        self.recorded = self.step_n
        self.step(1)

    def adjoint_step(self, w):
        self.reversed.append((self.recorded, w))

    def new_tape(self):
        return {"step": None}

    def step_record_tape(self, tape):
        tape["step"] = self.step_n
        self.step(1)

    def adjoint_step_tape(self, tape, w):
        self.reversed.append((tape["step"], w))

    def adjoint_read(self):
        return {"eps": np.zeros(1), "m_e": np.zeros(1), "A": 0.0}

    def adjoint_read_kappa(self):
        return np.zeros(1)


@pytest.mark.parametrize("tapes", [True, False])
@pytest.mark.parametrize("nsteps,K", [(1, 1), (7, 3), (12, 4), (10, 50), (50, 1)])
def test_every_step_reversed_once_last_first(tapes, nsteps, K):
    g = FakeGrid()
    roll = Rollout(g, [0.5], checkpoint_every=K, tapes=tapes)
    w = np.linspace(1.0, 2.0, nsteps)
    roll.forward(w)
    assert g.step_n == nsteps and g.forward_steps == nsteps
    roll.backward()
    W = float(np.sum(w))
    assert [s for s, _ in g.reversed] == list(range(nsteps - 1, -1, -1))
    assert np.allclose([x for _, x in g.reversed], w[::-1] / W, rtol=0, atol=1e-15)
    # forward passes: the sweep, then per segment a rerun (and with
    # snapshots, each step recorded again)
    reruns = g.forward_steps - nsteps
    assert reruns == (nsteps if tapes else nsteps + (nsteps - len(roll.checkpoints)))


def test_checkpoint_interval_must_be_positive():
    with pytest.raises(ValueError):
        Rollout(FakeGrid(), [0.5], checkpoint_every=0)


def test_thermal_box_is_refused():
    g = FakeGrid()
    g.params["kT"] = 1e-3
    with pytest.raises(ValueError):
        Rollout(g, [0.5])
