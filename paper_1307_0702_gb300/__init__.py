"""GB300-native inertial-coupling (IC) time step for acoustic forces on Brownian
particles (arXiv 1307.0702), as a CUDA library (libic.so, C ABI in include/ic.h)
with a thin Python binding.

    from paper_1307_0702_gb300 import Grid, workloads
    g = Grid(workloads.grid_params(32, wave_amp=1e-3))

``Grid`` needs the built library (``python -m paper_1307_0702_gb300.build``)
and a CUDA device; importing the package itself does neither.
"""
from . import workloads  # noqa: F401


def __getattr__(name):
    if name in ("Grid", "ICError", "Batch"):
        from . import ic
        return getattr(ic, name)
    raise AttributeError(name)
