"""ic_fluid_step_noalloc against ic_step, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device
memory when they step the fluid (inside another framework's stream capture,
or with all device memory reserved by their own pool): its scratch is a fixed
static device array.  It runs the same RK3 stage kernels as ic_step, so on a
box without particles two consecutive calls must reproduce two ic_step steps
to the parity tolerances (1e-11 FP64, 1e-4 FP32, normwise per field).

This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_1307_0702_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-4}


def c_params(gp, stream_handle):
    from paper_1307_0702_gb300 import _lib

    p = _lib.GridParams()
    for k in ("nx", "ny", "nz", "wave_axis", "plane_index"):
        setattr(p, k, int(gp[k]))
    for k in ("h", "rho0", "c", "eta", "zeta", "kT", "dt", "wave_amp", "wave_phase"):
        setattr(p, k, float(gp[k]))
    p.wave_nlambda = int(gp["wave_nlambda"])
    p.seed = int(gp["seed"])
    p.box = 0
    p.precision = {"fp64": _lib.IC_FP64, "fp32": _lib.IC_FP32}[gp["precision"]]
    p.forcing = {"none": _lib.IC_FORCE_NONE, "mode": _lib.IC_FORCE_MODE, "plane": _lib.IC_FORCE_PLANE}[gp["forcing"]]
    p.stream = stream_handle
    return p


def rel(a, b):
    scale = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0)


@pytest.mark.parametrize("shape,prec", [((20, 18, 22), "fp64"), ((20, 18, 22), "fp32"), ((32, 32, 32), "fp64")])
def test_noalloc_step_matches_ic_step_twice(shape, prec):
    """Two calls against two ic_step steps; 32^3 FP64 (the single-particle
    box's grid) is IC_NOALLOC_MAX_CELLS, the largest the scratch holds."""
    import torch

    from paper_1307_0702_gb300 import Grid, _lib

    lib = _lib.load()
    gp = W.grid_params(shape, kT=1e-3, wave_amp=2e-3, forcing="mode", zeta=0.3, seed=9, precision=prec)
    rho, g = W.random_fields(gp, seed=2)
    # reference: the context API, two steps
    ref = []
    with Grid(gp) as grid:
        grid.set_state(rho, g)
        for _ in range(2):
            grid.step(1)
            r, gg = grid.get_state()
            ref.append([r - gp["rho0"]] + gg)

    dt = torch.float64 if prec == "fp64" else torch.float32
    fields = [rho - gp["rho0"]] + g
    state = [torch.tensor(np.ascontiguousarray(f), dtype=dt, device="cuda") for f in fields]
    stream = torch.cuda.current_stream()
    params = c_params(gp, stream.cuda_stream)
    for n in range(2):
        out = [torch.empty_like(t) for t in state]
        ins = (ctypes.c_void_p * 4)(*[t.data_ptr() for t in state])
        outs = (ctypes.c_void_p * 4)(*[t.data_ptr() for t in out])
        st = lib.ic_fluid_step_noalloc(ctypes.byref(params), ins, outs, n)
        assert st == _lib.IC_OK
        torch.cuda.synchronize()
        got = [t.double().cpu().numpy() for t in out]
        for j in range(4):
            assert rel(got[j], ref[n][j]) <= TOL[prec], (n, j, rel(got[j], ref[n][j]))
        state = out


def test_noalloc_rejects_oversized_and_aliased():
    import torch

    from paper_1307_0702_gb300 import _lib

    lib = _lib.load()
    gp = W.grid_params(40, precision="fp32")          # 64000 cells > IC_NOALLOC_MAX_CELLS
    params = c_params(gp, torch.cuda.current_stream().cuda_stream)
    t = [torch.zeros(40 ** 3, device="cuda") for _ in range(8)]
    ins = (ctypes.c_void_p * 4)(*[x.data_ptr() for x in t[:4]])
    outs = (ctypes.c_void_p * 4)(*[x.data_ptr() for x in t[4:]])
    assert lib.ic_fluid_step_noalloc(ctypes.byref(params), ins, outs, 0) == _lib.IC_ERR_CAPACITY
    gp = W.grid_params(16, precision="fp32")
    params = c_params(gp, torch.cuda.current_stream().cuda_stream)
    assert lib.ic_fluid_step_noalloc(ctypes.byref(params), ins, ins, 0) == _lib.IC_ERR_ARG
    # partial overlaps: an output 8 bytes into an input, two outputs overlapping
    shifted = (ctypes.c_void_p * 4)(t[0].data_ptr() + 8, *[x.data_ptr() for x in t[5:8]])
    assert lib.ic_fluid_step_noalloc(ctypes.byref(params), ins, shifted, 0) == _lib.IC_ERR_ARG
    crossed = (ctypes.c_void_p * 4)(t[4].data_ptr(), t[4].data_ptr() + 4 * (16 ** 3 - 1), t[6].data_ptr(),
                                    t[7].data_ptr())
    assert lib.ic_fluid_step_noalloc(ctypes.byref(params), ins, crossed, 0) == _lib.IC_ERR_ARG
    # adjacent but disjoint arrays are accepted: the four outputs back to back in one buffer
    flat = torch.zeros(4 * 16 ** 3, device="cuda")
    packed = (ctypes.c_void_p * 4)(*[flat.data_ptr() + 4 * 16 ** 3 * j for j in range(4)])
    assert lib.ic_fluid_step_noalloc(ctypes.byref(params), ins, packed, 0) == _lib.IC_OK
    torch.cuda.synchronize()
