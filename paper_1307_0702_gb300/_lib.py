"""ctypes declarations of the C ABI in include/ic.h (argument marshalling only)."""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
# IC_LIBRARY=bounds selects the index-checking debug build (libic_bounds.so)
LIB_PATH = os.path.join(HERE, "libic_bounds.so" if os.environ.get("IC_LIBRARY") == "bounds" else "libic.so")

IC_OK, IC_ERR_ARG, IC_ERR_CUDA, IC_ERR_OOM, IC_ERR_NONFINITE, IC_ERR_TIMEOUT, IC_ERR_STATE, IC_ERR_CAPACITY = (
    0, -1, -2, -3, -4, -5, -6, -7)
IC_FP64, IC_FP32 = 0, 1
IC_FORCE_NONE, IC_FORCE_MODE, IC_FORCE_PLANE = 0, 1, 2

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p)


class GridParams(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int), ("nz", c_int),
        ("h", c_double), ("rho0", c_double), ("c", c_double), ("eta", c_double), ("zeta", c_double),
        ("kT", c_double), ("dt", c_double),
        ("seed", c_uint64), ("box", c_uint32),
        ("precision", c_int), ("forcing", c_int), ("wave_axis", c_int),
        ("wave_amp", c_double), ("wave_nlambda", c_int), ("plane_index", c_int), ("wave_phase", c_double),
        ("stream", c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", c_void_p),
    ]


class Views(ctypes.Structure):
    _fields_ = [("drho", c_void_p), ("gx", c_void_p), ("gy", c_void_p), ("gz", c_void_p),
                ("precision", c_int), ("n_particles", c_int), ("q", c_void_p)]


PD = POINTER(c_double)

# name -> (restype, argtypes); every function declared in include/ic.h
SIGNATURES = {
    "ic_create_grid": (c_int, [POINTER(GridParams), POINTER(c_void_p)]),
    "ic_set_state": (c_int, [c_void_p, PD, PD, PD, PD]),
    "ic_get_state": (c_int, [c_void_p, PD, PD, PD, PD]),
    "ic_init_thermal": (c_int, [c_void_p, c_uint64, c_int]),
    "ic_add_particles": (c_int, [c_void_p, c_int, PD, PD, PD, PD, PD, POINTER(c_int)]),
    "ic_step": (c_int, [c_void_p, c_int, PD]),
    "ic_forces": (c_int, [c_void_p, PD, PD, PD]),
    "ic_particle_density": (c_int, [c_void_p, PD]),
    "ic_time_average": (c_int, [c_void_p, PD, PD, PD, c_int]),
    "ic_stats": (c_int, [c_void_p, PD, PD, POINTER(c_int64)]),
    "ic_neighbour_rebuilds": (c_int, [c_void_p, POINTER(c_int64)]),
    "ic_bounds_check_build": (c_int, []),
    "ic_bounds_selftest": (c_int, []),
    "ic_objective": (c_int, [c_void_p, PD, PD, c_int]),
    "ic_adjoint_read_kappa": (c_int, [c_void_p, PD]),
    "ic_sync": (c_int, [c_void_p]),
    "ic_checkpoint": (c_int, [c_void_p, c_void_p, POINTER(c_size_t)]),
    "ic_restore": (c_int, [c_void_p, c_void_p, c_size_t]),
    "ic_device_views": (c_int, [c_void_p, POINTER(Views)]),
    "ic_batch_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p)]),
    "ic_batch_step": (c_int, [c_void_p, c_int, PD]),
    "ic_batch_destroy": (None, [c_void_p]),
    "ic_set_tile": (c_int, [c_void_p, c_int, c_int]),
    "ic_get_tile": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "ic_set_stage_copy": (c_int, [c_void_p, c_int]),
    "ic_forces_async": (c_int, [c_void_p, c_int]),
    "ic_philox4x32_10": (c_int, [c_int, POINTER(c_uint32), POINTER(c_uint32)]),
    "ic_fma64_rate": (c_int, [c_int, PD, PD]),
    "ic_forces_collect": (c_int, [c_void_p, c_int, PD]),
    "ic_get_stage_copy": (c_int, [c_void_p, POINTER(c_int)]),
    "ic_autotune": (c_int, [c_void_p, c_int, POINTER(c_int)]),
    "ic_batch_autotune": (c_int, [c_void_p, c_int]),
    "ic_profile": (c_int, [c_void_p, c_int]),
    "ic_profile_read": (c_int, [c_void_p, PD, POINTER(c_int64), c_int]),
    "ic_fluid_step_noalloc": (c_int, [POINTER(GridParams), POINTER(c_void_p), POINTER(c_void_p), c_int64]),
    "ic_adjoint_enable": (c_int, [c_void_p]),
    "ic_adjoint_reset": (c_int, [c_void_p, PD]),
    "ic_step_record": (c_int, [c_void_p]),
    "ic_adjoint_step": (c_int, [c_void_p, c_double]),
    "ic_adjoint_read": (c_int, [c_void_p, PD, PD, PD, PD, PD, PD, PD, PD, PD]),
    "ic_tape_size": (c_int, [c_void_p, POINTER(c_size_t)]),
    "ic_step_record_tape": (c_int, [c_void_p, c_void_p]),
    "ic_adjoint_step_tape": (c_int, [c_void_p, c_void_p, c_double]),
    "ic_snapshot_size": (c_int, [c_void_p, POINTER(c_size_t)]),
    "ic_snapshot_save": (c_int, [c_void_p, c_void_p]),
    "ic_snapshot_load": (c_int, [c_void_p, c_void_p]),
    "ic_last_error": (c_char_p, [c_void_p]),
    "ic_destroy": (None, [c_void_p]),
}

_lib = None


def load():
    """Load libic.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{os.path.basename(LIB_PATH)} is missing at {LIB_PATH}: build it with "
                "`python -m paper_1307_0702_gb300.build` (add --bounds-check for libic_bounds.so; "
                "needs nvcc for sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
