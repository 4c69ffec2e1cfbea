"""The C ABI boundary, checked without a GPU.

libic.so loads, exports every function declared in include/ic.h, the ctypes
mirror of the parameter structs matches the C layout (compiled here with gcc
from the header), and invalid parameters are rejected before any CUDA call.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ic.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1307_0702_gb300 import _lib, build

    build.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ic_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_calls():
    names = declared_functions()
    for required in ("ic_create_grid", "ic_add_particles", "ic_step", "ic_forces", "ic_time_average"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1307_0702_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ic_[a-z0-9_]+)", out))
    names = declared_functions()
    assert set(names) <= exported, set(names) - exported
    assert set(names) == set(_lib.SIGNATURES), "ctypes signatures must mirror the header"
    for n in names:
        assert getattr(lib, n) is not None


def test_struct_layout_matches_c(tmp_path):
    from paper_1307_0702_gb300 import _lib

    fields = [f for f, _ in _lib.GridParams._fields_]
    prog = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){",
            'printf("%zu\\n", sizeof(ic_grid_params));',
            'printf("%zu\\n", sizeof(ic_views));']
    prog += [f'printf("%zu\\n", offsetof(ic_grid_params, {f}));' for f in fields]
    prog += [f'printf("%zu\\n", offsetof(ic_views, {f}));' for f, _ in _lib.Views._fields_]
    prog += ["return 0;}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(c)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(_lib.GridParams)
    assert vals[1] == ctypes.sizeof(_lib.Views)
    offs = vals[2:2 + len(fields)]
    assert offs == [getattr(_lib.GridParams, f).offset for f in fields]
    voffs = vals[2 + len(fields):]
    assert voffs == [getattr(_lib.Views, f).offset for f, _ in _lib.Views._fields_]


def test_invalid_parameters_rejected_without_cuda(lib):
    from paper_1307_0702_gb300 import _lib

    gp = _lib.GridParams(nx=4, ny=32, nz=32, h=1.0, rho0=1.0, c=4.0, dt=0.025, wave_nlambda=1)
    ctx = ctypes.c_void_p()
    assert lib.ic_create_grid(ctypes.byref(gp), ctypes.byref(ctx)) == _lib.IC_ERR_ARG
    gp.nx = 32
    gp.c = -1.0
    assert lib.ic_create_grid(ctypes.byref(gp), ctypes.byref(ctx)) == _lib.IC_ERR_ARG
    gp.c = 4.0
    gp.precision = 7
    assert lib.ic_create_grid(ctypes.byref(gp), ctypes.byref(ctx)) == _lib.IC_ERR_ARG
    gp.precision = 0
    gp.plane_index = 40
    assert lib.ic_create_grid(ctypes.byref(gp), ctypes.byref(ctx)) == _lib.IC_ERR_ARG
    assert lib.ic_step(None, 1, None) == _lib.IC_ERR_ARG
    assert lib.ic_forces_async(None, 0) == _lib.IC_ERR_ARG
    assert lib.ic_forces_collect(None, 0, None) == _lib.IC_ERR_ARG
    assert lib.ic_set_stage_copy(None, 0) == _lib.IC_ERR_ARG
    assert lib.ic_philox4x32_10(-1, None, None) == _lib.IC_ERR_ARG
    assert lib.ic_philox4x32_10(3, None, None) == _lib.IC_ERR_ARG
    assert lib.ic_philox4x32_10(0, None, None) == _lib.IC_OK
    assert lib.ic_last_error(None) == b"null context"


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1307_0702_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing.so is missing at"):
        _lib.load()
