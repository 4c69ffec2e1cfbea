"""In-tree build of libic.so (CUDA, sm_103a) with nvcc.

    python -m paper_1307_0702_gb300.build [--force] [--bounds-check]

compiles the translation units of ``csrc/`` in parallel into ``_build/`` and
links ``libic.so`` next to this file.  No CMake, one -gencode, static cudart.
``--bounds-check`` builds the index-checking debug variant instead
(-DIC_BOUNDS_CHECK, objects in ``_build_bounds/``, ``libic_bounds.so``), which
the package loads when IC_LIBRARY=bounds is set.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
VARIANTS = {False: ("_build", "libic.so", []), True: ("_build_bounds", "libic_bounds.so", ["-DIC_BOUNDS_CHECK"])}
SOURCES = ["ic_capi.cu", "ic_fluid.cu", "ic_stage_rows.cu", "ic_particles.cu", "ic_noalloc.cu", "ic_adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: libic needs the CUDA toolkit to build")
    return path


def _compile(src, build_dir, extra):
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    log = os.path.join(build_dir, os.path.splitext(src)[0] + ".log")
    cmd = [nvcc(), *FLAGS, *extra, *ARCH, "-c", os.path.join(CSRC, src), "-o", obj]
    with open(log, "w") as f:
        r = subprocess.run(cmd, stdout=f, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        with open(log) as f:
            raise RuntimeError(f"nvcc failed on {src}:\n{f.read()[-4000:]}")
    return obj


def build(force=False, bounds_check=False):
    """Compile and link libic.so (or libic_bounds.so); returns its path."""
    sub, name, extra = VARIANTS[bool(bounds_check)]
    BUILD, LIB = os.path.join(HERE, sub), os.path.join(HERE, name)
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [
        os.path.join(HERE, "..", "include", "ic.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) > max(os.path.getmtime(d) for d in deps)):
        return LIB
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda src: _compile(src, BUILD, extra), SOURCES))
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc(), "-shared", *ARCH, "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, bounds_check="--bounds-check" in sys.argv))
