"""Python binding of libic: the C calls of include/ic.h with numpy marshalling.

Every step of the method runs in the CUDA library; this module only converts
arguments.  Device memory comes from PyTorch's caching allocator and work is
ordered on a torch CUDA stream.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import IC_FORCE_MODE, IC_FORCE_NONE, IC_FORCE_PLANE, IC_FP32, IC_FP64

_FORCING = {"none": IC_FORCE_NONE, "mode": IC_FORCE_MODE, "plane": IC_FORCE_PLANE}
_PRECISION = {"fp64": IC_FP64, "fp32": IC_FP32}


class ICError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libic error {status}: {message}")
        self.status = status


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_lib.PD)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def philox4x32_10(ctr_key):
    """The library's Philox4x32-10 evaluated on the current device:
    ctr_key (n, 6) uint32 rows (ctr0..ctr3, key0, key1) -> (n, 4) uint32."""
    lib = _lib.load()
    a = np.ascontiguousarray(np.asarray(ctr_key, dtype=np.uint32).reshape(-1, 6))
    out = np.empty((a.shape[0], 4), dtype=np.uint32)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    st = lib.ic_philox4x32_10(a.shape[0], a.ctypes.data_as(u32), out.ctypes.data_as(u32))
    if st != 0:
        raise ICError(st, "ic_philox4x32_10 failed")
    return out


class Grid:
    """One simulation box (an ic_ctx).

    params: dict with the keys of ``workloads.grid_params`` (nx, ny, nz, h,
    rho0, c, eta, zeta, kT, dt, seed, forcing, wave_axis, wave_amp,
    wave_nlambda, plane_index, wave_phase, precision) plus optional ``box``.
    """

    def __init__(self, params, device=None, stream=None, allocator="torch"):
        import torch

        self._lib = _lib.load()
        self.params = dict(params)
        self.shape = (int(params["nz"]), int(params["ny"]), int(params["nx"]))
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        gp = _lib.GridParams()
        for k in ("nx", "ny", "nz", "wave_axis", "wave_nlambda", "plane_index"):
            setattr(gp, k, int(params.get(k, 0)))
        for k in ("h", "rho0", "c", "eta", "zeta", "kT", "dt", "wave_amp", "wave_phase"):
            setattr(gp, k, float(params.get(k, 0.0)))
        gp.wave_nlambda = int(params.get("wave_nlambda", 1))
        gp.seed = int(params.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
        gp.box = int(params.get("box", 0))
        gp.precision = _PRECISION[params.get("precision", "fp64")]
        gp.forcing = _FORCING[params.get("forcing", "none")]
        gp.stream = self.stream.cuda_stream
        if allocator == "torch":
            dev, strm = self.device.index, self.stream

            def _alloc(nbytes, _ctx):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)

            def _free(ptr, _nbytes, _ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = _lib.ALLOC_FN(_alloc)
            self._free_cb = _lib.FREE_FN(_free)
            gp.alloc, gp.free = self._alloc_cb, self._free_cb
        self._gp = gp
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self._lib.ic_create_grid(ctypes.byref(gp), ctypes.byref(self._ctx))
        if st != 0:
            raise ICError(st, "ic_create_grid rejected the parameters" if st == -1 else "ic_create_grid failed")
        self.n_particles = 0

    # ------------------------------------------------------------------ utils
    def _check(self, st):
        if st != 0:
            msg = self._lib.ic_last_error(self._ctx)
            raise ICError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.ic_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ state
    def set_state(self, rho, g=None):
        rho = _f64(rho, self.shape)
        g = [None] * 3 if g is None else [_f64(a, self.shape) for a in g]
        self._check(self._lib.ic_set_state(self._ctx, _ptr(rho), _ptr(g[0]), _ptr(g[1]), _ptr(g[2])))

    def get_state(self):
        rho = np.empty(self.shape)
        g = [np.empty(self.shape) for _ in range(3)]
        self._check(self._lib.ic_get_state(self._ctx, _ptr(rho), _ptr(g[0]), _ptr(g[1]), _ptr(g[2])))
        return rho, g

    def init_thermal(self, seed, add=True):
        self._check(self._lib.ic_init_thermal(self._ctx, int(seed) & 0xFFFFFFFFFFFFFFFF, 1 if add else 0))

    def add_particles(self, q, m_e, kappa_ratio, k_spring=None, u=None):
        q = _f64(q).reshape(-1, 3)
        n = q.shape[0]
        m_e = _f64(np.broadcast_to(np.asarray(m_e, float), (n,)))
        kr = _f64(np.broadcast_to(np.asarray(kappa_ratio, float), (n,)))
        ks = None if k_spring is None else _f64(np.broadcast_to(np.asarray(k_spring, float), (n,)))
        u = None if u is None else _f64(u).reshape(n, 3)
        first = ctypes.c_int()
        self._check(self._lib.ic_add_particles(self._ctx, n, _ptr(q), _ptr(u), _ptr(m_e), _ptr(kr), _ptr(ks),
                                               ctypes.byref(first)))
        self.n_particles += n
        return first.value

    def step(self, nsteps=1, weights=None):
        w = None if weights is None else _f64(weights)
        if w is not None and w.size != nsteps:
            raise ValueError("weights must have nsteps entries")
        self._check(self._lib.ic_step(self._ctx, int(nsteps), _ptr(w)))

    def sync(self):
        self._check(self._lib.ic_sync(self._ctx))

    def forces(self, out=None):
        """(lambda, u, q), each (n, 3); ``out`` may give preallocated arrays."""
        n = self.n_particles
        lam, u, q = out if out is not None else (np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3)))
        self._check(self._lib.ic_forces(self._ctx, _ptr(lam), _ptr(u), _ptr(q)))
        return lam, u, q

    def forces_async(self, slot):
        """Queue the read-back of this step's lambda into pinned slot 0 or 1 (no synchronisation)."""
        self._check(self._lib.ic_forces_async(self._ctx, int(slot)))

    def forces_collect(self, slot, out=None):
        """Wait for the slot's queued read-back alone; lambda (n, 3) (into ``out`` if given)."""
        lam = out if out is not None else np.empty((self.n_particles, 3))
        self._check(self._lib.ic_forces_collect(self._ctx, int(slot), _ptr(lam)))
        return lam

    def particle_density(self):
        """J rho^{n+1} per particle (n,)."""
        out = np.empty(self.n_particles)
        self._check(self._lib.ic_particle_density(self._ctx, _ptr(out)))
        return out

    def time_average(self, reset=False):
        """(<F_spring>_w, <lambda>_w, <A^2>_w)."""
        n = self.n_particles
        f, lam, a2 = np.empty((n, 3)), np.empty((n, 3)), ctypes.c_double()
        self._check(self._lib.ic_time_average(self._ctx, _ptr(f), _ptr(lam), ctypes.byref(a2), 1 if reset else 0))
        return f, lam, a2.value

    def objective(self, direction=None, reset=False):
        """Phi = sum_p d_p . <F_p>_w from the context's sums (ic_objective)."""
        phi = ctypes.c_double()
        d = None if direction is None else np.ascontiguousarray(direction, dtype=np.float64).reshape(-1, 3)
        self._check(self._lib.ic_objective(self._ctx, _ptr(d), ctypes.byref(phi), 1 if reset else 0))
        return phi.value

    def adjoint_read_kappa(self):
        """dPhi / d(kappa_p / kappa_f) of every particle (ic_adjoint_read_kappa)."""
        out = np.empty(self.n_particles)
        self._check(self._lib.ic_adjoint_read_kappa(self._ctx, _ptr(out)))
        return out

    def stats(self):
        """(total momentum (3,), driven-mode amplitude A, step)."""
        p = np.empty(3)
        a = ctypes.c_double()
        s = ctypes.c_int64()
        self._check(self._lib.ic_stats(self._ctx, _ptr(p), ctypes.byref(a), ctypes.byref(s)))
        return p, a.value, s.value

    def neighbour_rebuilds(self):
        """Neighbour-list rebuilds made so far (counting sort into cell bins)."""
        n = ctypes.c_int64()
        self._check(self._lib.ic_neighbour_rebuilds(self._ctx, ctypes.byref(n)))
        return n.value

    def checkpoint(self):
        size = ctypes.c_size_t()
        self._check(self._lib.ic_checkpoint(self._ctx, None, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        self._check(self._lib.ic_checkpoint(self._ctx, buf, ctypes.byref(size)))
        return buf.raw[:size.value]

    def restore(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self._lib.ic_restore(self._ctx, buf, len(blob)))
        self.n_particles = int(np.frombuffer(blob[28:32], dtype=np.int32)[0])

    # ---------------------------------------------------------------- adjoint
    def adjoint_enable(self):
        """Allocate the tape and adjoint fields (deterministic boxes only)."""
        self._check(self._lib.ic_adjoint_enable(self._ctx))

    def adjoint_reset(self, direction=None):
        """Zero the adjoint and gradients; direction (n, 3) of the objective (default x)."""
        d = None if direction is None else _f64(direction).reshape(self.n_particles, 3)
        self._check(self._lib.ic_adjoint_reset(self._ctx, _ptr(d)))

    def step_record(self):
        """One step forward that keeps the tape of its reverse sweep."""
        self._check(self._lib.ic_step_record(self._ctx))

    def adjoint_step(self, weight):
        """Reverse the recorded step, adding weight * sum_p d_p . F_p to the objective."""
        self._check(self._lib.ic_adjoint_step(self._ctx, float(weight)))

    def adjoint_read(self):
        """Gradients and state adjoints: dict m_e, eps (n,), A, rho, g (3 fields), q, u (n, 3)."""
        n = self.n_particles
        me, eps, A = np.empty(n), np.empty(n), np.empty(1)
        rho = np.empty(self.shape)
        g = [np.empty(self.shape) for _ in range(3)]
        q, u = np.empty((n, 3)), np.empty((n, 3))
        self._check(self._lib.ic_adjoint_read(self._ctx, _ptr(me), _ptr(eps), _ptr(A), _ptr(rho), _ptr(g[0]),
                                              _ptr(g[1]), _ptr(g[2]), _ptr(q), _ptr(u)))
        return dict(m_e=me, eps=eps, A=float(A[0]), rho=rho, g=g, q=q, u=u)

    def tape_size(self):
        size = ctypes.c_size_t()
        self._check(self._lib.ic_tape_size(self._ctx, ctypes.byref(size)))
        return size.value

    def new_tape(self):
        """A device buffer (torch uint8 tensor) for the tape of one step."""
        import torch

        return torch.empty(self.tape_size(), dtype=torch.uint8, device=self.device)

    def step_record_tape(self, buf):
        """One step forward, its reverse-sweep inputs copied into buf."""
        self._check(self._lib.ic_step_record_tape(self._ctx, ctypes.c_void_p(buf.data_ptr())))

    def adjoint_step_tape(self, buf, weight):
        """Reverse the step taped in buf, adding weight * sum_p d_p . F_p to the objective."""
        self._check(self._lib.ic_adjoint_step_tape(self._ctx, ctypes.c_void_p(buf.data_ptr()), float(weight)))

    def snapshot_size(self):
        size = ctypes.c_size_t()
        self._check(self._lib.ic_snapshot_size(self._ctx, ctypes.byref(size)))
        return size.value

    def new_snapshot(self):
        """A device buffer (torch uint8 tensor) for one snapshot of this box."""
        import torch

        return torch.empty(self.snapshot_size(), dtype=torch.uint8, device=self.device)

    def snapshot_save(self, buf):
        """Enqueue a device copy of the state (fields, q, u, step) into buf."""
        self._check(self._lib.ic_snapshot_save(self._ctx, ctypes.c_void_p(buf.data_ptr())))

    def snapshot_load(self, buf):
        """Restore a state saved by snapshot_save."""
        self._check(self._lib.ic_snapshot_load(self._ctx, ctypes.c_void_p(buf.data_ptr())))

    def set_tile(self, tile_x, zchunk):
        """Stage-kernel tiling: tile_x 32 or 16 (column tiles) or 0 (bands of whole x
        rows, FP32 with nx a multiple of 4 up to 128), zchunk >= 8 planes."""
        self._check(self._lib.ic_set_tile(self._ctx, int(tile_x), int(zchunk)))

    def tile(self):
        """(tile_x, tile_y, zchunk) of the stage kernel."""
        t = [ctypes.c_int() for _ in range(3)]
        self._check(self._lib.ic_get_tile(self._ctx, *[ctypes.byref(x) for x in t]))
        return tuple(x.value for x in t)

    STAGE_COPY = ("thread", "bulk", "rows16")

    def set_stage_copy(self, mode):
        """FP32 wide-tile stage loads: "thread" (per-thread 4-byte copies),
        "bulk" (TMA bulk row copies) or "rows16" (16-byte row copies); the row
        modes apply where the grid allows.  Results are unchanged."""
        self._check(self._lib.ic_set_stage_copy(self._ctx, self.STAGE_COPY.index(mode)))

    def stage_copy(self):
        """The staging mode the next step's stage kernels use."""
        v = ctypes.c_int()
        self._check(self._lib.ic_get_stage_copy(self._ctx, ctypes.byref(v)))
        return self.STAGE_COPY[v.value]

    def autotune(self, reps=5):
        """Time every stage-kernel tiling on scratch buffers, keep the fastest; returns it."""
        out = (ctypes.c_int * 3)()
        self._check(self._lib.ic_autotune(self._ctx, int(reps), out))
        return tuple(out)

    def profile(self, enable=True):
        """Kernel timing on/off (graphs are off while it is on)."""
        self._check(self._lib.ic_profile(self._ctx, 1 if enable else 0))

    PROFILE_CLASSES = ("fluid", "particles", "end", "adjoint_stage", "adjoint_grid", "adjoint_particles")

    def profile_read(self, reset=True):
        """{class: (ms, launches)} per kernel class (PROFILE_CLASSES) since the last reset."""
        k = len(self.PROFILE_CLASSES)
        ms = np.empty(k)
        n = (ctypes.c_int64 * k)()
        self._check(self._lib.ic_profile_read(self._ctx, _ptr(ms), n, 1 if reset else 0))
        return {c: (float(ms[i]), int(n[i])) for i, c in enumerate(self.PROFILE_CLASSES)}

    def views(self):
        """Zero-copy torch tensors over the current device state (delta rho, g, q)."""
        import torch

        v = _lib.Views()
        self._check(self._lib.ic_device_views(self._ctx, ctypes.byref(v)))
        typestr = "<f4" if v.precision == IC_FP32 else "<f8"

        class _Arr:
            def __init__(self, ptr, shape, ts):
                self.__cuda_array_interface__ = {"shape": shape, "typestr": ts, "data": (ptr, False),
                                                 "version": 3, "strides": None}

        out = {k: torch.as_tensor(_Arr(getattr(v, k), self.shape, typestr), device=self.device)
               for k in ("drho", "gx", "gy", "gz")}
        if v.n_particles:
            # FP64: positions in length units; FP32: int64 fixed point q/h * 2^40
            out["q"] = torch.as_tensor(_Arr(v.q, (v.n_particles, 3), "<i8" if v.precision == IC_FP32 else "<f8"),
                                       device=self.device)
        return out


class Batch:
    """An ensemble of Grids advanced together: one CUDA graph launch per step
    holds every box's kernels as parallel branches (ic_batch_*).  The Grids
    stay usable on their own; the batch does not own them."""

    def __init__(self, grids):
        self._lib = _lib.load()
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g._ctx.value for g in self.grids])
        self._b = ctypes.c_void_p()
        st = self._lib.ic_batch_create(arr, len(self.grids), ctypes.byref(self._b))
        if st != 0:
            raise ICError(st, "ic_batch_create failed (each grid may appear once)")

    def step(self, nsteps=1, weights=None):
        w = None if weights is None else _f64(weights)
        st = self._lib.ic_batch_step(self._b, int(nsteps), _ptr(w))
        if st != 0:
            msg = self._lib.ic_last_error(self.grids[0]._ctx)
            raise ICError(st, msg.decode() if msg else "ic_batch_step failed")

    def autotune(self, reps=5):
        """Tune the stage tiling once per distinct box shape; returns each box's tiling."""
        st = self._lib.ic_batch_autotune(self._b, int(reps))
        if st != 0:
            raise ICError(st, "ic_batch_autotune failed")
        return [g.tile() for g in self.grids]

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self._lib.ic_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
