"""GB300 hybrid lattice Boltzmann (HLBM) library: Python binding of libhlbm.so.

The binding only marshals arguments; every step of the method runs in the
library's CUDA kernels.  PyTorch supplies the CUDA stream and (optionally) the
device allocator.  The functions mirror the C ABI in include/hlbm.h:
hlbm_create, hlbm_step, hlbm_forces, hlbm_fields, hlbm_populations,
hlbm_info, hlbm_inspect, hlbm_sync, hlbm_destroy, hlbm_last_error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HLBM_DEBUG=1 selects the build with the kernels' index bounds checks
LIB_PATH = os.path.join(_HERE, "libhlbm_debug.so" if os.environ.get("HLBM_DEBUG") == "1" else "libhlbm.so")

HLBM_OK, HLBM_EINVAL, HLBM_ENOMEM, HLBM_ECUDA = 0, -1, -2, -3
HLBM_EUNSTABLE, HLBM_ETIMEOUT, HLBM_ESTATE, HLBM_ENOTIMPL = -4, -5, -6, -7
HLBM_FP64, HLBM_FP32, HLBM_FP16S = 0, 1, 2
PRECISIONS = {"fp64": HLBM_FP64, "fp32": HLBM_FP32, "fp16s": HLBM_FP16S}


class HlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hlbm error {code}: {msg}")
        self.code = code


class hlbm_level(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("ox", C.c_int32), ("oy", C.c_int32)]


class hlbm_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("xy", C.POINTER(C.c_double)), ("n_tri", C.c_int32),
                ("tri", C.POINTER(C.c_int32)), ("kind", C.POINTER(C.c_uint8)), ("chord", C.c_double),
                ("pivot", C.c_double * 2), ("hole", C.c_double * 4)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class hlbm_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_sub", C.c_int32), ("seed", C.c_uint64), ("perturb", C.c_double),
                ("force_cap", C.c_int32), ("check_every", C.c_int32), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p), ("use_graphs", C.c_int32),
                ("wall_stats", C.c_int32), ("fv_variant", C.c_int32), ("fv_filter", C.c_double)]


_lib = None


def lib():
    """The loaded libhlbm.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2006_10487_gb300.build` (--debug for the bounds-checked "
                              "library; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.hlbm_create.argtypes = [C.POINTER(hlbm_level), C.c_int, C.POINTER(hlbm_mesh), C.c_double, C.c_double,
                                  C.c_double, C.POINTER(hlbm_options), C.POINTER(C.c_void_p)]
        L.hlbm_step.argtypes = [C.c_void_p, C.c_int]
        L.hlbm_forces.argtypes = [C.c_void_p, dp, dp, C.c_int, ip]
        L.hlbm_fields.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, C.c_size_t]
        L.hlbm_populations.argtypes = [C.c_void_p, C.c_int, dp, C.c_size_t]
        L.hlbm_info.argtypes = [C.c_void_p, C.c_char_p, dp]
        L.hlbm_inspect.argtypes = [C.POINTER(hlbm_level), C.c_int, C.POINTER(hlbm_mesh), C.c_double, C.c_double,
                                   C.c_double, C.POINTER(hlbm_options), C.c_char_p, dp, C.c_size_t,
                                   C.POINTER(C.c_size_t)]
        L.hlbm_time_kernel.argtypes = [C.c_void_p, C.c_char_p, C.c_int, dp]
        L.hlbm_wall_forces_static.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                              C.c_double, C.c_void_p, C.c_void_p]
        L.hlbm_fv_adjoint.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, dp, dp, C.c_size_t, dp,
                                      C.c_size_t, dp, C.c_size_t, dp]
        L.hlbm_adjoint.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, dp, dp, C.c_size_t, dp,
                                   C.c_size_t, dp, C.c_size_t, dp]
        L.hlbm_sync.argtypes = [C.c_void_p]
        L.hlbm_destroy.argtypes = [C.c_void_p]
        L.hlbm_last_error.argtypes = [C.c_void_p]
        L.hlbm_last_error.restype = C.c_char_p
        L.hlbm_wall_stats.argtypes = [C.c_void_p, dp, C.c_size_t, ip, C.POINTER(C.c_long)]
        L.hlbm_wall_stats_reset.argtypes = [C.c_void_p]
        L.hlbm_save.argtypes = [C.c_void_p, C.c_char_p]
        L.hlbm_load.argtypes = [C.c_void_p, C.c_char_p]
        L.hlbm_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
        L.hlbm_batch_step.argtypes = [C.c_void_p, C.c_int]
        L.hlbm_batch_sync.argtypes = [C.c_void_p]
        L.hlbm_batch_destroy.argtypes = [C.c_void_p]
        L.hlbm_batch_last_error.argtypes = [C.c_void_p]
        L.hlbm_batch_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def hlbm_last_error(ctx=None):
    return lib().hlbm_last_error(ctx).decode()


def _check(rc, ctx=None):
    if rc != HLBM_OK:
        raise HlbmError(rc, hlbm_last_error(ctx))


def _marshal(case, precision="fp64", n_sub=None, seed=None, perturb=None, force_cap=0, check_every=0,
             stream=None, use_graphs=True, allocator=None, wall_stats=False, fv_variant=0, fv_filter=None):
    """C structures for a workloads.Case (kept alive by the returned tuple)."""
    lv = (hlbm_level * case.n_levels)(*[hlbm_level(*map(int, r)) for r in case.levels])
    xy = np.ascontiguousarray(case.xy, dtype=np.float64).reshape(-1)
    tri = np.ascontiguousarray(case.tri, dtype=np.int32).reshape(-1)
    kind = np.ascontiguousarray(case.kind, dtype=np.uint8)
    m = hlbm_mesh()
    m.n_nodes = case.n_nodes
    m.xy = xy.ctypes.data_as(C.POINTER(C.c_double))
    m.n_tri = int(case.tri.shape[0]) if case.n_nodes else 0
    m.tri = tri.ctypes.data_as(C.POINTER(C.c_int32))
    m.kind = kind.ctypes.data_as(C.POINTER(C.c_uint8))
    m.chord = case.chord
    m.pivot[:] = list(map(float, case.pivot))
    m.hole[:] = list(map(float, case.hole))
    o = hlbm_options()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.n_sub = int(case.n_sub if n_sub is None else n_sub)
    o.seed = int(case.seed if seed is None else seed)
    o.perturb = float(case.perturb if perturb is None else perturb)
    o.force_cap = int(force_cap)
    o.check_every = int(check_every)
    o.stream = stream
    o.use_graphs = 1 if use_graphs else 0
    o.wall_stats = 1 if wall_stats else 0
    o.fv_variant = int(fv_variant)
    o.fv_filter = float(getattr(case, "fv_filter", 0.0) if fv_filter is None else fv_filter)
    if allocator is not None:
        o.alloc, o.free = allocator
    return lv, m, o, (xy, tri, kind)


def hlbm_inspect(case, table, **kw):
    """Host-only set-up table (no GPU needed), as float64 numpy array."""
    lv, m, o, keep = _marshal(case, **kw)
    n = C.c_size_t()
    L = lib()
    _check(L.hlbm_inspect(lv, case.n_levels, C.byref(m), case.Re, case.Ma, case.aoa_deg, C.byref(o),
                          table.encode(), None, 0, C.byref(n)))
    out = np.empty(n.value)
    _check(L.hlbm_inspect(lv, case.n_levels, C.byref(m), case.Re, case.Ma, case.aoa_deg, C.byref(o),
                          table.encode(), out.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n)))
    return out


def _torch_allocator():
    import torch
    dev = torch.cuda.current_device()

    def _alloc(size, _ctx):
        return torch.cuda.caching_allocator_alloc(int(size), dev, torch.cuda.current_stream(dev))

    def _free(ptr, _ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(_alloc), FREE_FN(_free)


class Solver:
    """One HLBM simulation on the current CUDA device (wraps an hlbm_ctx)."""

    def __init__(self, case, precision="fp64", n_sub=None, seed=None, perturb=None, force_cap=0, check_every=0,
                 use_graphs=True, stream=None, torch_memory=True, wall_stats=False, fv_variant=0, fv_filter=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the HLBM library needs a CUDA device (there is no CPU fallback)")
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._alloc = _torch_allocator() if torch_memory else None
        self._args = _marshal(case, precision, n_sub, seed, perturb, force_cap, check_every, stream, use_graphs,
                              self._alloc, wall_stats, fv_variant, fv_filter)
        lv, m, o, _ = self._args
        ctx = C.c_void_p()
        self._lib = lib()
        _check(self._lib.hlbm_create(lv, case.n_levels, C.byref(m), case.Re, case.Ma, case.aoa_deg, C.byref(o),
                                     C.byref(ctx)))
        self.ctx = ctx
        self.case = case

    def wall_stats(self):
        """Mean wall coefficients since creation or the last reset (Eq. 12-13):
        ([n_wall, 10] array with columns x/C, side, C_p, C_f, C_n, |N_P|, n_x,
        n_y, s_x, s_y; see hlbm_wall_stats), number of coarse steps averaged."""
        nw, ns = C.c_int(), C.c_long()
        _check(self._lib.hlbm_wall_stats(self.ctx, None, 0, C.byref(nw), C.byref(ns)), self.ctx)
        out = np.empty((nw.value, 10))
        _check(self._lib.hlbm_wall_stats(self.ctx, out.ctypes.data_as(C.POINTER(C.c_double)), out.size,
                                         C.byref(nw), C.byref(ns)), self.ctx)
        return out, ns.value

    def fv_adjoint(self, n_window, wd=1.0, wl=0.0):
        """Discrete adjoint of n_window finite-volume sub-steps and the force
        functional J = wd C_D + wl C_L (hlbm_fv_adjoint; FP64 contexts).
        Returns J, dJ/dg of the initial mesh populations ([n_nodes, 9], input
        order), dJ/d(s_x, s_y, C) of the Eq. 3 entries ([nnz, 3], the order of
        the "rowptr" / "col" set-up tables), dJ/dx of the input-frame node
        coordinates ([n_nodes, 2]) and dJ/d(angle of attack) per degree."""
        n, nnz = self.case.n_nodes, int(self.info("nnz"))
        J, da = np.zeros(1), np.zeros(1)
        gg, gc, gx = np.empty((n, 9)), np.empty((nnz, 3)), np.empty((n, 2))
        dp = C.POINTER(C.c_double)
        _check(self._lib.hlbm_fv_adjoint(self.ctx, int(n_window), float(wd), float(wl), J.ctypes.data_as(dp),
                                         gg.ctypes.data_as(dp), gg.size, gc.ctypes.data_as(dp), gc.size,
                                         gx.ctypes.data_as(dp), gx.size, da.ctypes.data_as(dp)), self.ctx)
        return float(J[0]), gg, gc, gx, float(da[0])

    def adjoint(self, n_steps, wd=1.0, wl=0.0, skip=0):
        """Discrete adjoint of n_steps coarse steps of an FP64 or FP32 solver
        (hlbm_adjoint; FP32: FP32 forward steps, FP64 reverse sweep and
        gradient sums): J = mean of wd C_D + wl C_L over the steps after the
        first `skip`, the
        gradients in every level's lattice populations (a list, level order,
        each [ny * nx, 9]) and in the mesh populations [n_nodes, 9] of the
        current state, dJ/dx of the mesh node coordinates [n_nodes, 2] (input
        frame) and dJ/d(angle of attack) per degree; the state is not changed."""
        sizes = [int(nx) * int(ny) for nx, ny in self.case.levels[:, :2]]
        J, da = np.zeros(1), np.zeros(1)
        gl, gm, gx = np.empty((sum(sizes), 9)), np.empty((self.case.n_nodes, 9)), np.empty((self.case.n_nodes, 2))
        dp = C.POINTER(C.c_double)
        _check(self._lib.hlbm_adjoint(self.ctx, int(n_steps), int(skip), float(wd), float(wl), J.ctypes.data_as(dp),
                                      gl.ctypes.data_as(dp), gl.size, gm.ctypes.data_as(dp), gm.size,
                                      gx.ctypes.data_as(dp), gx.size, da.ctypes.data_as(dp)), self.ctx)
        parts = np.split(gl, np.cumsum(sizes)[:-1])
        return float(J[0]), parts, gm, gx, float(da[0])

    def save(self, path):
        """Checkpoint of the whole evolving state (hlbm_save)."""
        _check(self._lib.hlbm_save(self.ctx, os.fsencode(path)), self.ctx)

    def load(self, path):
        """Resume from a checkpoint of a Solver made from the same inputs (hlbm_load)."""
        _check(self._lib.hlbm_load(self.ctx, os.fsencode(path)), self.ctx)

    def wall_stats_reset(self):
        _check(self._lib.hlbm_wall_stats_reset(self.ctx), self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.hlbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_coarse=1):
        _check(self._lib.hlbm_step(self.ctx, int(n_coarse)), self.ctx)

    def sync(self):
        _check(self._lib.hlbm_sync(self.ctx), self.ctx)

    def info(self, key):
        v = C.c_double()
        _check(self._lib.hlbm_info(self.ctx, key.encode(), C.byref(v)), self.ctx)
        return v.value

    def forces(self, cap=1 << 20):
        cd, cl = np.empty(cap), np.empty(cap)
        n = C.c_int()
        dp = C.POINTER(C.c_double)
        _check(self._lib.hlbm_forces(self.ctx, cd.ctypes.data_as(dp), cl.ctypes.data_as(dp), cap, C.byref(n)),
               self.ctx)
        return cd[:n.value].copy(), cl[:n.value].copy()

    def time_kernel(self, kernel, reps=50):
        """Mean duration (ms) of one kernel of the step ("fv", "collide<l>"),
        from CUDA events; consumes the state (only readback afterwards)."""
        v = C.c_double()
        _check(self._lib.hlbm_time_kernel(self.ctx, kernel.encode(), int(reps), C.byref(v)), self.ctx)
        return v.value

    def _size(self, grid):
        if grid == -1:
            return self.case.n_nodes
        nx, ny = self.case.levels[grid][:2]
        return int(nx) * int(ny)

    def fields(self, grid):
        n = self._size(grid)
        r, x, y = np.empty(n), np.empty(n), np.empty(n)
        dp = C.POINTER(C.c_double)
        _check(self._lib.hlbm_fields(self.ctx, grid, r.ctypes.data_as(dp), x.ctypes.data_as(dp),
                                     y.ctypes.data_as(dp), n), self.ctx)
        return r, x, y

    def populations(self, grid):
        n = self._size(grid)
        out = np.empty(9 * n)
        _check(self._lib.hlbm_populations(self.ctx, grid, out.ctypes.data_as(C.POINTER(C.c_double)), 9 * n),
               self.ctx)
        return out.reshape(n, 9)


class Batch:
    """Independent cases (Solvers created with use_graphs=True) advanced together:
    one CUDA graph launch per coarse step runs every case's step on its own
    branch (hlbm_batch_create / hlbm_batch_step).  The Solvers must outlive the
    Batch; read results through them."""

    def __init__(self, solvers, stream=None):
        import torch
        self._lib = lib()
        self.solvers = list(solvers)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx for s in self.solvers])
        b = C.c_void_p()
        rc = self._lib.hlbm_batch_create(arr, len(self.solvers), C.c_void_p(stream), C.byref(b))
        if rc != HLBM_OK:
            raise HlbmError(rc, self._lib.hlbm_batch_last_error(None).decode())
        self.b = b

    def _check(self, rc):
        if rc != HLBM_OK:
            raise HlbmError(rc, self._lib.hlbm_batch_last_error(self.b).decode())

    def step(self, n_coarse=1):
        self._check(self._lib.hlbm_batch_step(self.b, int(n_coarse)))

    def sync(self):
        self._check(self._lib.hlbm_batch_sync(self.b))

    def info(self, key):
        """Sum over the cases of a Solver.info key (e.g. node updates per step)."""
        return sum(s.info(key) for s in self.solvers)

    def close(self):
        if getattr(self, "b", None):
            self._lib.hlbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# names of the C ABI, for callers that prefer the flat interface
def hlbm_create(case, **kw):
    return Solver(case, **kw)


def hlbm_step(solver, n_coarse=1):
    return solver.step(n_coarse)


def hlbm_forces(solver, cap=1 << 20):
    return solver.forces(cap)


def hlbm_fields(solver, grid):
    return solver.fields(grid)


def hlbm_populations(solver, grid):
    return solver.populations(grid)


def hlbm_info(solver, key):
    return solver.info(key)


def hlbm_time_kernel(solver, kernel, reps=50):
    return solver.time_kernel(kernel, reps)


def hlbm_sync(solver):
    return solver.sync()


def hlbm_destroy(solver):
    return solver.close()
