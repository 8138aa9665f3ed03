"""Python access to the HLBM oracle (plain FP64 C, built with gcc).

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA library.  Only the test
suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use
it; the library never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS = {}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def _so_path(openmp):
    return os.path.join(_BUILD, "libhlbm_oracle_omp.so" if openmp else "libhlbm_oracle.so")


def _compile(src, out, openmp=False):
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(openmp=False, force=False):
    """Compile the oracle (gcc -O2, no FMA contraction, no fast-math)."""
    out = _so_path(openmp)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    return _compile(_SRC, out, openmp)


def source():
    """The oracle's C source text."""
    with open(_SRC) as fh:
        return fh.read()


def build_variant(text, out):
    """Compile C source `text` (a modified copy of the oracle, for tests that
    plant a mistake in it and check that a pin catches it) to `out`."""
    src = out[:-3] + ".c"
    with open(src, "w") as fh:
        fh.write(text)
    return _compile(src, out)


def _declare(L):
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.c_int, _ip, C.c_int, _dp, C.c_int, _ip, C.c_char_p,
                             C.c_double, _dp, _dp, C.c_double, C.c_double, C.c_double,
                             C.c_int, C.c_uint64, C.c_double, C.c_int, C.c_char_p, C.c_int]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_step.argtypes = [C.c_void_p, C.c_int]
    L.orc_n_sub.argtypes = [C.c_void_p]
    L.orc_threads.argtypes = []
    L.orc_tau.argtypes = [C.c_void_p, C.c_int]
    L.orc_tau.restype = C.c_double
    L.orc_step_count.argtypes = [C.c_void_p]
    L.orc_step_count.restype = C.c_long
    L.orc_n_forces.argtypes = [C.c_void_p]
    L.orc_forces.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_wall_coeffs.argtypes = [C.c_void_p, _dp]
    L.orc_fields.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp]
    L.orc_populations.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_set_populations.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_apply_outer_bc.argtypes = [C.c_void_p]
    L.orc_set_fv_filter.argtypes = [C.c_void_p, C.c_double]
    L.orc_fv_filter.argtypes = [C.c_int, _ip, _ip, _dp, C.c_char_p, C.c_double, _dp, _dp]
    L.orc_table.argtypes = [C.c_void_p, C.c_char_p, _dp]
    L.orc_table.restype = C.c_long
    L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
    L.orc_moments.argtypes = [_dp, _dp, _dp, _dp]
    L.orc_bgk_collide.argtypes = [_dp, C.c_double]
    L.orc_lattice_periodic.argtypes = [_dp, C.c_int, C.c_int, C.c_double, C.c_int]
    L.orc_lattice_channel.argtypes = [_dp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int]
    L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.orc_uniform.restype = C.c_double
    L.orc_fv_operators.argtypes = [C.c_int, _dp, C.c_int, _ip, _dp, _ip, _ip, _dp, _dp, _dp, _dp]
    L.orc_fv_substep.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_double, C.c_double, _dp, _dp]
    L.orc_fv_substep_literal.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_double, C.c_double, _dp, _dp]
    L.orc_fv_channel_run.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_double, C.c_double, C.c_char_p,
                                     C.c_double, C.c_double, C.c_int, _dp]
    L.orc_wall_rule.argtypes = [_dp]
    L.orc_eq4_post.argtypes = [_dp, C.c_double, _dp]
    L.orc_feq_diff.argtypes = [C.c_double] * 6 + [_dp]
    L.orc_eq5_base.argtypes = [_dp, C.c_double, _dp]
    L.orc_quad6_weights.argtypes = [_dp, C.c_double, C.c_double, _dp]
    L.orc_biquad9_weights.argtypes = [C.c_double, C.c_double, _dp]
    L.orc_wall_force.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp]
    L.orc_fv_window.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, _dp, C.c_double, _dp,
                                C.c_double, _dp, C.c_double, C.c_double, _dp]
    return L


def lib(openmp=False, path=None):
    """The oracle library (the OpenMP build if openmp; a variant built by
    build_variant if path is given)."""
    key = path or openmp
    with _LOCK:
        if key not in _LIBS:
            _LIBS[key] = _declare(C.CDLL(path or build(openmp)))
        return _LIBS[key]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(_dp)


def _pi(a):
    return a.ctypes.data_as(_ip)


# ------------------------------------------------------------ primitives ----
def feq(rho, ux, uy):
    out = np.empty(9)
    lib().orc_feq(rho, ux, uy, _pd(out))
    return out


def moments(f):
    f = _d(f)
    r, x, y = C.c_double(), C.c_double(), C.c_double()
    lib().orc_moments(_pd(f), C.byref(r), C.byref(x), C.byref(y))
    return r.value, x.value, y.value


def bgk_collide(f, tau):
    f = _d(f).copy()
    lib().orc_bgk_collide(_pd(f), tau)
    return f


def lattice_periodic(f, tau, nsteps):
    """f: [ny, nx, 9]; returns the state after nsteps periodic BGK steps."""
    f = _d(f).copy()
    ny, nx, _ = f.shape
    lib().orc_lattice_periodic(_pd(f), nx, ny, tau, nsteps)
    return f


def uniform(seed, gid, idx):
    return lib().orc_uniform(seed, gid, idx)


def fv_operators(xy, tri, tri_xy=None):
    """Eq. 3 operators: (rowptr, col, sx, sy, cc, area)."""
    xy, tri = _d(xy), _i(tri)
    n, ntri = xy.shape[0], tri.shape[0]
    cap = n + 6 * ntri
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(cap, np.int32)
    sx, sy, cc = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    area = np.zeros(n)
    txy = None if tri_xy is None else _d(tri_xy)
    nnz = lib().orc_fv_operators(n, _pd(xy), ntri, _pi(tri), None if txy is None else _pd(txy),
                                 _pi(rowptr), _pi(col), _pd(sx), _pd(sy), _pd(cc), _pd(area))
    if nnz < 0:
        raise ValueError("degenerate or inverted triangle")
    return rowptr, col[:nnz].copy(), sx[:nnz].copy(), sy[:nnz].copy(), cc[:nnz].copy(), area


def fv_substep(ops, dt, tau_u, g):
    rowptr, col, sx, sy, cc, _ = ops
    g = _d(g)
    out = np.empty_like(g)
    lib().orc_fv_substep(g.shape[0], _pi(rowptr), _pi(col), _pd(sx), _pd(sy), _pd(cc), dt, tau_u,
                         _pd(g), _pd(out))
    return out


def fv_substep_literal(ops, dt, tau_u, g):
    """Eq. 3 exactly as printed, on populations (orc_fv_substep_literal)."""
    rowptr, col, sx, sy, cc, _ = ops
    g = _d(g)
    out = np.empty_like(g)
    lib().orc_fv_substep_literal(g.shape[0], _pi(rowptr), _pi(col), _pd(sx), _pd(sy), _pd(cc), dt, tau_u,
                                 _pd(g), _pd(out))
    return out


def fv_channel_run(ops, dt, tau_u, wall, force, nsteps, g):
    """nsteps sub-steps of the solver's Eq. 3 update with a body force and the
    wall rule on the nodes where wall != 0 (orc_fv_channel_run)."""
    rowptr, col, sx, sy, cc, _ = ops
    g = _d(g).copy()
    w = np.ascontiguousarray(wall, dtype=np.uint8)
    lib().orc_fv_channel_run(g.shape[0], _pi(rowptr), _pi(col), _pd(sx), _pd(sy), _pd(cc), dt, tau_u,
                             w.ctypes.data_as(C.c_char_p), float(force[0]), float(force[1]), int(nsteps), _pd(g))
    return g


def lattice_channel(f, tau, Fx, nsteps):
    """f: [ny, nx, 9]; nsteps of Eq. 1 in a channel periodic in x with
    half-way bounce-back walls and a Guo body force Fx (orc_lattice_channel)."""
    f = _d(f).copy()
    ny, nx, _ = f.shape
    lib().orc_lattice_channel(_pd(f), nx, ny, tau, Fx, nsteps)
    return f


def fv_filter(ops, sigma, g, kind=None):
    """One application of the odd-even filter of the mesh state (orc_fv_filter)."""
    rowptr, col, _, _, cc, _ = ops
    g = _d(g)
    out = np.empty_like(g)
    k = None if kind is None else np.ascontiguousarray(kind, dtype=np.uint8)
    lib().orc_fv_filter(g.shape[0], _pi(rowptr), _pi(col), _pd(cc), None if k is None else k.ctypes.data_as(C.c_char_p),
                        float(sigma), _pd(g), _pd(out))
    return out


def wall_rule(g):
    g = _d(g).copy()
    lib().orc_wall_rule(_pd(g))
    return g


def feq_diff(ra, uax, uay, rb, ubx, uby):
    """f^eq(rho_a, u_a) - f^eq(rho_b, u_b) through moment differences."""
    out = np.empty(9)
    lib().orc_feq_diff(ra, uax, uay, rb, ubx, uby, _pd(out))
    return out


def eq4_post(q, tau_s):
    """Eq. 4 post-collision structured state from q = (rho, ux, uy, f^neq[9])."""
    q, out = _d(q), np.empty(9)
    lib().orc_eq4_post(_pd(q), tau_s, _pd(out))
    return out


def eq5_base(q, tau_s):
    """Eq. 5-6 structured part of an unstructured interface state."""
    q, out = _d(q), np.empty(9)
    lib().orc_eq5_base(_pd(q), tau_s, _pd(out))
    return out


def quad6_weights(pts, x, y):
    pts = _d(pts)
    w = np.zeros(6)
    if lib().orc_quad6_weights(_pd(pts), x, y, _pd(w)):
        raise ValueError("singular 6-node stencil")
    return w


def biquad9_weights(fx, fy):
    w = np.zeros(9)
    lib().orc_biquad9_weights(fx, fy, _pd(w))
    return w


def wall_force(ea, eb, xy, g):
    ea, eb, xy, g = _i(ea), _i(eb), _d(xy), _d(g)
    F = np.zeros(2)
    lib().orc_wall_force(ea.shape[0], _pi(ea), _pi(eb), _pd(xy), _pd(g), _pd(F))
    return F


# ---------------------------------------------------------------- solver ----
class Oracle:
    """The whole coupled HLBM on the CPU, FP64."""

    def __init__(self, case, n_sub=None, openmp=False, periodic0=False, literal_fv=False, lib_path=None,
                 fv_filter=None):
        self._lib = lib(openmp, lib_path)
        lv = _i(case.levels).reshape(-1)
        xy = _d(case.xy).reshape(-1) if case.n_nodes else np.zeros(2)
        tri = _i(case.tri).reshape(-1) if case.n_nodes else np.zeros(3, np.int32)
        kind = np.ascontiguousarray(case.kind, dtype=np.uint8)
        pivot, hole = _d(case.pivot), _d(case.hole)
        err = C.create_string_buffer(256)
        self._keep = (lv, xy, tri, kind, pivot, hole)
        ns = case.n_sub if n_sub is None else n_sub
        self.h = self._lib.orc_create(case.n_levels, _pi(lv), case.n_nodes, _pd(xy), int(case.tri.shape[0]),
                                      _pi(tri), kind.ctypes.data_as(C.c_char_p), case.chord, _pd(pivot),
                                      _pd(hole), case.Re, case.Ma, case.aoa_deg, int(ns), int(case.seed),
                                      case.perturb, (1 if periodic0 else 0) | (2 if literal_fv else 0), err, 256)
        if not self.h:
            raise ValueError("oracle set-up failed: " + err.value.decode())
        self.case = case
        sigma = getattr(case, "fv_filter", 0.0) if fv_filter is None else fv_filter
        if sigma:
            self._lib.orc_set_fv_filter(self.h, float(sigma))

    def close(self):
        if getattr(self, "h", None):
            self._lib.orc_destroy(self.h)
            self.h = None

    __del__ = close

    @property
    def n_sub(self):
        return self._lib.orc_n_sub(self.h)

    def tau(self, level):
        """Relaxation time of level `level` (-1: the triangular mesh)."""
        return self._lib.orc_tau(self.h, level)

    @property
    def step_count(self):
        return self._lib.orc_step_count(self.h)

    def step(self, ncoarse=1):
        self._lib.orc_step(self.h, int(ncoarse))

    def _grid_size(self, grid):
        if grid == -1:
            return self.case.n_nodes
        nx, ny = self.case.levels[grid][:2]
        return int(nx) * int(ny)

    def fields(self, grid):
        n = self._grid_size(grid)
        r, x, y = np.empty(n), np.empty(n), np.empty(n)
        self._lib.orc_fields(self.h, grid, _pd(r), _pd(x), _pd(y))
        return r, x, y

    def populations(self, grid):
        out = np.empty(self._grid_size(grid) * 9)
        self._lib.orc_populations(self.h, grid, _pd(out))
        return out.reshape(-1, 9)

    def set_populations(self, grid, f):
        f = _d(f).reshape(-1)
        if f.size != self._grid_size(grid) * 9:
            raise ValueError("wrong population count")
        self._lib.orc_set_populations(self.h, grid, _pd(f))

    def apply_outer_bc(self):
        """Apply the level-0 outer conditions to the current state."""
        self._lib.orc_apply_outer_bc(self.h)

    def forces(self):
        n = self._lib.orc_n_forces(self.h)
        cd, cl = np.empty(n), np.empty(n)
        self._lib.orc_forces(self.h, _pd(cd), _pd(cl))
        return cd, cl

    def wall_coeffs(self):
        """Per wall node (ascending index), Eq. 12-13 of the current state:
        columns x/C, side (+1 upper / -1 lower), C_p, C_f, C_n, |N_P|, n_x, n_y,
        s_x, s_y (see orc_wall_coeffs)."""
        n = self._lib.orc_wall_coeffs(self.h, None)
        out = np.empty((n, 10))
        self._lib.orc_wall_coeffs(self.h, _pd(out))
        return out

    def fv_window(self, n_window, wd=1.0, wl=0.0, dg=None, hg=0.0, dcoef=None, hc=0.0, dxy=None, hx=0.0,
                  daoa=0.0):
        """J = wd C_D + wl C_L after n_window finite-volume sub-steps from the
        current mesh state with the interface data of the current lattice held
        fixed (orc_fv_window), optionally with the initial populations moved
        by hg * dg ([n][9]), the operator entries by hc * dcoef ([nnz][3]), the
        input-frame node coordinates by hx * dxy ([n][2]) and the angle of
        attack by daoa degrees (geometry rebuilt, state kept)."""
        J = np.zeros(1)
        # converted arrays are kept alive through the call
        dg = None if dg is None else _d(dg).reshape(-1)
        dcoef = None if dcoef is None else _d(dcoef).reshape(-1)
        dxy = None if dxy is None else _d(dxy).reshape(-1)
        ptr = [None if a is None else _pd(a) for a in (dg, dcoef, dxy)]
        if self._lib.orc_fv_window(self.h, int(n_window), float(wd), float(wl), ptr[0], float(hg), ptr[1],
                                   float(hc), ptr[2], float(hx), float(daoa), _pd(J)) != 0:
            raise ValueError("fv_window needs a mesh, 1 <= n_window <= n_sub and a valid moved mesh")
        return float(J[0])

    def table(self, name):
        n = self._lib.orc_table(self.h, name.encode(), None)
        if n < 0:
            raise KeyError(name)
        out = np.empty(n)
        self._lib.orc_table(self.h, name.encode(), _pd(out))
        return out
