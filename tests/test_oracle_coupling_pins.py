"""Pins of the oracle's Eq. 3 update, its coupling schedule, its outer rules
and its wall treatment against what the paper and the mathematics fix.

* The re-cast finite-volume update (state held as (rho, u, f^neq), streaming
  in difference form) against Eq. 3 written out literally on populations.
* The lattice <-> mesh coupling in motion (Eq. 4-9 with the time schedule of
  one structured step): a body-free square mesh inside a lattice hole keeps a
  uniform stream uniform, and a transverse wave advected across the overlap
  band stays as close to the lattice-only solution as that solution is to the
  analytic one.
* Poiseuille flow on both grids: the lattice with half-way bounce-back walls
  and Guo forcing (exact at tau = 1/2 + sqrt(3/16), a parabola plus a uniform
  slip otherwise), and the finite-volume mesh with the wall rule (second order).
* The level-0 outer rules in closed form on a prescribed non-uniform state.

The last test plants plausible mistakes in copies of the oracle and checks
that one of these pins fails for each.
"""
import math

import numpy as np
import pytest

from workloads import patch_case
from workloads.naca import Case

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EPS = np.finfo(float).eps


def _feq(rho, ux, uy):
    """Eq. 2 with c_s^2 = 1/3, vectorised over nodes."""
    rho, ux, uy = (np.asarray(a, float)[..., None] for a in (rho, ux, uy))
    cu = CX * ux + CY * uy
    return W * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))


def _moments(g):
    rho = g.sum(-1)
    return rho, (g * CX).sum(-1) / rho, (g * CY).sum(-1) / rho


# ------------------------------------------------ literal Eq. 3 ------------
def _random_state(n, rng):
    g = _feq(1 + 0.05 * rng.uniform(-1, 1, n), 0.1 * rng.uniform(-1, 1, n), 0.1 * rng.uniform(-1, 1, n))
    return g + 1e-3 * W * rng.uniform(-1, 1, (n, 9))


def test_literal_eq3_matches_the_recast_update(orc):
    """Eq. 3 as printed (populations, sums over P and its neighbours) and the
    solver's re-cast update ((rho, u, f^neq) state, streaming as
    sum_k S_ik [g(P_k) - g(P)], f^eq differences through moment differences)
    are the same mathematics.  On random far-from-equilibrium states of the
    80 x 65 airfoil mesh (wall and outer-ring rows included) they agree to the
    rounding of the literal sum: |diff| <= 32 eps B with
    B = |g| + dt sum_k |S_ik g_k| + (dt/tau) sum_k |C_k (g_k - g^eq_k)|.
    The increments themselves are ~1e-2, so a wrong constant in the velocity
    update or in the rebuilt f^neq_0..2 misses by thirteen orders."""
    from workloads import make_case
    case = make_case("hlbm_small")
    ops = orc.fv_operators(case.xy, case.tri)
    rowptr, col, sx, sy, cc, _ = ops
    n = case.n_nodes
    rng = np.random.default_rng(5)
    dt, tau = 1 / 72, 0.013856406460551019
    for _ in range(2):
        g = _random_state(n, rng)
        a = orc.fv_substep(ops, dt, tau, g)
        b = orc.fv_substep_literal(ops, dt, tau, g)
        neq = g - _feq(*_moments(g))
        rows = np.repeat(np.arange(n), np.diff(rowptr))
        S = CX[None, :] * sx[:, None] + CY[None, :] * sy[:, None]
        B = np.abs(g).copy()
        np.add.at(B, rows, dt * np.abs(S * g[col]) + dt / tau * np.abs(cc[:, None] * neq[col]))
        assert np.abs(b - g).max() > 1e-3
        assert (np.abs(a - b) / (EPS * B)).max() <= 32


@pytest.mark.parametrize("name,steps", [("hlbm_small", 20), ("hlbm_mini2", 10)])
def test_solver_with_literal_eq3_matches(orc, name, steps):
    """The whole coupled step (every part the same) with the literal Eq. 3 in
    place of the re-cast update: density and velocity on every grid within
    1e-11 of the field scale and the force series within 1e-12, at 8 degrees.
    (The literal form loses relative precision in f^neq, which it recovers as
    the small difference g - f^eq; that is the only difference.)"""
    from workloads import make_case
    case = make_case(name, aoa_deg=8.0)
    a, b = orc.Oracle(case), orc.Oracle(case, literal_fv=True)
    a.step(steps)
    b.step(steps)
    for grid in list(range(case.n_levels)) + [-1]:
        (ar, ax, ay), (br, bx, by) = a.fields(grid), b.fields(grid)
        m = np.isfinite(br)
        assert np.array_equal(np.isfinite(ar), m)
        assert np.abs(ar[m] - br[m]).max() <= 1e-11 * np.abs(br[m]).max()
        assert np.hypot(ax[m] - bx[m], ay[m] - by[m]).max() <= 1e-11 * np.hypot(bx[m], by[m]).max()
    (cd, cl), (cd2, cl2) = a.forces(), b.forces()
    assert np.abs(cd - cd2).max() <= 1e-12 * np.abs(cd2).max()
    assert np.abs(cl - cl2).max() <= 1e-12 * np.abs(cl2).max()


# ------------------------------------------------ outer rules ---------------
def _outer_rules_error(orc, lib_path=None):
    """Max deviation of the oracle's level-0 outer conditions from their
    closed form on a random non-uniform state (12 x 9 level)."""
    nx, ny = 12, 9
    u0 = 0.1 / math.sqrt(3)
    case = Case("bc", np.asarray([[nx, ny, 0, 0]], np.int32), np.zeros((0, 2)), np.zeros((0, 3), np.int32),
                np.zeros(0, np.uint8), chord=10.0, pivot=(0, 0), hole=(0, 0, 0, 0), Re=100.0, Ma=0.1,
                aoa_deg=0.0, perturb=0.0)
    o = orc.Oracle(case, lib_path=lib_path)
    rng = np.random.default_rng(12)
    n = nx * ny
    rho = 1 + 0.02 * rng.uniform(-1, 1, n)
    ux, uy = u0 + 0.02 * rng.uniform(-1, 1, n), 0.02 * rng.uniform(-1, 1, n)
    neq = 1e-3 * W * rng.uniform(-1, 1, (n, 9))
    neq -= np.outer(neq.sum(1), W)                           # no mass ...
    neq -= 3 * np.outer((neq * CX).sum(1), W * CX) + 3 * np.outer((neq * CY).sum(1), W * CY)  # ... nor momentum
    f = _feq(rho, ux, uy) + neq
    o.set_populations(0, f)
    o.apply_outer_bc()
    got = o.populations(0).reshape(ny, nx, 9)
    f = f.reshape(ny, nx, 9)
    rho, ux, uy, neq = (a.reshape(ny, nx, *a.shape[1:]) for a in (rho, ux, uy, neq))
    want = f.copy()
    for y in range(ny):
        for x in range(nx):
            if 0 < x < nx - 1 and 0 < y < ny - 1:
                continue
            xn, yn = min(max(x, 1), nx - 2), min(max(y, 1), ny - 2)
            if x == 0:      # inlet: u = (u0, 0), rho and f^neq from the interior neighbour
                want[y, x] = _feq(rho[yn, xn], u0, 0.0) + neq[yn, xn]
            elif x == nx - 1:   # outlet: rho = 1, u and f^neq from the interior neighbour
                want[y, x] = _feq(1.0, ux[yn, xn], uy[yn, xn]) + neq[yn, xn]
            else:           # top and bottom: zero gradient of every population
                want[y, x] = f[yn, xn]
    return np.abs(got - want).max()


def test_outer_rules_closed_form(orc):
    """Level-0 outer conditions (Section 4; reading: inlet f^eq(rho_n, (u0, 0)) +
    f^neq_n, outlet f^eq(1, u_n) + f^neq_n, top and bottom copies, corners with
    the inlet or outlet rule, n the nearest interior node) on a prescribed
    random state, against the closed form node by node.  Swapping the inlet
    and outlet rules, extrapolating rho at the outlet, or taking the wrong
    neighbour each miss by at least 1e-4."""
    assert _outer_rules_error(orc) < 1e-15


# ------------------------------------------------ coupling in motion --------
def _patch_oracle(orc, mesh, m=32, lib_path=None):
    return orc.Oracle(patch_case(m=m, mesh=mesh), periodic0=True, lib_path=lib_path)


def _uniform_patch_deviation(orc, lib_path=None, steps=30):
    """Largest deviation from (rho, u) = (1, (u0, 0)) on the lattice and the
    body-free mesh after `steps` coupled steps of a uniform stream."""
    o = _patch_oracle(orc, True, lib_path=lib_path)
    o.step(steps)
    u0 = 0.1 / math.sqrt(3)
    dev = 0.0
    for grid in (0, -1):
        r, ux, uy = o.fields(grid)
        m = np.isfinite(r)
        dev = max(dev, np.abs(r[m] - 1).max(), np.abs(ux[m] - u0).max(), np.abs(uy[m]).max())
    return dev


def test_uniform_stream_through_the_body_free_coupling(orc):
    """A uniform stream (rho 1, u = (u0, 0)) through a periodic lattice with a
    body-free square mesh in a circular hole stays uniform to rounding through
    Eq. 4 with Eq. 8 (hole boundary), Eq. 5-7 with Eq. 9 (outer ring, linear
    in time) and the Eq. 3 sub-steps: every interpolation reproduces constants
    and the closed control volumes have sum_k S_ik = 0."""
    assert _uniform_patch_deviation(orc) < 1e-14


def _band_wave(orc, lib_path=None, T=200):
    """A transverse wave u = (u0, U sin(k x)) (k = 2 pi / 64, U = 1e-3,
    nu = 0.1, Ma = 0.1) advected T steps through the periodic 64 x 64 lattice,
    once alone and once with the body-free 33 x 33-node mesh (spacing 0.75,
    placed off the lattice nodes) over a circular hole of radius 8.  Returns,
    in units of U:
      e_lat   lattice-only error against U sin(k (x - u0 t)) exp(-nu k^2 t),
      e_cpl   the coupled run's error on its computed lattice nodes, same,
      d_lat   coupled minus lattice-only on those nodes,
      d_mesh  mesh u_y minus the lattice-only solution at the mesh nodes
              (its sine fit, exact to 1e-12 since that solution is a pure
              travelling sine)."""
    n0, U, u0 = 64, 1e-3, 0.1 / math.sqrt(3)
    k = 2 * math.pi / n0
    runs = []
    for mesh in (False, True):
        o = _patch_oracle(orc, mesh, lib_path=lib_path)

        def state(x, tau):
            # equilibrium plus the first-order Chapman-Enskog part of du_y/dx
            return _feq(1.0, u0, U * np.sin(k * x)) - (tau * 3 * W * CX * CY * U * k) * np.cos(k * x)[:, None]

        o.set_populations(0, state(np.tile(np.arange(n0, dtype=float), n0), o.tau(0)))
        if mesh:
            o.set_populations(-1, state(o.case.xy[:, 0], o.tau(-1)))
        o.step(T)
        runs.append(o)
    nu = (runs[0].tau(0) - 0.5) / 3
    x = np.tile(np.arange(n0, dtype=float), n0)
    exact = U * np.sin(k * (x - u0 * T)) * math.exp(-nu * k * k * T)
    uy1, uy2 = runs[0].fields(0)[2], runs[1].fields(0)[2]
    m = np.isfinite(uy2)
    row = uy1[:n0]
    A = np.stack([np.sin(k * np.arange(n0)), np.cos(k * np.arange(n0))], axis=1)
    coef = np.linalg.lstsq(A, row, rcond=None)[0]
    assert np.abs(A @ coef - row).max() < 1e-10 * U
    if not m.any() or not np.isfinite(uy2[m]).all():
        return dict(e_lat=np.abs(uy1 - exact).max() / U, e_cpl=np.inf, d_lat=np.inf, d_mesh=np.inf)
    xm = runs[1].case.xy[:, 0]
    fit = coef[0] * np.sin(k * xm) + coef[1] * np.cos(k * xm)
    return dict(e_lat=np.abs(uy1 - exact).max() / U, e_cpl=np.abs(uy2[m] - exact[m]).max() / U,
                d_lat=np.abs(uy2[m] - uy1[m]).max() / U, d_mesh=np.abs(runs[1].fields(-1)[2] - fit).max() / U)


def _band_wave_ok(r):
    return (r["e_lat"] < 2e-3 and r["e_cpl"] <= 1.25 * r["e_lat"]
            and r["d_lat"] <= r["e_lat"] and r["d_mesh"] <= r["e_lat"])


def test_advected_wave_crosses_the_overlap_band(orc):
    """The coupling in motion (Section 2: the two schemes "solved consistently
    in time"; Eq. 4 from the mesh state at t, the lattice step t -> t+1, the
    ring's Eq. 9 data linear in time at theta = m/n for sub-step m): a wave
    crossing the band stays within 25 % of the lattice-only error against the
    analytic solution, and the mesh and the coupled lattice stay closer to the
    lattice-only solution than that solution is to the analytic one.
    Measured: e_lat 1.51e-3, e_cpl 1.76e-3, d_lat 3.2e-4, d_mesh 1.22e-3.
    A lag of one sub-step in theta gives d_mesh 2.05e-3, time interpolation
    run backwards 3.7e-3, no time interpolation 5.8e-3 (and e_cpl 1.9 e_lat)."""
    r = _band_wave(orc)
    assert _band_wave_ok(r), r


# ------------------------------------------------ Poiseuille ----------------
def _lattice_poiseuille(orc, tau, ny=16, F=1e-5, steps=60000, lib_path=None):
    lib = orc.lib(path=lib_path) if lib_path else orc.lib()
    f = np.ascontiguousarray(np.tile(W, (ny, 2, 1)))
    lib.orc_lattice_channel(orc._pd(f), 2, ny, tau, F, steps)
    rho = f.sum(-1)
    ux = ((f * CX).sum(-1) + 0.5 * F) / rho
    nu = (tau - 0.5) / 3
    y = np.arange(ny)
    exact = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    return (ux[:, 0] - exact) / exact.max(), np.abs(ux[:, 0] - ux[:, 1]).max()


def test_lattice_poiseuille_with_bounce_back(orc):
    """Eq. 1 (BGK collide-stream with Eq. 2) in a force-driven channel between
    half-way bounce-back walls (test-only walls; Guo forcing): the steady
    velocity is the Navier-Stokes parabola F/(2 nu) (y + 1/2)(H - 1/2 - y) with
    nu = (tau - 1/2)/3, exactly (to rounding) at tau = 1/2 + sqrt(3/16), and a
    parabola plus a uniform slip otherwise, the slip changing sign at that tau.
    A wrong viscosity, weight or streaming direction breaks the parabola."""
    d, dx = _lattice_poiseuille(orc, 0.5 + math.sqrt(3 / 16))
    assert np.abs(d).max() < 5e-12 and dx < 1e-18
    slips = []
    for tau in (0.6, 1.2):
        d, _ = _lattice_poiseuille(orc, tau)
        assert np.ptp(d) < 1e-11
        slips.append(d.mean())
    assert slips[0] < -1e-3 and slips[1] > 1e-3


def _strip(nxm, m, H):
    """Periodic-in-x triangulated strip 0 <= y <= H, m cells across, with wall
    nodes on y = 0 and y = H (unwrapped triangle coordinates for the wrap)."""
    h = H / m
    xy = np.array([[i * h, j * h] for j in range(m + 1) for i in range(nxm)], float)
    tri, txy = [], []
    for j in range(m):
        for i in range(nxm):
            a, b = j * nxm + i, j * nxm + (i + 1) % nxm
            c, d = (j + 1) * nxm + i, (j + 1) * nxm + (i + 1) % nxm
            pa, pb, pc, pd = (i * h, j * h), ((i + 1) * h, j * h), (i * h, (j + 1) * h), ((i + 1) * h, (j + 1) * h)
            if (i + j) % 2 == 0:
                tri += [(a, b, d), (a, d, c)]
                txy += [(pa, pb, pd), (pa, pd, pc)]
            else:
                tri += [(a, b, c), (b, d, c)]
                txy += [(pa, pb, pc), (pb, pd, pc)]
    wall = np.array([j in (0, m) for j in range(m + 1) for _ in range(nxm)], np.uint8)
    return xy, np.array(tri, np.int32), np.array(txy, float), wall


def _fv_poiseuille_error(orc, m, H=8.0, tau_u=0.1, F=1e-5):
    xy, tri, txy, wall = _strip(4, m, H)
    ops = orc.fv_operators(xy, tri, txy)
    nu = tau_u / 3
    dt = 0.1
    y = xy[:, 1]
    exact = F / (2 * nu) * y * (H - y)
    g = _feq(np.ones_like(y), exact, np.zeros_like(y))
    steps = int(8 * H * H / (math.pi**2 * nu) / dt)     # eight e-folds of the slowest mode
    g = orc.fv_channel_run(ops, dt, tau_u, wall, (F, 0.0), steps, g)
    return np.abs(_moments(g)[1] - exact).max() / exact.max()


def test_fv_poiseuille_is_second_order(orc):
    """Eq. 3 with the wall rule (u = 0 at wall nodes, rho and f^neq kept) in a
    force-driven periodic strip of the triangular mesh: the steady profile
    converges to the Navier-Stokes parabola with nu = c_s^2 tau_u at second
    order in the mesh spacing (errors 3.8e-2 and 9.5e-3 of u_max at 8 and 16
    cells across)."""
    e8, e16 = _fv_poiseuille_error(orc, 8), _fv_poiseuille_error(orc, 16)
    assert e16 < 0.012
    assert 3.6 < e8 / e16 < 4.4


# ------------------------------------------------ planted mistakes ----------
MUTANTS = {
    # coupling schedule and overlap formulas
    "theta lags one sub-step": ("ring_set(o, (double)m / o->n_sub);", "ring_set(o, (double)(m + 1) / o->n_sub);"),
    "no time interpolation": ("ring_set(o, (double)m / o->n_sub);", "ring_set(o, 0.0);"),
    "time interpolation reversed": (
        "q[m] = (1.0 - theta) * o->Q0[12 * (size_t)r + m] + theta * o->Q1[12 * (size_t)r + m];",
        "q[m] = theta * o->Q0[12 * (size_t)r + m] + (1.0 - theta) * o->Q1[12 * (size_t)r + m];"),
    "ring data at t taken after the lattice step": (
        "    if (finest && o->n) ring_interp(o, o->Q0);\n    collide_stream(o, c);",
        "    collide_stream(o, c);\n    if (finest && o->n) ring_interp(o, o->Q0);"),
    "mesh advanced before the lattice (Eq. 4 from t+1)": (
        "    if (finest && o->n) ring_interp(o, o->Q0);\n    collide_stream(o, c);\n"
        "    if (c == 0) { if (!o->periodic0) apply_outer_bc(o); }\n    else prolong(o, c - 1, theta_next);\n"
        "    if (finest && o->n) {\n        ring_interp(o, o->Q1);\n        fv_steps(o);\n    }",
        "    if (finest && o->n) { ring_interp(o, o->Q0); ring_interp(o, o->Q1); fv_steps(o); }\n"
        "    collide_stream(o, c);\n    if (c == 0) { if (!o->periodic0) apply_outer_bc(o); }\n"
        "    else prolong(o, c - 1, theta_next);"),
    "Eq. 4 factor": ("from_q(q, 2.0 * (tau_s - 1.0) / (2.0 * tau_s - 1.0), f);", "from_q(q, (tau_s - 1.0) / tau_s, f);"),
    "Eq. 5 factor dropped": ("qu[3 + i] = (1.0 - 1.0 / (2.0 * tau_s)) * q[3 + i];", "qu[3 + i] = q[3 + i];"),
    "Eq. 9 weights transposed": ("for (int a = 0; a < 3; a++) w[b * 3 + a] = lx[a] * ly[b];",
                                 "for (int a = 0; a < 3; a++) w[a * 3 + b] = lx[a] * ly[b];"),
    # the re-cast Eq. 3 update
    "velocity update without the density change": ("qo[1] = qp[1] + (djx - drho * qp[1]) / rho;",
                                                    "qo[1] = qp[1] + djx / rho;"),
    "f^neq_1 rebuilt with a wrong sign": ("n[1] = n[3] - n[5] + n[6] + n[7] - n[8];",
                                          "n[1] = n[3] - n[5] + n[6] - n[7] - n[8];"),
    "collision on the population, not f^neq": (
        "acc[i] += dt * s * (dfe[i] + qk[3 + i] - qp[3 + i]) - (dt / tau_u) * cc[e] * qk[3 + i];",
        "acc[i] += dt * s * (dfe[i] + qk[3 + i] - qp[3 + i]) - (dt / tau_u) * cc[e] * (qk[3 + i] + dfe[i]);"),
    # outer rules and walls
    "inlet and outlet swapped": ("if (x == 0) { q[1] = o->u0; q[2] = 0.0; from_q(q, 1.0, fb); }\n"
                                 "            else if (x == nx - 1) { q[0] = 1.0; from_q(q, 1.0, fb); }",
                                 "if (x == nx - 1) { q[1] = o->u0; q[2] = 0.0; from_q(q, 1.0, fb); }\n"
                                 "            else if (x == 0) { q[0] = 1.0; from_q(q, 1.0, fb); }"),
    "outlet density extrapolated": ("else if (x == nx - 1) { q[0] = 1.0; from_q(q, 1.0, fb); }",
                                    "else if (x == nx - 1) { from_q(q, 1.0, fb); }"),
    "wall rule keeps u_x": ("            o->gnew[12 * (size_t)o->wall[w] + 1] = 0.0;\n",
                            ""),
}


def _literal_ok(orc, lib_path):
    from workloads import make_case
    lib = orc.lib(path=lib_path)
    case = make_case("hlbm_small")
    rowptr, col, sx, sy, cc, _ = orc.fv_operators(case.xy, case.tri)
    g = _random_state(case.n_nodes, np.random.default_rng(3))
    a, b = np.empty_like(g), np.empty_like(g)
    args = (case.n_nodes, orc._pi(rowptr), orc._pi(col), orc._pd(sx), orc._pd(sy), orc._pd(cc), 1 / 72, 0.0139)
    lib.orc_fv_substep(*args, orc._pd(g), orc._pd(a))
    lib.orc_fv_substep_literal(*args, orc._pd(g), orc._pd(b))
    return np.abs(a - b).max() < 1e-13


def _wall_ok(orc, lib_path):
    from workloads import make_case
    case = make_case("hlbm_small", aoa_deg=8.0)
    o = orc.Oracle(case, lib_path=lib_path)
    o.step(1)
    r, ux, uy = o.fields(-1)
    wall = case.kind == 1
    return np.abs(ux[wall]).max() == 0.0 and np.abs(uy[wall]).max() == 0.0


def test_pins_catch_planted_mistakes(orc, tmp_path):
    """Each plausible mistake, planted in a copy of the oracle, fails at least
    one of the pins above (coupling in motion, uniform stream, literal Eq. 3,
    outer rules, wall velocity), checked cheapest first."""
    src = orc.source()
    for i, (name, (old, new)) in enumerate(MUTANTS.items()):
        assert old in src, name
        # the first occurrence: the solver's sub-step, where a pattern also
        # appears in a later helper
        path = orc.build_variant(src.replace(old, new, 1), str(tmp_path / f"mutant{i}.so"))
        caught = (not _literal_ok(orc, path) or _outer_rules_error(orc, path) > 1e-12
                  or not _wall_ok(orc, path) or _uniform_patch_deviation(orc, path) > 1e-14
                  or not _band_wave_ok(_band_wave(orc, path)))
        assert caught, name


# ------------------------------------------------ host-parallel oracle -------
def test_openmp_build_is_bitwise_the_serial_one(orc):
    """The OpenMP build (node loops on several host threads; each output
    written by one iteration) gives bitwise the serial build's populations and
    force series: 10 coarse steps of the two-level case at 8 degrees."""
    from workloads import make_case
    case = make_case("hlbm_mini2", aoa_deg=8.0)
    a, b = orc.Oracle(case), orc.Oracle(case, openmp=True)
    a.step(10)
    b.step(10)
    for grid in list(range(case.n_levels)) + [-1]:
        assert np.array_equal(a.populations(grid), b.populations(grid), equal_nan=True)
    assert np.array_equal(np.asarray(a.forces()), np.asarray(b.forces()))


# ------------------------------------------------ odd-even filter ------------
def test_fv_filter_conserves_and_damps_the_odd_even_mode(orc):
    """The optional filter g <- g - sigma L L g with (L g)_i(P) = sum_{k != P}
    C_Pk [g_i(P_k) - g_i(P)] (not part of the paper's method) on periodic
    triangulated squares: a uniform state is a fixed point; mass and momentum
    weighted by the control-volume areas are conserved (A_P C_Pk is
    symmetric); the node-to-node checkerboard of u_x is multiplied by exactly
    1 - sigma (14/27)^2 (14/27 is its eigenvalue of L on this triangulation:
    the four opposite-colour neighbours carry 7/108 x 2 A_T / A_P each); a
    smooth shear wave decays like a hyper-diffusion (7/54)^2 sigma h^4 k^4,
    approached at second order in h."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_pins import _periodic_mesh
    sigma = 0.3
    prev = None
    for n in (8, 16):
        xy, tri, txy = _periodic_mesh(n)
        ops = orc.fv_operators(xy.astype(float), tri, txy)
        area = ops[5]
        g = np.tile(orc.feq(1.02, 0.03, -0.01), (xy.shape[0], 1))
        assert np.abs(orc.fv_filter(ops, sigma, g) - g).max() < 1e-16
        rng = np.random.default_rng(3)
        g = _feq(1 + 0.01 * rng.standard_normal(len(xy)), 0.05 * rng.standard_normal(len(xy)),
                 0.05 * rng.standard_normal(len(xy))) + 1e-3 * W * rng.standard_normal((len(xy), 9))
        g2 = orc.fv_filter(ops, sigma, g)
        for mom in (np.ones(9), CX, CY):
            assert abs((area[:, None] * g2 * mom).sum() - (area[:, None] * g * mom).sum()) < 1e-14
        U = 1e-3
        sign = np.array([(-1) ** (int(x) + int(y)) for x, y in xy])
        cb = _feq(np.ones(len(xy)), U * sign, np.zeros(len(xy)))
        ux = _moments(orc.fv_filter(ops, sigma, cb))[1]
        assert np.abs(ux / (U * sign) - (1 - sigma * (14 / 27) ** 2)).max() < 1e-12
        k = 2 * math.pi / n
        wave = _feq(np.ones(len(xy)), U * np.sin(k * xy[:, 1]), np.zeros(len(xy)))
        ux = _moments(orc.fv_filter(ops, sigma, wave))[1]
        amp = 2 / n**2 * (ux * np.sin(k * xy[:, 1])).sum() / U
        D4 = (1 - amp) / (sigma * k**4)           # hyper-diffusion per unit sigma, h = 1
        err = abs(D4 - (7 / 54) ** 2)
        if prev is not None:
            assert 3.5 < prev / err < 4.5
        prev = err
    assert prev < 1e-3
