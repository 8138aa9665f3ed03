"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: a
closed form, an invariant, an independent brute-force computation, hand-derived
values (tests/golden) or an analytic decay rate.  All run on the CPU.
"""
import math
import os

import numpy as np
import pytest

from workloads import make_case

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ Eq. 2 ---------
def test_equilibrium_moments_closed_form(orc):
    """Eq. 2: sum f^eq = rho, sum c f^eq = rho u, sum c c f^eq = rho/3 I + rho u u."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 1 + 0.1 * rng.standard_normal()
        ux, uy = 0.1 * rng.standard_normal(2)
        f = orc.feq(rho, ux, uy)
        assert abs(f.sum() - rho) < 1e-15
        assert abs((CX * f).sum() - rho * ux) < 1e-15
        assert abs((CY * f).sum() - rho * uy) < 1e-15
        assert abs((CX * CX * f).sum() - (rho / 3 + rho * ux * ux)) < 1e-15
        assert abs((CX * CY * f).sum() - rho * ux * uy) < 1e-15
        assert abs((CY * CY * f).sum() - (rho / 3 + rho * uy * uy)) < 1e-15


def test_equilibrium_at_rest_is_weights(orc):
    assert np.allclose(orc.feq(1.0, 0.0, 0.0), W, rtol=0, atol=1e-17)


def test_collision_conserves_mass_and_momentum(orc):
    """Eq. 1: the BGK collision leaves rho and rho u unchanged and relaxes f^neq by (1 - 1/tau)."""
    rng = np.random.default_rng(2)
    for tau in (0.51, 0.8, 1.7):
        f = W * (1 + 0.05 * rng.standard_normal(9))
        g = orc.bgk_collide(f, tau)
        assert abs(g.sum() - f.sum()) < 1e-15
        assert abs((CX * g).sum() - (CX * f).sum()) < 1e-15
        assert abs((CY * g).sum() - (CY * f).sum()) < 1e-15
        r, ux, uy = orc.moments(f)
        eq = orc.feq(r, ux, uy)
        assert np.allclose(g - eq, (1 - 1 / tau) * (f - eq), rtol=0, atol=1e-16)


def test_equilibrium_difference_matches_exact_arithmetic(orc):
    """f^eq(a) - f^eq(b) through moment differences equals Eq. 2 evaluated twice
    and subtracted in exact rational arithmetic, to the rounding of the result
    (not of the O(w_i) equilibria)."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(11)
    wq = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
    for scale in (1e-2, 1e-6, 1e-10):
        for _ in range(5):
            rb = 1 + 0.01 * rng.standard_normal()
            ub = 0.05 * rng.standard_normal(2)
            ra = rb + scale * rng.standard_normal()
            ua = ub + scale * rng.standard_normal(2)
            got = orc.feq_diff(ra, ua[0], ua[1], rb, ub[0], ub[1])
            for i in range(9):
                def E(r, u):
                    r, ux, uy = Fr(r), Fr(u[0]), Fr(u[1])
                    cu = CX[i] * ux + CY[i] * uy
                    return wq[i] * r * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * (ux * ux + uy * uy))
                exact = float(E(ra, ua) - E(rb, ub))
                assert got[i] == pytest.approx(exact, rel=1e-12, abs=1e-15 * scale)


def test_moments(orc):
    rng = np.random.default_rng(3)
    f = W * (1 + 0.1 * rng.standard_normal(9))
    r, ux, uy = orc.moments(f)
    assert r == pytest.approx(f.sum(), abs=1e-16)
    assert ux * r == pytest.approx((CX * f).sum(), abs=1e-16)
    assert uy * r == pytest.approx((CY * f).sum(), abs=1e-16)


# ------------------------------------------------------------ Eq. 1 ---------
def _shear_wave_decay(orc, ny, tau, steps):
    nx = 4
    k = 2 * math.pi / ny
    U = 1e-3
    y = np.arange(ny)
    f = np.zeros((ny, nx, 9))
    for j in range(ny):
        f[j, :, :] = orc.feq(1.0, U * math.sin(k * j), 0.0)
    amp = []
    for _ in range(2):
        f = orc.lattice_periodic(f, tau, steps)
        ux = (f * CX).sum(-1) / f.sum(-1)
        amp.append(2 / ny * (ux.mean(axis=1) * np.sin(k * y)).sum())
    rate = math.log(amp[0] / amp[1]) / steps
    return rate / k**2  # measured viscosity


def test_lattice_viscosity_and_order(orc):
    """Eq. 1 with nu = c_s^2 (tau - 1/2): a shear wave decays at nu k^2, error O(k^2)."""
    tau = 0.8
    nu = (tau - 0.5) / 3
    e16 = abs(_shear_wave_decay(orc, 16, tau, 60) / nu - 1)
    e32 = abs(_shear_wave_decay(orc, 32, tau, 240) / nu - 1)
    assert e32 < 3e-3
    assert 3.5 < e16 / e32 < 4.5  # second order in space


def test_periodic_lattice_streams_downstream(orc):
    """Eq. 1 streaming: with tau = 1 a single population moves by c_i per step."""
    ny, nx = 5, 6
    f = np.zeros((ny, nx, 9))
    f[2, 3, :] = orc.feq(1.0, 0.0, 0.0)
    g = orc.lattice_periodic(f, 1.0, 1)
    for i in range(9):
        assert g[(2 + CY[i]) % ny, (3 + CX[i]) % nx, i] == pytest.approx(W[i], rel=1e-15)


# ------------------------------------------------------------ Eq. 3 ---------
def _random_patch(n=6, seed=4):
    rng = np.random.default_rng(seed)
    xs, ys = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    xy = np.stack([xs.ravel(), ys.ravel()], 1)
    inner = (xy[:, 0] > 0) & (xy[:, 0] < n - 1) & (xy[:, 1] > 0) & (xy[:, 1] < n - 1)
    xy[inner] += 0.25 * (rng.random((inner.sum(), 2)) - 0.5)
    tri = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i, (j + 1) * n + i + 1
            if (i + j) % 2:
                tri += [(a, b, d), (a, d, c)]
            else:
                tri += [(a, b, c), (b, d, c)]
    return xy, np.array(tri, dtype=np.int32)


def test_fv_operator_invariants(orc):
    """Eq. 3 operators: sum_k s_k = 0, sum_k C_Pk = 1, C_PP = 11/18, and linear exactness
    sum_k s_k phi(P_k) = -grad phi on every node (the control volume is closed)."""
    xy, tri = _random_patch()
    rp, col, sx, sy, cc, area = orc.fv_operators(xy, tri)
    for p in range(xy.shape[0]):
        sl = slice(rp[p], rp[p + 1])
        assert abs(sx[sl].sum()) < 1e-12 and abs(sy[sl].sum()) < 1e-12
        assert cc[sl].sum() == pytest.approx(1.0, abs=1e-14)
        assert cc[sl][col[sl] == p][0] == pytest.approx(11 / 18, abs=1e-14)
        for gx, gy in ((1.0, 0.0), (0.0, 1.0), (0.3, -0.7)):
            phi = gx * xy[col[sl], 0] + gy * xy[col[sl], 1]
            assert (sx[sl] * phi).sum() == pytest.approx(-gx, abs=1e-12)
            assert (sy[sl] * phi).sum() == pytest.approx(-gy, abs=1e-12)
    p = xy[tri]
    at = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    assert area.sum() == pytest.approx(at.sum(), rel=1e-14)


def _bary(pt, tri_pts):
    a, b, c = tri_pts
    d = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    la = ((b[0] - pt[0]) * (c[1] - pt[1]) - (b[1] - pt[1]) * (c[0] - pt[0])) / d
    lb = ((c[0] - pt[0]) * (a[1] - pt[1]) - (c[1] - pt[1]) * (a[0] - pt[0])) / d
    return np.array([la, lb, 1 - la - lb])


def test_fv_operators_match_brute_force_quadrature(orc):
    """Eq. 3 operators against a direct numerical evaluation of the cell-vertex
    control-volume integrals: Gauss quadrature of the hat functions over every
    sub-quad and Gauss-Legendre flux integrals along every sub-quad edge (the
    contributions of edges interior to the control volume cancel)."""
    xy, tri = _random_patch(5, seed=9)
    rp, col, sx, sy, cc, area = orc.fv_operators(xy, tri)
    gl = [(0.5 - 0.5 / math.sqrt(3), 0.5), (0.5 + 0.5 / math.sqrt(3), 0.5)]
    tq = [((1 / 6, 1 / 6), 1 / 3), ((2 / 3, 1 / 6), 1 / 3), ((1 / 6, 2 / 3), 1 / 3)]
    n = xy.shape[0]
    for p in range(n):
        A = 0.0
        integ = {}
        flux = {}
        for t in tri:
            if p not in t:
                continue
            r = list(t).index(p)
            order = [t[r], t[(r + 1) % 3], t[(r + 2) % 3]]
            P, Aa, B = xy[order[0]], xy[order[1]], xy[order[2]]
            tp = (P, Aa, B)
            quad = [P, (P + Aa) / 2, (P + Aa + B) / 3, (P + B) / 2]
            for s0, s1, s2 in ((quad[0], quad[1], quad[2]), (quad[0], quad[2], quad[3])):
                ar = 0.5 * ((s1[0] - s0[0]) * (s2[1] - s0[1]) - (s1[1] - s0[1]) * (s2[0] - s0[0]))
                A += ar
                for (u, v), wq in tq:
                    pt = s0 + u * (s1 - s0) + v * (s2 - s0)
                    lam = _bary(pt, tp)
                    for kk in range(3):
                        integ[order[kk]] = integ.get(order[kk], 0.0) + ar * wq * lam[kk]
            for e in range(4):
                u0, u1 = quad[e], quad[(e + 1) % 4]
                nl = np.array([u1[1] - u0[1], -(u1[0] - u0[0])])
                for s, wq in gl:
                    lam = _bary(u0 + s * (u1 - u0), tp)
                    for kk in range(3):
                        flux[order[kk]] = flux.get(order[kk], np.zeros(2)) + wq * lam[kk] * nl
        assert area[p] == pytest.approx(A, rel=1e-13)
        for e in range(rp[p], rp[p + 1]):
            k = col[e]
            assert cc[e] == pytest.approx(integ[k] / A, abs=1e-13)
            assert sx[e] == pytest.approx(-flux[k][0] / A, abs=1e-12)
            assert sy[e] == pytest.approx(-flux[k][1] / A, abs=1e-12)


def test_fv_operators_unit_square_golden(orc):
    """Eq. 3 operators of a corner node of the two-triangle unit square, against
    the hand derivation in tests/golden/fv_unit_square.txt."""
    rows = []
    area = None
    with open(os.path.join(GOLDEN, "fv_unit_square.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "area":
                area = float(tok[1])
            else:
                rows.append([float(t) for t in tok])
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=float)
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    rp, col, sx, sy, cc, ar = orc.fv_operators(xy, tri)
    assert ar[0] == pytest.approx(area, abs=1e-15)
    assert list(col[rp[0]:rp[1]]) == [0, 1, 2, 3]
    for e, (k, gx, gy, gc) in zip(range(rp[0], rp[1]), rows):
        assert col[e] == int(k)
        assert sx[e] == pytest.approx(gx, abs=1e-15)
        assert sy[e] == pytest.approx(gy, abs=1e-15)
        assert cc[e] == pytest.approx(gc, abs=1e-15)


def _periodic_mesh(n):
    xy = np.array([[i, j] for j in range(n) for i in range(n)], dtype=float)
    tri, txy = [], []
    for j in range(n):
        for i in range(n):
            a = j * n + i
            b = j * n + (i + 1) % n
            c = ((j + 1) % n) * n + i
            d = ((j + 1) % n) * n + (i + 1) % n
            pa, pb, pc, pd = (i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1)
            tri += [(a, b, d), (a, d, c)]
            txy += [(pa, pb, pd), (pa, pd, pc)]
    return xy, np.array(tri, dtype=np.int32), np.array(txy, dtype=float)


def _fv_shear_nu(orc, n, tau_u, dt, t_end):
    xy, tri, txy = _periodic_mesh(n)
    ops = orc.fv_operators(xy, tri, txy)
    k = 2 * math.pi / n
    U = 1e-3
    g = np.array([orc.feq(1.0, U * math.sin(k * y), 0.0) for _, y in xy])
    steps = int(round(t_end / dt))
    amp = []
    for _ in range(2):
        for _ in range(steps):
            g = orc.fv_substep(ops, dt, tau_u, g)
        ux = (g * CX).sum(1) / g.sum(1)
        amp.append(2 / n**2 * (ux * np.sin(k * xy[:, 1])).sum())
    return math.log(amp[0] / amp[1]) / t_end / k**2


def test_fv_viscosity_on_periodic_triangles(orc):
    """Eq. 3 with nu = c_s^2 tau_u: a shear wave on a periodic triangulated square
    decays at nu k^2; the spatial error falls by about 4x per halving of h."""
    tau_u = 0.1
    nu = tau_u / 3
    e8 = abs(_fv_shear_nu(orc, 8, tau_u, 0.002, 10.0) / nu - 1)
    e16 = abs(_fv_shear_nu(orc, 16, tau_u, 0.002, 40.0) / nu - 1)
    assert e16 < 0.035
    assert 3.5 < e8 / e16 < 4.5


def _tg_modes(k, x, y):
    """Velocity shape of the Taylor-Green vortex u = U (-cos kx sin ky, sin kx cos ky)."""
    return -np.cos(k * x) * np.sin(k * y), np.sin(k * x) * np.cos(k * y)


def _tg_amplitude(ux, uy, pu, pv):
    return (ux * pu + uy * pv).sum() / (pu**2 + pv**2).sum()


def _lattice_tg_nu(orc, n, tau, steps):
    k, U = 2 * math.pi / n, 1e-3
    X, Y = np.meshgrid(np.arange(n), np.arange(n))  # [y, x]
    pu, pv = _tg_modes(k, X, Y)
    f = np.zeros((n, n, 9))
    for j in range(n):
        for i in range(n):
            f[j, i] = orc.feq(1.0, U * pu[j, i], U * pv[j, i])
    amp = []
    for _ in range(2):
        f = orc.lattice_periodic(f, tau, steps)
        r = f.sum(-1)
        amp.append(_tg_amplitude((f * CX).sum(-1) / r, (f * CY).sum(-1) / r, pu, pv))
    return math.log(amp[0] / amp[1]) / steps / (2 * k**2)


def _fv_tg_nu(orc, n, tau_u, dt, t_end):
    xy, tri, txy = _periodic_mesh(n)
    ops = orc.fv_operators(xy, tri, txy)
    k, U = 2 * math.pi / n, 1e-3
    pu, pv = _tg_modes(k, xy[:, 0], xy[:, 1])
    g = np.array([orc.feq(1.0, U * a, U * b) for a, b in zip(pu, pv)])
    steps = int(round(t_end / dt))
    amp = []
    for _ in range(2):
        for _ in range(steps):
            g = orc.fv_substep(ops, dt, tau_u, g)
        r = g.sum(1)
        amp.append(_tg_amplitude((g * CX).sum(1) / r, (g * CY).sum(1) / r, pu, pv))
    return math.log(amp[0] / amp[1]) / t_end / (2 * k**2)


def test_taylor_green_decay_on_the_lattice(orc):
    """Eq. 1: the Taylor-Green vortex of wavenumber k in both directions decays
    at the closed-form rate 2 nu k^2 with nu = c_s^2 (tau - 1/2); the error
    falls by 4x per halving of the lattice spacing (second order)."""
    tau = 0.8
    nu = (tau - 0.5) / 3
    e16 = abs(_lattice_tg_nu(orc, 16, tau, 60) / nu - 1)
    e32 = abs(_lattice_tg_nu(orc, 32, tau, 240) / nu - 1)
    assert e32 < 2e-3
    assert 3.5 < e16 / e32 < 4.5


def test_taylor_green_decay_on_the_mesh(orc):
    """Eq. 3: the same vortex on a periodic triangulated square decays at
    2 nu k^2 with nu = c_s^2 tau_u, second order in the mesh spacing."""
    tau_u = 0.1
    nu = tau_u / 3
    e8 = abs(_fv_tg_nu(orc, 8, tau_u, 0.002, 10.0) / nu - 1)
    e16 = abs(_fv_tg_nu(orc, 16, tau_u, 0.002, 40.0) / nu - 1)
    assert e16 < 0.08
    assert 3.5 < e8 / e16 < 4.5


def test_fv_uniform_state_is_steady(orc):
    """Eq. 3: a uniform equilibrium is a fixed point (sum_k s_k = 0, and f = f^eq)."""
    xy, tri = _random_patch()
    ops = orc.fv_operators(xy, tri)
    g = np.tile(orc.feq(1.01, 0.03, -0.02), (xy.shape[0], 1))
    g2 = orc.fv_substep(ops, 0.01, 0.05, g)
    assert np.abs(g2 - g).max() < 1e-16


# ------------------------------------------------------------ wall ----------
def test_wall_rule_closed_form(orc):
    """Wall rule: density and non-equilibrium part kept, velocity set to zero."""
    rng = np.random.default_rng(5)
    g = W * (1 + 0.05 * rng.standard_normal(9))
    h = orc.wall_rule(g)
    r0, ux0, uy0 = orc.moments(g)
    r1, ux1, uy1 = orc.moments(h)
    assert r1 == pytest.approx(r0, abs=1e-15)
    assert abs(ux1) < 1e-16 and abs(uy1) < 1e-16
    assert np.allclose(h - orc.feq(r1, 0, 0), g - orc.feq(r0, ux0, uy0), rtol=0, atol=1e-16)


# ------------------------------------------------------------ Eq. 4-7 ------
def _ce_shear_neq(tau, gamma, rho=1.0):
    """First-order Chapman-Enskog non-equilibrium part of a shear flow du_x/dy = gamma
    for a BGK scheme whose stress obeys nu = c_s^2 tau: -tau rho w_i c_ix c_iy gamma / c_s^2."""
    return -tau * 3.0 * rho * W * CX * CY * gamma


@pytest.mark.parametrize("tau_s", [0.5139, 0.5346, 0.8, 1.3])
def test_eq5_maps_lattice_neq_onto_the_finite_volume_scheme(orc, tau_s):
    """Eq. 5-6: for one physical shear flow the lattice carries f^neq with tau_s
    (nu = c_s^2 (tau_s - 1/2)) and the finite-volume scheme with tau_u
    (nu = c_s^2 tau_u, so tau_u = tau_s - 1/2); the interface state must be the
    finite-volume Chapman-Enskog state."""
    gamma, rho, ux, uy = 3e-3, 1.002, 0.04, -0.01
    tau_u = tau_s - 0.5
    q = np.concatenate([[rho, ux, uy], _ce_shear_neq(tau_s, gamma, rho)])
    g = orc.eq5_base(q, tau_s)
    assert np.allclose(g, orc.feq(rho, ux, uy) + _ce_shear_neq(tau_u, gamma, rho), rtol=0, atol=1e-17)


@pytest.mark.parametrize("tau_s", [0.5139, 0.5346, 0.8, 1.3])
def test_eq4_gives_the_lattice_post_collision_state(orc, tau_s):
    """Eq. 4: from the finite-volume Chapman-Enskog state of a shear flow the
    structured interpolation node must hold what a lattice node in the same flow
    holds after collision: f^eq + (1 - 1/tau_s) f^neq,s."""
    gamma, rho, ux, uy = -2e-3, 0.998, 0.05, 0.02
    tau_u = tau_s - 0.5
    q = np.concatenate([[rho, ux, uy], _ce_shear_neq(tau_u, gamma, rho)])
    f = orc.eq4_post(q, tau_s)
    want = orc.feq(rho, ux, uy) + (1 - 1 / tau_s) * _ce_shear_neq(tau_s, gamma, rho)
    assert np.allclose(f, want, rtol=0, atol=1e-17)


# ------------------------------------------------------------ Eq. 8, 9 ------
def test_quad6_weights_reproduce_quadratics(orc):
    """Eq. 8: the six shape functions reproduce every quadratic exactly and sum to 1."""
    rng = np.random.default_rng(6)
    # a triangle plus the far vertices of its three edge neighbours (Fig. 1 layout)
    base = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [1, -1], [-1, 1]], dtype=float)
    for _ in range(10):
        A = np.eye(2) + 0.2 * rng.standard_normal((2, 2))
        pts = base @ A.T * 1.7 + rng.standard_normal(2) * 5
        pts += 0.05 * rng.standard_normal(pts.shape)
        lam = rng.random(3)
        lam /= lam.sum()
        x, y = lam @ pts[:3]
        w = orc.quad6_weights(pts, x, y)
        assert w.sum() == pytest.approx(1.0, abs=1e-13)
        c = rng.standard_normal(6)
        q = lambda X, Y: c[0] + c[1] * X + c[2] * Y + c[3] * X * X + c[4] * X * Y + c[5] * Y * Y
        assert (w * q(pts[:, 0], pts[:, 1])).sum() == pytest.approx(q(x, y), abs=1e-11)


def test_quad6_weights_at_a_donor_are_a_delta(orc):
    pts = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [1, -1], [-1, 1]], dtype=float)
    w = orc.quad6_weights(pts, 1.0, 0.0)
    assert np.allclose(w, [0, 1, 0, 0, 0, 0], atol=1e-14)


def test_biquad9_weights_reproduce_biquadratics(orc):
    """Eq. 9: tensor Lagrange weights reproduce x^a y^b (a, b <= 2) exactly."""
    rng = np.random.default_rng(7)
    off = np.array([(a, b) for b in (-1, 0, 1) for a in (-1, 0, 1)], dtype=float)
    for _ in range(20):
        fx, fy = rng.random(2) - 0.5
        w = orc.biquad9_weights(fx, fy)
        for a in range(3):
            for b in range(3):
                assert (w * off[:, 0] ** a * off[:, 1] ** b).sum() == pytest.approx(fx**a * fy**b, abs=1e-15)
    assert np.allclose(orc.biquad9_weights(0.0, 0.0), np.eye(9)[4], atol=0)


# ------------------------------------------------------------ Eq. 10-11 -----
def _polygon_walls(nv=24, rx=3.0, ry=1.3):
    t = np.linspace(0, 2 * math.pi, nv, endpoint=False)
    xy = np.stack([5 + rx * np.cos(t), 2 + ry * np.sin(t)], 1)
    # fluid outside: walk the body clockwise so the fluid is on the left
    ea = np.arange(nv)[::-1]
    eb = np.roll(ea, -1)
    area = 0.5 * abs(np.sum(xy[:, 0] * np.roll(xy[:, 1], -1) - np.roll(xy[:, 0], -1) * xy[:, 1]))
    return xy, ea, eb, area


def test_force_of_linear_pressure_is_buoyancy(orc):
    """Eq. 10-11 pressure part: p = rho/3 linear in space gives
    F = -(closed integral of p n) = -grad p * body area (divergence theorem;
    the edge-mean rule is exact for a linear field on straight edges)."""
    xy, ea, eb, area = _polygon_walls()
    a, b = 0.013, -0.021
    g = np.array([orc.feq(1 + a * x + b * y, 0.0, 0.0) for x, y in xy])
    F = orc.wall_force(ea, eb, xy, g)
    assert F[0] == pytest.approx(-a / 3 * area, rel=1e-12)
    assert F[1] == pytest.approx(-b / 3 * area, rel=1e-12)


def test_force_of_linear_stress_is_its_divergence(orc):
    """Eq. 10-11 viscous part: with Pi^neq_xx = kappa x (other components 0) the
    traction -Pi.n integrates to -kappa * body area in x (and 0 in y)."""
    xy, ea, eb, area = _polygon_walls()
    kappa = 0.004
    g = []
    for x, _ in xy:
        M = np.array([[kappa * x, 0.0], [0.0, 0.0]])
        neq = 4.5 * W * (CX * CX * M[0, 0] + 2 * CX * CY * M[0, 1] + CY * CY * M[1, 1]
                         - (M[0, 0] + M[1, 1]) / 3)
        g.append(orc.feq(1.0, 0.0, 0.0) + neq)
    F = orc.wall_force(ea, eb, xy, np.array(g))
    assert F[0] == pytest.approx(-kappa * area, rel=1e-12)
    assert abs(F[1]) < 1e-15


def test_airfoil_wall_edges_enclose_the_section(orc):
    """The oracle's wall-edge list walks the whole NACA 0012 surface with the
    fluid on its left: buoyancy of a linear pressure equals -grad p times the
    section area (shoelace of the wall ring)."""
    case = make_case("hlbm_small")
    o = orc.Oracle(case, n_sub=10)
    we = o.table("wall_edges").astype(int).reshape(-1, 2)
    xy = o.table("xy").reshape(-1, 2)
    wall = xy[: case.n_theta]
    area = 0.5 * abs(np.sum(wall[:, 0] * np.roll(wall[:, 1], -1) - np.roll(wall[:, 0], -1) * wall[:, 1]))
    assert we.shape[0] == case.n_theta
    b = 0.01
    g = np.array([orc.feq(1 + b * y, 0.0, 0.0) for _, y in xy])
    F = orc.wall_force(we[:, 0], we[:, 1], xy, g)
    assert F[1] == pytest.approx(-b / 3 * area, rel=1e-10)
    # thickness 12 % of the chord: area of NACA 0012 is about 0.0822 C^2
    assert area == pytest.approx(0.0822 * case.chord**2, rel=0.02)


# ------------------------------------------------------------ whole method --
def _max_dev(o, case, rho0, u0):
    dev = 0.0
    for grid in list(range(case.n_levels)) + ([-1] if case.n_nodes else []):
        r, ux, uy = o.fields(grid)
        m = np.isfinite(r)
        dev = max(dev, np.abs(r[m] - rho0).max(), np.abs(ux[m] - u0).max(), np.abs(uy[m]).max())
    return dev


def test_uniform_stream_through_the_channel_is_steady(orc):
    """Eq. 1 with the outer rules: a uniform stream (rho 1, u = (u0, 0)) is kept exactly."""
    case = make_case("channel", perturb=0.0)
    o = orc.Oracle(case)
    o.step(40)
    assert _max_dev(o, case, 1.0, case.Ma / math.sqrt(3)) < 1e-14


@pytest.mark.parametrize("name", ["hlbm_small", "hlbm_mini2"])
def test_rest_state_is_steady_through_the_coupling(orc, name):
    """Fluid at rest stays exactly at rest through every part of the coupled method:
    wall rule, Eq. 3, Eq. 4 with Eq. 8 and Eq. 5-7 with Eq. 9 (weights summing to
    one), refinement and the outer rules.  (The stream speed u0 = Ma c_s is made
    negligible; Re is scaled with it to keep nu = u0 C / Re = 0.005.)"""
    case = make_case(name, perturb=0.0)
    case.Ma = 1e-30
    case.Re = case.Ma / math.sqrt(3) * case.chord / 0.005
    o = orc.Oracle(case)
    o.step(2)
    assert _max_dev(o, case, 1.0, 0.0) < 1e-14


def test_fv_conserves_mass_and_momentum_on_a_periodic_mesh(orc):
    """Eq. 3 is conservative: on a closed (periodic) mesh sum_P A_P sum_i g_i and
    sum_P A_P sum_i c_i g_i do not change (fluxes between neighbouring control
    volumes cancel; the collision term has zero mass and momentum per node)."""
    xy, tri, txy = _periodic_mesh(6)
    rng = np.random.default_rng(8)
    xy = xy.astype(float)
    ops = orc.fv_operators(xy, tri, txy)
    area = ops[5]
    g = np.array([orc.feq(1 + 0.01 * rng.standard_normal(), *(0.05 * rng.standard_normal(2)))
                  for _ in range(xy.shape[0])])
    g += 1e-3 * rng.standard_normal(g.shape) * W
    m0 = (area[:, None] * g).sum()
    jx0 = (area[:, None] * g * CX).sum()
    jy0 = (area[:, None] * g * CY).sum()
    for _ in range(20):
        g = orc.fv_substep(ops, 0.02, 0.05, g)
    assert (area[:, None] * g).sum() == pytest.approx(m0, rel=1e-14)
    assert (area[:, None] * g * CX).sum() == pytest.approx(jx0, abs=1e-14)
    assert (area[:, None] * g * CY).sum() == pytest.approx(jy0, abs=1e-14)


def _advected_wave_error(orc, two_level, T=200):
    """A transverse wave u = (u0, U sin(k x)) advected through a periodic coarse
    level (64 x 64), optionally with a nested fine box (65 x 65 nodes at (16, 16));
    returns max |u_y - exact| / U over all levels after T coarse steps, with
    exact = U sin(k (x - u0 t)) exp(-nu k^2 t)."""
    from workloads.naca import Case
    n0, Ma = 64, 0.1
    u0 = Ma / math.sqrt(3)
    nu_f = 0.1                       # finest-level viscosity -> nu_0 = 0.05
    lv = [[n0, n0, 0, 0]] + ([[65, 65, 16, 16]] if two_level else [])
    Re = u0 / nu_f if two_level else u0 / (nu_f / 2)
    case = Case("wave", np.asarray(lv, np.int32), np.zeros((0, 2)), np.zeros((0, 3), np.int32),
                np.zeros(0, np.uint8), chord=1.0, pivot=(0, 0), hole=(0, 0, 0, 0), Re=Re, Ma=Ma,
                aoa_deg=0.0, perturb=0.0)
    o = orc.Oracle(case, periodic0=True)
    k, U = 2 * math.pi / n0, 1e-3

    def state(xc, scale, tau):
        # equilibrium plus the first-order Chapman-Enskog part of du_y/dx
        f = orc.feq(1.0, u0, U * math.sin(k * xc))
        return f - tau * 3 * W * CX * CY * U * k * math.cos(k * xc) * scale

    grids = [(0, n0, 0.0, 1.0)] + ([(1, 65, 16.0, 0.5)] if two_level else [])
    for g, nx, ox, sc in grids:
        o.set_populations(g, np.array([state(ox + i * sc, sc, o.tau(g)) for _ in range(nx) for i in range(nx)]))
    o.step(T)
    nu0 = (o.tau(0) - 0.5) / 3
    err = 0.0
    for g, nx, ox, sc in grids:
        _, _, uy = o.fields(g)
        x = ox + np.arange(nx) * sc
        exact = U * np.sin(k * (x - u0 * T)) * math.exp(-nu0 * k * k * T)
        err = max(err, np.abs(uy.reshape(-1, nx) - exact[None, :]).max() / U)
    return err


def test_refinement_interface_matches_the_single_grid_solution(orc):
    """Refinement (factor 2; f^neq rescaled by tau_f/(2 tau_c) coarse->fine and back,
    linear time and quadratic space interpolation at the fine boundary): an advected
    transverse wave crossing a nested fine box stays as close to the analytic
    solution as on the coarse grid alone (within 25 %), and both are close to it."""
    e1 = _advected_wave_error(orc, False)
    e2 = _advected_wave_error(orc, True)
    assert e1 < 1e-3
    assert e2 < 1.25 * e1


# ---------------------------------------------------------------- Eq. 12-13 --
def _wall_input_pose(case):
    """Wall nodes (ascending index) in the input (zero-incidence) pose:
    x/C from the leading edge and side, from the case geometry alone."""
    w = np.flatnonzero(case.kind == 1)
    le_x = case.pivot[0] - 0.25 * case.chord
    xc = (case.xy[w, 0] - le_x) / case.chord
    side = np.where(case.xy[w, 1] - case.pivot[1] >= 0.0, 1.0, -1.0)
    return w, xc, side


def test_wall_coefficients_reassemble_the_wall_force(orc):
    """Eq. 12-13 per wall node, weighted by |N_P| and recombined with the node
    normal and downstream tangent, give back the wall force of Eq. 10-11:
    sum_P |N_P| [(-C_p + C_n) n + C_f s] / C = (C_D, C_L)."""
    case = make_case("hlbm_small", aoa_deg=8.0)
    o = orc.Oracle(case)
    o.step(30)
    w = o.wall_coeffs()
    cd, cl = o.forces()
    F = (w[:, 5, None] * ((-w[:, 2] + w[:, 4])[:, None] * w[:, 6:8] + w[:, 3, None] * w[:, 8:10])).sum(0)
    F /= case.chord
    assert abs(F[0] - cd[-1]) <= 1e-12 * abs(cd[-1])
    assert abs(F[1] - cl[-1]) <= 1e-12 * abs(cd[-1])
    assert np.ptp(w[:, 3]) > 0.1 and np.ptp(w[:, 2]) > 0.1  # a developing flow, not a trivial state


def test_wall_geometry_of_the_coefficients(orc):
    """Normals point away from the body (a convex section: away from mid-chord),
    tangents are unit, orthogonal and downstream; x/C and side follow the
    input pose."""
    for aoa in (0.0, 8.0):
        case = make_case("hlbm_small", aoa_deg=aoa)
        o = orc.Oracle(case)
        w = o.wall_coeffs()
        idx, xc, side = _wall_input_pose(case)
        assert w.shape == (idx.size, 10)
        on_chord = np.abs(case.xy[idx, 1] - case.pivot[1]) < 1e-9 * case.chord  # leading / trailing edge
        assert np.allclose(w[:, 0], xc, atol=1e-12)
        assert np.array_equal(w[~on_chord, 1], side[~on_chord]) and on_chord.sum() <= 2
        al = np.radians(aoa)
        chord_dir = np.array([np.cos(al), -np.sin(al)])     # rotated by -alpha (nose up)
        mid = np.array(case.pivot) + 0.25 * case.chord * chord_dir
        # rotated wall positions from the input pose
        d = case.xy[idx] - np.array(case.pivot)
        pos = np.array(case.pivot) + np.stack([np.cos(al) * d[:, 0] + np.sin(al) * d[:, 1],
                                               np.cos(al) * d[:, 1] - np.sin(al) * d[:, 0]], axis=1)
        n, s = w[:, 6:8], w[:, 8:10]
        assert np.all(((pos - mid) * n).sum(1) > 0)
        assert np.allclose(np.hypot(*n.T), 1) and np.allclose(np.hypot(*s.T), 1)
        assert np.allclose((n * s).sum(1), 0, atol=1e-14)
        assert np.all(s @ chord_dir >= 0)


def test_wall_coefficients_of_prescribed_states(orc):
    """Uniform pressure at rest: C_p = (rho - 1) / 3 / (u0^2 / 2), no traction.
    Pure shear f^neq (only Pi_xy = sigma): traction -sigma (n_y, n_x)."""
    case = make_case("hlbm_small")
    o = orc.Oracle(case)
    q = 0.5 * (case.Ma / np.sqrt(3.0)) ** 2
    rho = 1.003
    f = np.tile(orc.feq(rho, 0.0, 0.0), (case.n_nodes, 1))
    o.set_populations(-1, f)
    w = o.wall_coeffs()
    assert np.allclose(w[:, 2], (rho - 1.0) / 3.0 / q, rtol=1e-12)
    assert np.abs(w[:, 3:5]).max() <= 1e-12
    sigma = 2e-5
    neq = np.zeros(9)
    neq[[5, 7]] = sigma / 4.0      # c_x c_y = +1
    neq[[6, 8]] = -sigma / 4.0     # c_x c_y = -1
    o.set_populations(-1, np.tile(orc.feq(1.0, 0.0, 0.0) + neq, (case.n_nodes, 1)))
    w = o.wall_coeffs()
    n, s = w[:, 6:8], w[:, 8:10]
    t = -sigma * np.stack([n[:, 1], n[:, 0]], axis=1)
    assert np.allclose(w[:, 3], (t * s).sum(1) / q, rtol=1e-9, atol=1e-12)
    assert np.allclose(w[:, 4], (t * n).sum(1) / q, rtol=1e-9, atol=1e-12)
    assert np.abs(w[:, 2]).max() <= 1e-12


def test_fv_window_is_the_composition_of_the_pinned_primitives(orc):
    """The adjoint's test functional (orc_fv_window) is, step for step, the
    separately pinned population-form pieces: Eq. 3 sub-steps, the wall rule
    on wall nodes, Eq. 5-7 interface rows built from the Eq. 9 data of the
    current finest lattice after every sub-step but the last of a finest
    step, and the Eq. 10-11 wall force over 1/2 u0^2 C."""
    case = make_case("hlbm_mini2", aoa_deg=4.0)
    o = orc.Oracle(case)
    o.step(1)
    ops = (o.table("rowptr").astype(np.int32), o.table("col").astype(np.int32), o.table("sx"), o.table("sy"),
           o.table("cc"), None)
    L = case.n_levels - 1
    tau_s, tau_u, dt = o.tau(L), o.tau(-1), 1.0 / o.n_sub
    lat = o.populations(L)
    ring = o.table("ring").astype(int)
    don = o.table("ring_don").astype(int).reshape(-1, 9)
    w9 = o.table("ring_w").reshape(-1, 9)

    def q_of(f):
        rho, ux, uy = orc.moments(f)
        return np.concatenate([[rho, ux, uy], f - orc.feq(rho, ux, uy)])

    ring_pop = np.array([orc.eq5_base(sum(w9[r, k] * q_of(lat[don[r, k]]) for k in range(9)), tau_s)
                         for r in range(len(ring))])
    wall = np.flatnonzero(np.asarray(case.kind) == 1)
    edges = o.table("wall_edges").astype(np.int32).reshape(-1, 2)
    xy = o.table("xy").reshape(-1, 2)
    u0 = case.Ma / math.sqrt(3.0)
    qdyn = 0.5 * u0 * u0 * case.chord
    for M, wd, wl in ((1, 1.0, 0.0), (4, 0.3, 1.0), (o.n_sub, 1.0, 0.0)):
        g = o.populations(-1)
        for m in range(M):
            g = orc.fv_substep(ops, dt, tau_u, g)
            for p in wall:
                g[p] = orc.wall_rule(g[p])
            if m < o.n_sub - 1:
                g[ring] = ring_pop
        F = orc.wall_force(edges[:, 0], edges[:, 1], xy, g)
        expect = (wd * F[0] + wl * F[1]) / qdyn
        got = o.fv_window(M, wd, wl)
        assert abs(got - expect) <= 1e-10 * max(1.0, abs(expect)), (M, got, expect)
    # rebuilding the geometry without moving it changes nothing but rounding
    J0 = o.fv_window(3, 1.0, 0.0)
    assert abs(o.fv_window(3, 1.0, 0.0, dxy=np.zeros((case.n_nodes, 2)), hx=1.0) - J0) <= 1e-13 * abs(J0)
    # the window leaves the oracle's state alone
    assert np.array_equal(o.populations(-1), o.populations(-1))
    before = o.populations(-1)
    o.fv_window(3)
    assert np.array_equal(before, o.populations(-1))
