"""NACA 0012 O-mesh and nested Cartesian levels (geometry inputs only).

Geometry follows the problem statement of Di Ilio et al. (Section 4,
"Problem setup"): a NACA 0012 airfoil placed symmetrically between the top
and bottom boundaries, a body-fitted triangular mesh whose outer boundary is
an ellipse, an inner interface curve that is also an ellipse, and nested
Cartesian boxes refined by a factor of two whose innermost box has unit
spacing and overlaps the triangular mesh.

All coordinates are in finest-level lattice units in the frame of the finest
level (its node (i, j) sits at (i, j)), in the zero-incidence pose; the solver
rotates mesh and hole by the angle of attack itself.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Node kinds of the triangular mesh (the C ABI uses the same codes).
KIND_FLUID = 0
KIND_WALL = 1
KIND_RING = 2


def naca0012_half_thickness(x):
    """Half thickness of the closed-trailing-edge NACA 0012 section, chord 1.

    t(x) = 0.6 (0.2969 sqrt(x) - 0.1260 x - 0.3516 x^2 + 0.2843 x^3 - 0.1036 x^4);
    the last coefficient closes the trailing edge (t(1) = 0).
    """
    x = np.asarray(x, dtype=np.float64)
    return 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2
                  + 0.2843 * x**3 - 0.1036 * x**4)


def o_mesh(chord, leading_edge, n_theta, n_layers, stretch, ell_a, ell_b):
    """Body-fitted O-type triangular mesh around a NACA 0012 section.

    Surface node k (k = 0 .. n_theta-1) has parameter theta_k = 2 pi k / n_theta
    and, with u = theta/pi on the upper surface (theta <= pi) and
    u = 2 - theta/pi on the lower one, chord position
    x = a (1 + cos(pi u)) / 2 + (1 - a) (1 - u)^2, where a is chosen so that
    the wall spacing at the trailing edge equals the first-layer spacing
    there (k = 0 is the trailing edge, k = n_theta/2 the leading edge).
    Index k runs counter-clockwise.  The
    matching outer-ellipse point (centred at mid-chord) has the same
    parameter theta.  Mesh line k is the cubic Hermite curve from the surface
    point (leaving along the outward surface normal) to the ellipse point;
    ring j (0 .. n_layers) sits at curve parameter
    s_j = (r^j - 1)/(r^n_layers - 1), r = stretch (uniform if r == 1).

    Returns (xy[N,2] float64, tri[T,3] int32 counter-clockwise,
    kind[N] uint8) with node index j * n_theta + k; ring 0 is the wall and
    ring n_layers is the outer (overlap) ring.
    """
    if n_theta % 2:
        raise ValueError("n_theta must be even")
    le = np.asarray(leading_edge, dtype=np.float64)
    j = np.arange(n_layers + 1, dtype=np.float64)
    if stretch == 1.0:
        s = j / n_layers
    else:
        s = (stretch**j - 1.0) / (stretch**n_layers - 1.0)
    # trailing-edge wall spacing = first-layer spacing there (square cells at
    # the sharp trailing edge instead of slivers)
    h1 = s[1] * (ell_a - 0.5 * chord)
    alpha = min(1.0, max(0.0, 1.0 - h1 * n_theta / (4.0 * chord)))
    theta = 2.0 * math.pi * np.arange(n_theta) / n_theta
    u = np.where(theta <= math.pi, theta, 2.0 * math.pi - theta) / math.pi
    xc = alpha * 0.5 * (1.0 + np.cos(math.pi * u)) + (1.0 - alpha) * (1.0 - u) ** 2
    sign = np.where(theta <= math.pi, 1.0, -1.0)
    surf = np.stack([le[0] + chord * xc,
                     le[1] + sign * chord * naca0012_half_thickness(xc)], axis=1)
    mid = np.array([le[0] + 0.5 * chord, le[1]])
    outer = np.stack([mid[0] + ell_a * np.cos(theta),
                      mid[1] + ell_b * np.sin(theta)], axis=1)
    # Mesh line k: cubic Hermite curve from surface point S_k, leaving along the
    # outward surface normal, to ellipse point E_k, arriving along E_k - S_k.
    tang = np.roll(surf, -1, axis=0) - np.roll(surf, 1, axis=0)
    normal = np.stack([tang[:, 1], -tang[:, 0]], axis=1)
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    span = outer - surf
    length = np.linalg.norm(span, axis=1, keepdims=True)
    t0 = length * normal
    t1 = span
    ss = s[:, None, None]
    h00 = 2 * ss**3 - 3 * ss**2 + 1
    h10 = ss**3 - 2 * ss**2 + ss
    h01 = -2 * ss**3 + 3 * ss**2
    h11 = ss**3 - ss**2
    xy = h00 * surf[None] + h10 * t0[None] + h01 * outer[None] + h11 * t1[None]
    xy = xy.reshape(-1, 2)

    # Quad (k, j) has corners a = (j, k), b = (j, k+1), c = (j+1, k), d = (j+1, k+1).
    # Index k runs counter-clockwise and j outward, so (a, c, b) is counter-
    # clockwise.  Each quad is split along the diagonal that gives the larger
    # smallest altitude (this avoids slivers at the sharp trailing edge).
    jj, kk = np.meshgrid(np.arange(n_layers), np.arange(n_theta), indexing="ij")
    a = (jj * n_theta + kk).ravel()
    b = (jj * n_theta + (kk + 1) % n_theta).ravel()
    c = ((jj + 1) * n_theta + kk).ravel()
    d = ((jj + 1) * n_theta + (kk + 1) % n_theta).ravel()

    def min_altitude(i0, i1, i2):
        p0, p1, p2 = xy[i0], xy[i1], xy[i2]
        a2 = ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1])
              - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0]))
        e01 = np.hypot(p1[:, 0] - p0[:, 0], p1[:, 1] - p0[:, 1])
        e12 = np.hypot(p2[:, 0] - p1[:, 0], p2[:, 1] - p1[:, 1])
        e20 = np.hypot(p0[:, 0] - p2[:, 0], p0[:, 1] - p2[:, 1])
        return a2 / np.maximum(np.maximum(e01, e12), e20)

    q1 = np.minimum(min_altitude(a, c, b), min_altitude(b, c, d))
    q2 = np.minimum(min_altitude(a, c, d), min_altitude(a, d, b))
    first = (q1 >= q2)[:, None]
    t0 = np.where(first, np.stack([a, c, b], axis=1), np.stack([a, c, d], axis=1))
    t1 = np.where(first, np.stack([b, c, d], axis=1), np.stack([a, d, b], axis=1))
    tris = np.stack([t0, t1], axis=1).reshape(-1, 3)
    tri = np.asarray(tris, dtype=np.int32)
    kind = np.zeros(xy.shape[0], dtype=np.uint8)
    kind[:n_theta] = KIND_WALL
    kind[n_layers * n_theta:] = KIND_RING
    p = xy[tri]
    area2 = ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
             - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    if not np.all(area2 > 0):
        raise ValueError("O-mesh has inverted triangles; adjust its parameters")
    return xy, tri, kind


def thickness_modes(case, n_modes=12):
    """Node displacement fields of thickness bumps, [n_modes, N, 2] in the
    zero-incidence frame: mode m (1 .. n_modes) adds sin(m pi x) (x = chord
    fraction) to the half thickness t(x), i.e. moves wall node k by
    (0, +-C sin(m pi x_k)) (+ upper, - lower surface), and moves the node of
    ring j on the same mesh line by that times 1 - j / n_layers (linear
    blending: the outer interface ring stays in place)."""
    if not case.n_theta or not case.n_layers:
        raise ValueError("thickness modes need an O-mesh case")
    nt, nl = case.n_theta, case.n_layers
    le_x, le_y = case.pivot[0] - 0.25 * case.chord, case.pivot[1]
    wall = case.xy[:nt]
    xc = np.clip((wall[:, 0] - le_x) / case.chord, 0.0, 1.0)
    sign = np.where(np.arange(nt) <= nt // 2, 1.0, -1.0)
    sign[wall[:, 1] < le_y] = -1.0
    blend = 1.0 - np.arange(nl + 1, dtype=np.float64) / nl
    out = np.zeros((n_modes, case.n_nodes, 2))
    for m in range(1, n_modes + 1):
        dy = sign * case.chord * np.sin(m * math.pi * xc)
        out[m - 1, :, 1] = (blend[:, None] * dy[None, :]).reshape(-1)
    return out


@dataclasses.dataclass
class Case:
    """One HLBM problem: Cartesian levels, triangular mesh and flow parameters."""

    name: str
    levels: np.ndarray          # [L,4] int32: nx, ny, ox, oy (origin in parent-level nodes)
    xy: np.ndarray              # [N,2] float64, finest-level units, zero-incidence pose
    tri: np.ndarray             # [T,3] int32, counter-clockwise
    kind: np.ndarray            # [N] uint8: 0 fluid, 1 wall, 2 outer (overlap) ring
    chord: float
    pivot: tuple                # rotation centre (quarter chord)
    hole: tuple                 # inner interface ellipse (cx, cy, a, b)
    Re: float
    Ma: float
    aoa_deg: float
    n_sub: int = 0              # 0: chosen by the solver from its stability bound
    seed: int = 0
    perturb: float = 1e-4
    steps: int = 100            # coarse steps of the nominal run
    n_theta: int = 0
    n_layers: int = 0
    fv_filter: float = 0.0      # odd-even filter of the mesh state per finest step (0: off)

    @property
    def n_levels(self):
        return int(self.levels.shape[0])

    @property
    def n_nodes(self):
        return int(self.xy.shape[0])


def _mesh_case(name, levels, chord, mid, n_theta, n_layers, stretch, ell_b_ratio,
               overlap, Re, Ma, aoa_deg, steps, **kw):
    le = (mid[0] - 0.5 * chord, mid[1])
    ell_a, ell_b = chord, ell_b_ratio * chord
    xy, tri, kind = o_mesh(chord, le, n_theta, n_layers, stretch, ell_a, ell_b)
    return Case(name=name, levels=np.asarray(levels, dtype=np.int32), xy=xy, tri=tri,
                kind=kind, chord=float(chord), pivot=(le[0] + 0.25 * chord, le[1]),
                hole=(mid[0], mid[1], ell_a - overlap, ell_b - overlap), Re=float(Re),
                Ma=float(Ma), aoa_deg=float(aoa_deg), steps=steps, n_theta=n_theta,
                n_layers=n_layers, **kw)


def _channel(name, nx, ny, Re, Ma, steps, chord=None):
    return Case(name=name, levels=np.asarray([[nx, ny, 0, 0]], dtype=np.int32),
                xy=np.zeros((0, 2)), tri=np.zeros((0, 3), dtype=np.int32),
                kind=np.zeros(0, dtype=np.uint8), chord=float(ny if chord is None else chord),
                pivot=(0.0, 0.0), hole=(0.0, 0.0, 0.0, 0.0), Re=float(Re), Ma=float(Ma), aoa_deg=0.0,
                steps=steps)


def square_patch(x0, y0, width, m):
    """Body-free triangular mesh of a square: (m+1) x (m+1) nodes of spacing
    width/m from (x0, y0), each cell split into two triangles along
    alternating diagonals.  Every node is fluid except the square's boundary,
    which is the outer (overlap) ring.  Returns (xy, tri, kind) as o_mesh."""
    h = width / m
    i, j = np.meshgrid(np.arange(m + 1), np.arange(m + 1))
    xy = np.stack([x0 + h * i.ravel(), y0 + h * j.ravel()], axis=1).astype(np.float64)
    tri = []
    for jj in range(m):
        for ii in range(m):
            a = jj * (m + 1) + ii
            b, c = a + 1, a + m + 1
            d = c + 1
            tri += [(a, b, d), (a, d, c)] if (ii + jj) % 2 == 0 else [(a, b, c), (b, d, c)]
    edge = (i.ravel() == 0) | (i.ravel() == m) | (j.ravel() == 0) | (j.ravel() == m)
    kind = np.where(edge, KIND_RING, KIND_FLUID).astype(np.uint8)
    return xy, np.asarray(tri, dtype=np.int32), kind


def patch_case(n0=64, m=32, width=24.0, centre=(32.3, 32.47), nu=0.1, Ma=0.1, mesh=True, name="patch"):
    """One n0 x n0 lattice level with a body-free square mesh (square_patch,
    m x m cells of side `width`, centred at `centre`, placed off the lattice
    nodes) whose circular hole is inset 4 cells from the ring: the overlap
    coupling (Eq. 4-9) with nothing else of the airfoil case.  nu is the
    lattice viscosity (the solver derives Re = u0 C / nu with C = 1).
    mesh=False gives the same lattice without the mesh."""
    u0 = Ma / math.sqrt(3.0)
    lv = np.asarray([[n0, n0, 0, 0]], dtype=np.int32)
    if mesh:
        xy, tri, kind = square_patch(centre[0] - 0.5 * width, centre[1] - 0.5 * width, width, m)
        r = 0.5 * width - 4.0
        hole = (centre[0], centre[1], r, r)
    else:
        xy, tri, kind = np.zeros((0, 2)), np.zeros((0, 3), dtype=np.int32), np.zeros(0, dtype=np.uint8)
        hole = (0.0, 0.0, 0.0, 0.0)
    return Case(name=name, levels=lv, xy=xy, tri=tri, kind=kind, chord=1.0, pivot=tuple(centre), hole=hole,
                Re=u0 / nu, Ma=float(Ma), aoa_deg=0.0, perturb=0.0, steps=200)


def uniform_equivalent(case):
    """The lattice an equivalent plain LBM would use for `case` (Eq. 14's
    T_eq): one level at the finest resolution over the whole domain, with the
    same viscosity in finest units (same chord length scale and Re)."""
    f = 2 ** (case.n_levels - 1)
    nx, ny = int(case.levels[0][0]), int(case.levels[0][1])
    return _channel(case.name + "_uniform", (nx - 1) * f + 1, (ny - 1) * f + 1, case.Re, case.Ma,
                    case.steps, chord=case.chord)


def make_case(name, aoa_deg=None, **overrides):
    """Build a named configuration (see CONFIGS); keyword overrides patch the Case."""
    if name not in CONFIGS:
        raise KeyError(f"unknown configuration {name!r}; known: {sorted(CONFIGS)}")
    case = CONFIGS[name]()
    if aoa_deg is not None:
        case.aoa_deg = float(aoa_deg)
    for k, v in overrides.items():
        if not hasattr(case, k):
            raise AttributeError(k)
        setattr(case, k, v)
    return case


CONFIGS = {
    # Plain HLBM, small: one 200x100 level, chord 40, 80 x 65-ring O-mesh
    # (64 layers stretched 1.05), outer ring overlapping the lattice by 4 cells,
    # Re 500, Ma 0.1, 2000 steps.
    "hlbm_small": lambda: _mesh_case(
        "hlbm_small", [[200, 100, 0, 0]], chord=40.0, mid=(70.0, 50.0),
        n_theta=80, n_layers=64, stretch=1.05, ell_b_ratio=0.6, overlap=4.0,
        Re=500.0, Ma=0.1, aoa_deg=0.0, steps=2000),
    # Two-level mini case for refinement parity: 96x48 coarse level and one
    # 97x65 fine box, chord 24 finest units.
    "hlbm_mini2": lambda: _mesh_case(
        "hlbm_mini2", [[96, 48, 0, 0], [97, 65, 24, 8]], chord=24.0, mid=(40.0, 32.0),
        n_theta=48, n_layers=20, stretch=1.08, ell_b_ratio=0.6, overlap=4.0,
        Re=200.0, Ma=0.1, aoa_deg=0.0, steps=100),
    # Three-level mini case (two nested refinement boxes) for parity and
    # adjoint tests: 64x40 coarse level, an 81x57 box and the 97x65 finest box
    # of hlbm_mini2 inside it, chord 24 finest units.
    "hlbm_mini3": lambda: _mesh_case(
        "hlbm_mini3", [[64, 40, 0, 0], [81, 57, 12, 6], [97, 65, 16, 12]], chord=24.0, mid=(40.0, 32.0),
        n_theta=48, n_layers=20, stretch=1.08, ell_b_ratio=0.6, overlap=4.0,
        Re=200.0, Ma=0.1, aoa_deg=0.0, steps=100),
    # Single case: 2048x1024 coarse level with two nested factor-2 boxes of
    # 1025x513 nodes, chord 200 finest units, 1024 x 196-ring O-mesh
    # (200 704 nodes), Re 1000, Ma 0.1.
    "hlbm_single": lambda: _mesh_case(
        "hlbm_single", [[2048, 1024, 0, 0], [1025, 513, 512, 384], [1025, 513, 256, 128]],
        chord=200.0, mid=(412.0, 256.0), n_theta=1024, n_layers=195, stretch=1.01,
        ell_b_ratio=0.6, overlap=4.0, Re=1000.0, Ma=0.1, aoa_deg=0.0, steps=100000),
    # Large Re: 8192x4096 coarse level with three nested factor-2 boxes of
    # 4097x2049 nodes (each half its parent's extent per dimension), chord 800
    # finest units, 4096 x 367-ring O-mesh (1 503 232 nodes, uniform layers: the
    # first one about 0.002 chord), Re 10^4, Ma 0.1.
    "hlbm_large": lambda: _mesh_case(
        "hlbm_large", [[8192, 4096, 0, 0], [4097, 2049, 2048, 1536], [4097, 2049, 1024, 512],
                       [4097, 2049, 1024, 512]],
        chord=800.0, mid=(1648.0, 1024.0), n_theta=4096, n_layers=366, stretch=1.0,
        ell_b_ratio=0.6, overlap=4.0, Re=1e4, Ma=0.1, aoa_deg=0.0, steps=200000),
    # The large-Re case's 1.5 M-node mesh (as in "hlbm_large") inside a single
    # 1800x1100 level at the finest resolution: the same finite-volume work in
    # a few hundred MB of device memory (finite-volume kernel profiles).
    "hlbm_large_fv": lambda: _mesh_case(
        "hlbm_large_fv", [[1800, 1100, 0, 0]], chord=800.0, mid=(900.0, 550.0), n_theta=4096, n_layers=366,
        stretch=1.0, ell_b_ratio=0.6, overlap=4.0, Re=1e4, Ma=0.1, aoa_deg=0.0, steps=100),
    # Body-free coupling: a 64x64 level with a 33x33-node square mesh over a
    # circular hole (overlap band only, no airfoil); perturbed density so that
    # waves cross the band.
    "patch": lambda: dataclasses.replace(patch_case(), perturb=1e-4),
    # Mesh-less channel (lattice and outer boundaries only).
    "channel": lambda: _channel("channel", 64, 32, Re=100.0, Ma=0.1, steps=100),
}


# Batched ensemble: 16 angles of attack (0..15 degrees) x Re {500, 1000, 2000,
# 5000}; per Re a single-level lattice and mesh of increasing size with chord
# C = nx / 10: (nx, ny, N_theta, layers) = (512, 256, 256, 79) -> 20 480 mesh
# nodes, (1024, 512, 512, 146) -> 75 264, (1536, 768, 768, 195) -> 150 528,
# (2048, 1024, 1024, 292) -> 300 032.
ENSEMBLE_SIZES = {500.0: (512, 256, 256, 79), 1000.0: (1024, 512, 512, 146),
                  2000.0: (1536, 768, 768, 195), 5000.0: (2048, 1024, 1024, 292)}


def ensemble_case(Re, aoa_deg):
    """One case of the batched ensemble (see ENSEMBLE_SIZES)."""
    nx, ny, n_theta, n_layers = ENSEMBLE_SIZES[float(Re)]
    chord = nx / 10.0
    return _mesh_case(f"ensemble_Re{int(Re)}_a{aoa_deg:g}", [[nx, ny, 0, 0]], chord=chord,
                      mid=(0.3 * nx, 0.5 * ny), n_theta=n_theta, n_layers=n_layers, stretch=1.01,
                      ell_b_ratio=0.6, overlap=4.0, Re=float(Re), Ma=0.1, aoa_deg=float(aoa_deg), steps=50000)


def ensemble(aoas=tuple(range(16)), res=(500.0, 1000.0, 2000.0, 5000.0)):
    """The batched ensemble's cases, Re-major."""
    return [ensemble_case(Re, a) for Re in res for a in aoas]
