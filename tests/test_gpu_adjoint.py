"""Discrete adjoint of the finite-volume part (hlbm_fv_adjoint, FP64) against
the oracle: the functional matches the oracle's window, and the gradients,
contracted with random directions, match central differences of the oracle's
window (orc_fv_window) in the initial populations and in the Eq. 3 operator
entries."""
import numpy as np
import pytest

from workloads import make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_10487_gb300 import build
    build.build()
    import paper_2006_10487_gb300 as H
    return H


@pytest.fixture(scope="module")
def pair(H):
    import oracle
    case = make_case("hlbm_mini2", aoa_deg=4.0)
    s = H.Solver(case, precision="fp64")
    o = oracle.Oracle(case)
    s.step(2)
    o.step(2)
    return case, s, o


def _directions(case, s, seed):
    rng = np.random.default_rng(seed)
    dg = rng.standard_normal((case.n_nodes, 9)) * 1e-3
    rp = s_tables(s, "rowptr").astype(int)
    col = s_tables(s, "col").astype(int)
    mag = np.abs(np.stack([s_tables(s, "sx"), s_tables(s, "sy"), s_tables(s, "cc")], axis=1))
    dc = rng.standard_normal((len(col), 3)) * mag
    for p in range(case.n_nodes):  # self entries are fixed by construction
        for e in range(rp[p], rp[p + 1]):
            if col[e] == p:
                dc[e] = 0.0
    return dg, dc


_TABLES = {}


def s_tables(s, name):
    import paper_2006_10487_gb300 as H
    key = (id(s.case), name)
    if key not in _TABLES:
        _TABLES[key] = H.hlbm_inspect(s.case, name, precision="fp64")
    return _TABLES[key]


@pytest.mark.parametrize("M,wd,wl", [(1, 1.0, 0.0), (5, 0.0, 1.0), (None, 1.0, 0.5)])
def test_fv_adjoint_matches_oracle_finite_differences(H, pair, M, wd, wl):
    case, s, o = pair
    M = o.n_sub if M is None else M
    f_before = s.fields(-1)
    J, gg, gc, gx, da = s.fv_adjoint(M, wd, wl)
    # the window ran on scratch: the solver's state is untouched
    for a, b in zip(f_before, s.fields(-1)):
        assert np.array_equal(a, b)
    J_o = o.fv_window(M, wd, wl)
    assert abs(J - J_o) <= 1e-11 * max(1.0, abs(J_o)), (J, J_o)
    dg, dc = _directions(case, s, seed=M)
    hg = 1e-4
    fd_g = (o.fv_window(M, wd, wl, dg=dg, hg=hg) - o.fv_window(M, wd, wl, dg=dg, hg=-hg)) / (2 * hg)
    ad_g = float(np.sum(gg * dg))
    assert abs(ad_g - fd_g) <= 1e-6 * abs(fd_g) + 1e-10, (ad_g, fd_g)
    hc = 1e-5
    fd_c = (o.fv_window(M, wd, wl, dcoef=dc, hc=hc) - o.fv_window(M, wd, wl, dcoef=dc, hc=-hc)) / (2 * hc)
    ad_c = float(np.sum(gc * dc))
    assert abs(ad_c - fd_c) <= 1e-6 * abs(fd_c) + 1e-10, (ad_c, fd_c)
    # geometry: node coordinates (input frame) and the angle of attack, the
    # oracle rebuilding its operators and wall normals for the moved mesh
    dxy = np.random.default_rng(100 + M).standard_normal((case.n_nodes, 2))
    hx = 1e-5
    fd_x = (o.fv_window(M, wd, wl, dxy=dxy, hx=hx) - o.fv_window(M, wd, wl, dxy=dxy, hx=-hx)) / (2 * hx)
    ad_x = float(np.sum(gx * dxy))
    assert abs(ad_x - fd_x) <= 1e-6 * abs(fd_x) + 1e-9, (ad_x, fd_x)
    ha = 1e-3
    fd_a = (o.fv_window(M, wd, wl, daoa=ha) - o.fv_window(M, wd, wl, daoa=-ha)) / (2 * ha)
    assert abs(da - fd_a) <= 1e-6 * abs(fd_a) + 1e-9, (da, fd_a)
    # self entries carry no gradient
    rp, col = s_tables(s, "rowptr").astype(int), s_tables(s, "col").astype(int)
    diag = np.array([e for p in range(case.n_nodes) for e in range(rp[p], rp[p + 1]) if col[e] == p])
    assert np.all(gc[diag] == 0.0)


def test_thickness_and_incidence_gradients_match_oracle(H, pair):
    """dJ/dA_m of the 12 thickness bumps (workloads.thickness_modes: the
    node displacement of t(x) += A_m sin(m pi x), blended to zero at the
    interface ring) and dJ/d(angle of attack), over a full finest step's
    sub-steps, against oracle central differences."""
    from workloads import thickness_modes
    case, s, o = pair
    M = o.n_sub
    J, gg, gc, gx, da = s.fv_adjoint(M, 1.0, 0.0)
    modes = thickness_modes(case)
    h = 1e-6
    for m, field in enumerate(modes):
        ad = float(np.sum(gx * field))
        fd = (o.fv_window(M, 1.0, 0.0, dxy=field, hx=h) - o.fv_window(M, 1.0, 0.0, dxy=field, hx=-h)) / (2 * h)
        assert abs(ad - fd) <= 1e-5 * abs(fd) + 1e-7, (m + 1, ad, fd)


def test_fv_adjoint_is_deterministic_and_localised(H, pair):
    """Two calls agree bitwise; after one sub-step only wall nodes and their
    neighbours carry a state gradient (the functional reads wall nodes)."""
    case, s, o = pair
    J1, g1, c1, x1, a1 = s.fv_adjoint(1)
    J2, g2, c2, x2, a2 = s.fv_adjoint(1)
    assert J1 == J2 and np.array_equal(g1, g2) and np.array_equal(c1, c2)
    assert np.array_equal(x1, x2) and a1 == a2
    rp, col = s_tables(s, "rowptr").astype(int), s_tables(s, "col").astype(int)
    wall = set(np.flatnonzero(np.asarray(case.kind) == 1))
    near = set(wall)
    for p in wall:
        near.update(col[rp[p]:rp[p + 1]])
    nz = set(np.flatnonzero(np.any(g1 != 0.0, axis=1)))
    assert nz <= near and wall <= nz


def test_fv_adjoint_rejects_what_it_does_not_cover(H):
    case = make_case("hlbm_mini2")
    s = H.Solver(case, precision="fp32")
    with pytest.raises(H.HlbmError) as e:
        s.fv_adjoint(1)
    assert e.value.code == H.HLBM_ENOTIMPL
    s64 = H.Solver(case, precision="fp64")
    for bad in (0, int(s64.info("n_sub")) + 1):
        with pytest.raises(H.HlbmError) as e:
            s64.fv_adjoint(bad)
        assert e.value.code == H.HLBM_EINVAL


# ---------------------------------------------------------------------------
# Adjoint of whole coarse steps (single level): lattice, outer conditions,
# overlap interpolations, interface rows, finite-volume sub-steps, forces.

@pytest.fixture(scope="module")
def small(H):
    case = make_case("hlbm_small", aoa_deg=4.0)
    s = H.Solver(case, precision="fp64")
    s.step(1)
    s.forces()  # drain
    return case, s


def _oracle_mean_force(case, K, wd, wl, dlat=None, dmesh=None, h=0.0, skip=0):
    """Mean of wd C_D + wl C_L over coarse steps 2 + skip .. K + 1 of the
    oracle, its state after step 1 moved by h * (dlat, dmesh) in populations."""
    import oracle
    o = oracle.Oracle(case)
    o.step(1)
    if dlat is not None:
        f = o.populations(0)
        o.set_populations(0, np.where(np.isnan(f), f, f + h * dlat))
    if dmesh is not None:
        o.set_populations(-1, o.populations(-1) + h * dmesh)
    o.step(K)
    cd, cl = o.forces()
    return float(np.mean(wd * cd[1 + skip:] + wl * cl[1 + skip:]))


@pytest.mark.parametrize("K,wd,wl,skip", [(1, 1.0, 0.0, 0), (3, 0.4, 1.0, 0), (3, 1.0, 0.0, 2)])
def test_coupled_adjoint_matches_oracle_finite_differences(H, small, K, wd, wl, skip):
    case, s = small
    before = [a.copy() for a in s.fields(0)] + [a.copy() for a in s.fields(-1)]
    J, (gl,), gm, _, _ = s.adjoint(K, wd, wl, skip)
    after = list(s.fields(0)) + list(s.fields(-1))
    for a, b in zip(before, after):
        assert np.array_equal(a, b, equal_nan=True)
    assert abs(J - _oracle_mean_force(case, K, wd, wl, skip=skip)) <= 1e-10 * max(1.0, abs(J))
    rng = np.random.default_rng(7 + K + skip)
    nx, ny = (int(v) for v in case.levels[0][:2])
    dlat = rng.standard_normal((nx * ny, 9)) * 1e-3
    dmesh = rng.standard_normal((case.n_nodes, 9)) * 1e-3
    h = 1e-4
    for dl, dm in ((dlat, None), (None, dmesh)):
        fd = (_oracle_mean_force(case, K, wd, wl, dl, dm, h, skip) -
              _oracle_mean_force(case, K, wd, wl, dl, dm, -h, skip)) / (2 * h)
        ad = float(np.nansum(gl * dl)) if dl is not None else float(np.sum(gm * dm))
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-10, (K, dl is not None, ad, fd)


def test_coupled_adjoint_value_is_the_next_force_samples(H, small):
    """J is the mean of the force samples the solver records over the same
    steps (the adjoint's forward replays the step on scratch copies)."""
    case, s = small
    J = s.adjoint(2, 1.0, 0.5)[0]
    t = H.Solver(case, precision="fp64")
    t.step(1)
    t.forces()
    t.step(2)
    cd, cl = t.forces()
    assert abs(J - float(np.mean(cd + 0.5 * cl))) <= 1e-13 * abs(J)


def test_coupled_adjoint_rejects_what_it_does_not_cover(H):
    for kw in (dict(precision="fp16s"), dict(precision="fp64", fv_filter=0.01)):
        s = H.Solver(make_case("hlbm_small"), **kw)
        with pytest.raises(H.HlbmError) as e:
            s.adjoint(1)
        assert e.value.code == H.HLBM_ENOTIMPL


@pytest.mark.parametrize("name,K", [("hlbm_small", 3), ("hlbm_mini2", 2)])
def test_fp32_forward_adjoint_matches_oracle_finite_differences(H, name, K):
    """FP32 forward steps with the reverse sweep and every gradient sum in FP64:
    J within 1e-5 of the oracle's (FP64) mean force, and the lattice and mesh
    population gradients, contracted with random directions, within 1e-4 of
    oracle central differences (h = 1e-4); the FP64 adjoint of the same case
    gives the same gradients to FP32 accuracy."""
    case = make_case(name, aoa_deg=4.0)
    s32, s64 = H.Solver(case, precision="fp32"), H.Solver(case, precision="fp64")
    for s in (s32, s64):
        s.step(1)
        s.forces()
    J, gls, gm, gx, da = s32.adjoint(K, 1.0, 0.4)
    J64, gls64, gm64, gx64, da64 = s64.adjoint(K, 1.0, 0.4)
    Jo = _oracle_mean_force_levels(case, K, 1.0, 0.4)
    assert abs(J - Jo) <= 1e-5 * abs(Jo), (J, Jo)
    rng = np.random.default_rng(11)
    dlev = [rng.standard_normal((int(nx) * int(ny), 9)) * 1e-3 for nx, ny in case.levels[:, :2]]
    dmesh = rng.standard_normal((case.n_nodes, 9)) * 1e-3
    h = 1e-4
    for dl, dm in ((dlev, None), (None, dmesh)):
        fd = (_oracle_mean_force_levels(case, K, 1.0, 0.4, dl, dm, h) -
              _oracle_mean_force_levels(case, K, 1.0, 0.4, dl, dm, -h)) / (2 * h)
        if dl is not None:
            ad = sum(float(np.nansum(g * d)) for g, d in zip(gls, dl))
            ad64 = sum(float(np.nansum(g * d)) for g, d in zip(gls64, dl))
        else:
            ad, ad64 = float(np.sum(gm * dm)), float(np.sum(gm64 * dm))
        assert abs(ad - fd) <= 1e-4 * abs(fd) + 1e-9, (name, dl is not None, ad, fd)
        assert abs(ad - ad64) <= 1e-4 * abs(ad64) + 1e-9
    assert abs(da - da64) <= 1e-3 * abs(da64) + 1e-9
    assert np.abs(gx - gx64).max() <= 1e-3 * np.abs(gx64).max()


def _oracle_mean_force_levels(case, K, wd, wl, dlev=None, dmesh=None, h=0.0, start=1):
    """As _oracle_mean_force for any number of levels: dlev is a list of
    per-level population directions (None to leave a level)."""
    import oracle
    o = oracle.Oracle(case)
    o.step(start)
    for l, d in enumerate(dlev or []):
        if d is not None:
            f = o.populations(l)
            o.set_populations(l, np.where(np.isnan(f), f, f + h * d))
    if dmesh is not None:
        o.set_populations(-1, o.populations(-1) + h * dmesh)
    o.step(K)
    cd, cl = o.forces()
    return float(np.mean(wd * cd[start:] + wl * cl[start:]))


@pytest.mark.parametrize("name,K", [("hlbm_mini2", 1), ("hlbm_mini2", 2), ("hlbm_mini3", 1)])
def test_refined_adjoint_matches_oracle_finite_differences(H, name, K):
    """Two and three levels (nested refinement boxes, the finest with the
    mesh): band snapshots, prolongation in time and space, restriction,
    sub-cycled finer steps."""
    case = make_case(name, aoa_deg=3.0)
    s = H.Solver(case, precision="fp64")
    s.step(1)
    s.forces()
    J, gls, gm, _, _ = s.adjoint(K, 1.0, 0.3)
    assert abs(J - _oracle_mean_force_levels(case, K, 1.0, 0.3)) <= 1e-10 * max(1.0, abs(J))
    rng = np.random.default_rng(30 + K)
    dirs = [rng.standard_normal(g.shape) * 1e-3 for g in gls]
    dmesh = rng.standard_normal(gm.shape) * 1e-3
    h = 1e-4
    cases = [([d if i == l else None for i, d in enumerate(dirs)], None) for l in range(len(dirs))]
    cases.append((None, dmesh))
    for dl, dm in cases:
        fd = (_oracle_mean_force_levels(case, K, 1.0, 0.3, dl, dm, h) -
              _oracle_mean_force_levels(case, K, 1.0, 0.3, dl, dm, -h)) / (2 * h)
        if dm is not None:
            ad = float(np.sum(gm * dm))
        else:
            ad = sum(float(np.nansum(g * d)) for g, d in zip(gls, dl) if d is not None)
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-10, (K, ad, fd)


def _oracle_moved(case, K, wd, wl, dxy=None, daoa=0.0, h=0.0):
    """Mean of wd C_D + wl C_L over the first K coarse steps of the oracle
    built on moved geometry (node coordinates + h dxy, angle + h daoa)."""
    import dataclasses
    import oracle
    moved = dataclasses.replace(case, xy=case.xy + (h * dxy if dxy is not None else 0.0),
                                aoa_deg=case.aoa_deg + h * daoa)
    o = oracle.Oracle(moved)
    o.step(K)
    cd, cl = o.forces()
    return float(np.mean(wd * cd + wl * cl))


@pytest.mark.parametrize("name", ["hlbm_small", "hlbm_mini2"])
def test_coupled_shape_gradients_match_oracle(H, name):
    """dJ/dx of the mesh nodes, dJ/d(angle of attack) and dJ/dA_m of the
    thickness bumps through whole coarse steps from the initial state (Eq. 3
    operators, wall normals, Eq. 8 and Eq. 9 weights), against central
    differences of the oracle rebuilt on moved geometry."""
    from workloads import thickness_modes
    case = make_case(name, aoa_deg=3.0)
    K, wd, wl = 2, 1.0, 0.5
    s = H.Solver(case, precision="fp64")
    J, _, _, gx, da = s.adjoint(K, wd, wl)
    assert abs(J - _oracle_moved(case, K, wd, wl)) <= 1e-10 * max(1.0, abs(J))
    h = 1e-6
    modes = thickness_modes(case)
    dirs = [modes[0], modes[5], np.random.default_rng(5).standard_normal((case.n_nodes, 2))]
    for d in dirs:
        fd = (_oracle_moved(case, K, wd, wl, dxy=d, h=h) - _oracle_moved(case, K, wd, wl, dxy=d, h=-h)) / (2 * h)
        ad = float(np.sum(gx * d))
        assert abs(ad - fd) <= 1e-5 * abs(fd) + 1e-8, (name, ad, fd)
    ha = 1e-4
    fd = (_oracle_moved(case, K, wd, wl, daoa=1.0, h=ha) - _oracle_moved(case, K, wd, wl, daoa=1.0, h=-ha)) / (2 * ha)
    assert abs(da - fd) <= 1e-5 * abs(fd) + 1e-8, (name, da, fd)


def test_torch_autograd_shape_function(H):
    """paper_2006_10487_gb300.shape.mean_force: its autograd gradient is the
    adjoint's, and agrees with central differences of the library's own
    forward runs on moved geometry."""
    import torch

    from paper_2006_10487_gb300.shape import mean_force
    case = make_case("hlbm_small", aoa_deg=2.0)
    a = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    alpha = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    J = mean_force(case, a, alpha, n_steps=2, wd=1.0, wl=0.0)
    J.backward()
    from workloads import thickness_modes
    modes = thickness_modes(case, 3)

    def forward_only(amps, aoa):
        import dataclasses
        moved = dataclasses.replace(case, xy=case.xy + np.tensordot(amps, modes, axes=1), aoa_deg=aoa)
        s = H.Solver(moved, precision="fp64")
        s.step(2)
        return float(np.mean(s.forces()[0]))

    Jv = float(J.detach())
    assert abs(Jv - forward_only(np.zeros(3), 2.0)) <= 1e-12 * abs(Jv)
    h = 1e-6
    e = np.eye(3)
    for m in range(3):
        fd = (forward_only(h * e[m], 2.0) - forward_only(-h * e[m], 2.0)) / (2 * h)
        assert abs(float(a.grad[m]) - fd) <= 1e-5 * abs(fd) + 1e-8
    fd = (forward_only(np.zeros(3), 2.0 + 1e-4) - forward_only(np.zeros(3), 2.0 - 1e-4)) / 2e-4
    assert abs(float(alpha.grad) - fd) <= 1e-5 * abs(fd) + 1e-8
