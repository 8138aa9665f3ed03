"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: FP64 max relative field difference (max|a - b| / max|b| per field and
grid) <= 1e-12; FP32 velocity relative L2 <= 1e-5 against FP64 and mean
C_D / C_L relative error <= 1e-3.
"""
import math

import numpy as np
import pytest

from workloads import make_case

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_10487_gb300 import build
    build.build()
    import paper_2006_10487_gb300 as H
    return H


def grids(case):
    return list(range(case.n_levels)) + ([-1] if case.n_nodes else [])


def rel_field_diff(a, b):
    fa, fb = np.isfinite(a), np.isfinite(b)
    assert np.array_equal(fa, fb), "NaN pattern (hole nodes) differs"
    if not fb.any():
        return 0.0
    scale = np.abs(b[fb]).max()
    return np.abs(a[fa] - b[fb]).max() / (scale if scale > 0 else 1.0)


def rel_velocity_diff(ax, ay, bx, by):
    """Velocity as one vector field: max |u_a - u_b| / max |u_b| over computed nodes."""
    m = np.isfinite(bx)
    assert np.array_equal(np.isfinite(ax), m), "NaN pattern (hole nodes) differs"
    scale = np.hypot(bx[m], by[m]).max()
    return np.hypot(ax[m] - bx[m], ay[m] - by[m]).max() / (scale if scale > 0 else 1.0)


UY_TOL = 1e-8


def compare_fields(sol, orc_sim, case, tol, label=""):
    """Relative field difference per grid: density max|d rho| / max|rho|; velocity
    as a vector field (its components share one scale, so the small cross-stream
    component is not measured against its own near-zero maximum).  The
    per-component differences max|d u_x| / max|u_x| and max|d u_y| / max|u_y|
    are printed beside it; u_y, whose own maximum is set by the 1e-4 density
    perturbation at zero incidence, is held to UY_TOL per field."""
    worst = 0.0
    for g in grids(case):
        (ar, ax, ay), (br, bx, by) = sol.fields(g), orc_sim.fields(g)
        d_rho = rel_field_diff(ar, br)
        d_u = rel_velocity_diff(ax, ay, bx, by)
        d_ux, d_uy = rel_field_diff(ax, bx), rel_field_diff(ay, by)
        print(f"PARITY {label} grid {g}: rho {d_rho:.2e} u {d_u:.2e} u_x {d_ux:.2e} u_y {d_uy:.2e}")
        assert d_rho <= tol, f"grid {g} density: relative difference {d_rho:.3e} > {tol:.1e}"
        assert d_u <= tol, f"grid {g} velocity: relative difference {d_u:.3e} > {tol:.1e}"
        assert d_uy <= UY_TOL, f"grid {g} u_y per field: relative difference {d_uy:.3e} > {UY_TOL:.1e}"
        worst = max(worst, d_rho, d_u)
    return worst


@pytest.mark.parametrize("name,steps,aoa", [("channel", 200, 0.0), ("hlbm_small", 100, 0.0),
                                            ("hlbm_small", 20, 8.0), ("hlbm_mini2", 100, 0.0),
                                            ("hlbm_mini2", 30, 5.0), ("hlbm_mini3", 40, 3.0),
                                            ("patch", 100, 0.0), ("patch", 60, 20.0)])
def test_fp64_matches_oracle(H, orc, name, steps, aoa):
    case = make_case(name, aoa_deg=aoa)
    sol = H.Solver(case, precision="fp64")
    sim = orc.Oracle(case)
    assert sol.info("n_sub") == sim.n_sub
    sol.step(steps)
    sim.step(steps)
    compare_fields(sol, sim, case, FP64_TOL, f"{name} {steps} steps aoa {aoa:g}")
    if case.n_nodes:
        cd, cl = sol.forces()
        ocd, ocl = sim.forces()
        assert len(cd) == steps
        assert np.abs(cd - ocd).max() <= FP64_TOL * np.abs(ocd).max()
        assert np.abs(cl - ocl).max() <= FP64_TOL * max(np.abs(ocl).max(), np.abs(ocd).max())


@pytest.mark.parametrize("name,steps,aoa", [("hlbm_small", 30, 8.0), ("hlbm_mini3", 20, 3.0)])
def test_fp64_with_the_odd_even_filter_matches_oracle(H, orc, name, steps, aoa):
    """The optional odd-even filter of the mesh state (fv_filter = 0.05, once
    per finest step): every grid and the force series within 1e-12 of the
    oracle's filtered run."""
    case = make_case(name, aoa_deg=aoa, fv_filter=0.05)
    sol = H.Solver(case, precision="fp64")
    sim = orc.Oracle(case)
    assert sol.info("fv_filter") == 0.05
    sol.step(steps)
    sim.step(steps)
    compare_fields(sol, sim, case, FP64_TOL, f"{name} filtered")
    cd, cl = sol.forces()
    ocd, ocl = sim.forces()
    assert np.abs(cd - ocd).max() <= FP64_TOL * np.abs(ocd).max()
    assert np.abs(cl - ocl).max() <= FP64_TOL * max(np.abs(ocl).max(), np.abs(ocd).max())


@pytest.mark.slow
def test_small_airfoil_full_run_fp64(H, orc):
    """The one-level airfoil case over its whole nominal run (2000 steps of the 200 x 100 lattice
    with the 5 200-node mesh, Re 500, zero incidence): the FP64 force series
    within 1e-10 of the oracle's (OpenMP build, bitwise the serial one) at every
    step, and every field within 1e-10 at the end."""
    case = make_case("hlbm_small")
    assert case.steps == 2000
    sol = H.Solver(case, precision="fp64", force_cap=4096)
    sim = orc.Oracle(case, openmp=True)
    cd, cl = [], []
    for _ in range(4):
        sol.step(500)
        sim.step(500)
        c, l_ = sol.forces()
        cd.append(c)
        cl.append(l_)
    cd, cl = np.concatenate(cd), np.concatenate(cl)
    ocd, ocl = sim.forces()
    assert len(cd) == len(ocd) == 2000
    assert np.abs(cd - ocd).max() <= 1e-10 * np.abs(ocd).max()
    assert np.abs(cl - ocl).max() <= 1e-10 * np.abs(ocd).max()
    compare_fields(sol, sim, case, 1e-10, "hlbm_small 2000 steps")


def test_populations_match_oracle(H, orc):
    case = make_case("hlbm_mini2")
    sol = H.Solver(case, precision="fp64")
    sim = orc.Oracle(case)
    sol.step(7)
    sim.step(7)
    for g in grids(case):
        a, b = sol.populations(g), sim.populations(g)
        fin = np.isfinite(b).all(axis=1)
        assert np.array_equal(np.isfinite(a).all(axis=1), fin)
        assert np.abs(a[fin] - b[fin]).max() <= FP64_TOL


def test_single_config_one_coarse_step_fp64(H, orc):
    """Full-size single case (2048x1024 + two nested boxes, 200 704-node mesh),
    the configuration the benchmark times, after one coarse step
    (4 finest steps x n_sub finite-volume sub-steps)."""
    case = make_case("hlbm_single")
    sol = H.Solver(case, precision="fp64")
    sim = orc.Oracle(case)
    sol.step(1)
    sim.step(1)
    compare_fields(sol, sim, case, FP64_TOL)


@pytest.mark.slow
def test_refined_airfoil_100_finest_steps_fp64(H, orc):
    """The benchmarked configuration (2048 x 1024 + two nested boxes, 200 704-node
    mesh) over 25 coarse steps = 100 steps of the finest lattice (3 100
    finite-volume sub-steps): every grid within 1e-12 of the oracle (OpenMP
    build, bitwise the serial one) and the force series within 1e-12."""
    case = make_case("hlbm_single")
    sol = H.Solver(case, precision="fp64")
    sim = orc.Oracle(case, openmp=True)
    sol.step(25)
    sim.step(25)
    compare_fields(sol, sim, case, FP64_TOL, "hlbm_single 25 coarse steps")
    cd, cl = sol.forces()
    ocd, ocl = sim.forces()
    assert np.abs(cd - ocd).max() <= FP64_TOL * np.abs(ocd).max()
    assert np.abs(cl - ocl).max() <= FP64_TOL * np.abs(ocd).max()


def test_single_config_fp32_against_fp64(H):
    """FP32 against the FP64 GPU path on the benchmarked configuration at 8
    degrees, 100 coarse steps: velocity relative L2 per grid at most 1e-5 and
    mean C_D, C_L within 1e-3 (measured: 2-5e-6 and ~1e-5)."""
    case = make_case("hlbm_single", aoa_deg=8.0)
    a, b = H.Solver(case, precision="fp32"), H.Solver(case, precision="fp64")
    a.step(100)
    b.step(100)
    for g in grids(case):
        _, ux, uy = a.fields(g)
        _, vx, vy = b.fields(g)
        m = np.isfinite(vx)
        err = math.sqrt(((ux[m] - vx[m]) ** 2 + (uy[m] - vy[m]) ** 2).sum() / (vx[m] ** 2 + vy[m] ** 2).sum())
        print(f"PARITY hlbm_single fp32 vs fp64 grid {g}: velocity relative L2 {err:.2e}")
        assert err <= 1e-5, f"grid {g}: velocity relative L2 {err:.2e}"
    (cd, cl), (cd64, cl64) = a.forces(), b.forces()
    assert abs(cd.mean() - cd64.mean()) <= 1e-3 * abs(cd64.mean())
    assert abs(cl.mean() - cl64.mean()) <= 1e-3 * abs(cl64.mean())


def test_single_config_one_coarse_step_fp32(H, orc):
    case = make_case("hlbm_single")
    sol = H.Solver(case, precision="fp32")
    sim = orc.Oracle(case)
    sol.step(1)
    sim.step(1)
    u0 = case.Ma / math.sqrt(3)
    for g in grids(case):
        r, ux, uy = sol.fields(g)
        orr, oux, ouy = sim.fields(g)
        m = np.isfinite(orr)
        err = math.sqrt(((ux[m] - oux[m]) ** 2 + (uy[m] - ouy[m]) ** 2).sum() / (oux[m] ** 2 + ouy[m] ** 2).sum())
        assert err <= 1e-5, f"grid {g}: velocity relative L2 {err:.2e}"
        assert np.abs(r[m] - orr[m]).max() <= 1e-5
        assert np.abs(ux[m] - oux[m]).max() <= 1e-4 * u0 * 10


@pytest.mark.parametrize("aoa", [0.0, 8.0])
def test_fp32_accuracy_against_fp64(H, aoa):
    case = make_case("hlbm_small", aoa_deg=aoa)
    a = H.Solver(case, precision="fp32")
    b = H.Solver(case, precision="fp64")
    a.step(400)
    b.step(400)
    for g in grids(case):
        _, ux, uy = a.fields(g)
        _, vx, vy = b.fields(g)
        m = np.isfinite(vx)
        err = math.sqrt(((ux[m] - vx[m]) ** 2 + (uy[m] - vy[m]) ** 2).sum() / (vx[m] ** 2 + vy[m] ** 2).sum())
        assert err <= 1e-5, f"grid {g}: velocity relative L2 {err:.2e}"
    cd32, cl32 = a.forces()
    cd64, cl64 = b.forces()
    mcd, mcl = cd64[100:].mean(), cl64[100:].mean()
    assert abs(cd32[100:].mean() - mcd) <= 1e-3 * abs(mcd)
    assert abs(cl32[100:].mean() - mcl) <= 1e-3 * max(abs(mcl), abs(mcd) if aoa == 0 else 0.0)


@pytest.mark.parametrize("aoa", [0.0, 8.0])
def test_fp16s_accuracy_against_fp64(H, aoa):
    """FP16S lattice storage (16-bit populations shifted by the free stream, FP32
    mesh and arithmetic): mean C_D / C_L within 1e-3 of FP64 (measured: about
    2e-5); the velocity field within 16-bit storage resolution (relative L2
    <= 2e-4, measured about 3e-5)."""
    case = make_case("hlbm_small", aoa_deg=aoa)
    a = H.Solver(case, precision="fp16s")
    b = H.Solver(case, precision="fp64")
    assert a.info("collide_bytes0") * 4 == b.info("collide_bytes0")
    a.step(400)
    b.step(400)
    for g in grids(case):
        _, ux, uy = a.fields(g)
        _, vx, vy = b.fields(g)
        m = np.isfinite(vx)
        assert np.array_equal(np.isfinite(ux), m)
        err = math.sqrt(((ux[m] - vx[m]) ** 2 + (uy[m] - vy[m]) ** 2).sum() / (vx[m] ** 2 + vy[m] ** 2).sum())
        assert err <= 2e-4, f"grid {g}: velocity relative L2 {err:.2e}"
    cd16, cl16 = a.forces()
    cd64, cl64 = b.forces()
    mcd, mcl = cd64[100:].mean(), cl64[100:].mean()
    assert abs(cd16[100:].mean() - mcd) <= 1e-3 * abs(mcd)
    assert abs(cl16[100:].mean() - mcl) <= 1e-3 * max(abs(mcl), abs(mcd) if aoa == 0 else 0.0)


def test_fp16s_single_config_one_coarse_step(H, orc):
    """Full-size single case in FP16S against the oracle after one coarse step."""
    case = make_case("hlbm_single")
    sol = H.Solver(case, precision="fp16s")
    sim = orc.Oracle(case)
    sol.step(1)
    sim.step(1)
    for g in grids(case):
        _, ux, uy = sol.fields(g)
        _, oux, ouy = sim.fields(g)
        m = np.isfinite(oux)
        assert np.array_equal(np.isfinite(ux), m)
        err = math.sqrt(((ux[m] - oux[m]) ** 2 + (uy[m] - ouy[m]) ** 2).sum() / (oux[m] ** 2 + ouy[m] ** 2).sum())
        assert err <= 2e-4, f"grid {g}: velocity relative L2 {err:.2e}"


@pytest.mark.slow
def test_large_re_one_coarse_step_fp64_matches_oracle(H, orc):
    """The largest configuration at its full size (8192 x 4096 coarse level,
    three nested boxes of 4097 x 2049, the 1.5 M-node mesh, Re 10^4; 8 finest
    steps and 368 finite-volume sub-steps in one coarse step), FP64 against
    the oracle (OpenMP build): every grid within FP64_TOL and the force
    sample within 1e-12 of the oracle's."""
    case = make_case("hlbm_large")
    sol = H.Solver(case, precision="fp64")
    sol.step(1)
    sim = orc.Oracle(case, openmp=True)
    sim.step(1)
    compare_fields(sol, sim, case, FP64_TOL, "hlbm_large fp64")
    (cd, cl), (ocd, ocl) = sol.forces(), sim.forces()
    assert len(cd) == 1
    assert abs(cd[0] - ocd[0]) <= 1e-12 * abs(ocd[0])
    assert abs(cl[0] - ocl[0]) <= 1e-12 * max(abs(ocl[0]), abs(ocd[0]))
    sol.close()


def test_large_re_fp32_and_fp16s_against_fp64(H):
    """Large-Re configuration (8192x4096 coarse level, three nested boxes,
    1.5 M-node mesh, Re 10^4): FP32 and FP16S against the FP64 GPU path on the
    same inputs, per field, after two coarse steps (16 finest steps, 736
    finite-volume sub-steps).  Measured: velocity relative L2 about 1e-6 in
    both modes, density about 7e-7."""
    case = make_case("hlbm_large")
    ref = H.Solver(case, precision="fp64")
    ref.step(2)
    want = {g: ref.fields(g) for g in grids(case)}
    cd64, cl64 = ref.forces()
    ref.close()
    for prec, tol_u, tol_rho in (("fp32", 1e-5, 1e-5), ("fp16s", 2e-5, 1e-5)):
        sol = H.Solver(case, precision=prec)
        sol.step(2)
        for g in grids(case):
            r, ux, uy = sol.fields(g)
            rr, vx, vy = want[g]
            m = np.isfinite(vx)
            assert np.array_equal(np.isfinite(ux), m)
            err = math.sqrt(((ux[m] - vx[m]) ** 2 + (uy[m] - vy[m]) ** 2).sum() / (vx[m] ** 2 + vy[m] ** 2).sum())
            assert err <= tol_u, f"{prec} grid {g}: velocity relative L2 {err:.2e}"
            d_rho = np.abs(r[m] - rr[m]).max()
            assert d_rho <= tol_rho, f"{prec} grid {g}: density max difference {d_rho:.2e}"
        cd, cl = sol.forces()
        assert abs(cd.mean() - cd64.mean()) <= 1e-3 * abs(cd64.mean())
        assert abs(cl.mean() - cl64.mean()) <= 1e-3 * abs(cd64.mean())
        sol.close()


def test_wall_stats_match_oracle(H, orc):
    """Mean C_p, C_f, C_n per wall node (Eq. 12-13), accumulated on the GPU
    (FP64) over 12 coarse steps, against the oracle's per-step values averaged
    over the same steps; then again after a reset."""
    case = make_case("hlbm_small", aoa_deg=8.0)
    sol = H.Solver(case, precision="fp64", wall_stats=True)
    sim = orc.Oracle(case)
    acc = 0.0
    for _ in range(12):
        sol.step(1)
        sim.step(1)
        acc = acc + sim.wall_coeffs()
    got, n = sol.wall_stats()
    want = acc / 12
    assert n == 12 and got.shape == want.shape
    assert np.allclose(got[:, 0], want[:, 0], atol=1e-12)
    assert np.allclose(got[:, 5:], want[:, 5:], rtol=1e-12, atol=1e-13)
    for col in (2, 3, 4):
        assert np.abs(got[:, col] - want[:, col]).max() <= FP64_TOL * np.abs(want[:, col]).max()
    sol.wall_stats_reset()
    acc = 0.0
    for _ in range(3):
        sol.step(1)
        sim.step(1)
        acc = acc + sim.wall_coeffs()
    got, n = sol.wall_stats()
    assert n == 3
    for col in (2, 3, 4):
        assert np.abs(got[:, col] - acc[:, col] / 3).max() <= FP64_TOL * np.abs(acc[:, col] / 3).max()


def test_wall_stats_reassemble_the_mean_forces(H):
    """In FP32: sum_P |N_P| [(-C_p + C_n) n + C_f s] / C of the mean
    coefficients is the mean of the recorded (C_D, C_L)."""
    case = make_case("hlbm_small", aoa_deg=8.0)
    sol = H.Solver(case, precision="fp32", wall_stats=True)
    sol.step(40)
    w, n = sol.wall_stats()
    cd, cl = sol.forces()
    F = (w[:, 5, None] * ((-w[:, 2] + w[:, 4])[:, None] * w[:, 6:8] + w[:, 3, None] * w[:, 8:10])).sum(0)
    F /= case.chord
    assert n == 40 == len(cd)
    assert abs(F[0] - cd.mean()) <= 1e-9 * abs(cd.mean())
    assert abs(F[1] - cl.mean()) <= 1e-9 * abs(cd.mean())


def test_fv_register_bounds_agree_bitwise_and_the_autotuner_reports(H):
    """The variants of the FP32 finite-volume kernel: on each tiling (128- and
    256-row tiles), registers bounded for the lower and the higher block count
    per SM, each with and without the L2 prefetch of a later tile, run the
    same arithmetic: identical results within a tiling, on a mesh of a few
    tiles and on the 200 k-node mesh.  The two tilings order each row's
    entries for their own shared-memory banks, so across tilings the fields
    agree to FP32 rounding.  The default (autotuned) context reports its
    choice and the timings of all eight."""
    for name, steps in (("hlbm_mini2", 9), ("hlbm_single", 1)):
        case = make_case(name, aoa_deg=3.0)
        groups = []
        for vs in ((1, 2, 3, 4), (5, 6, 7, 8)):
            runs = [H.Solver(case, precision="fp32", fv_variant=v) for v in vs]
            for v, s in zip(vs, runs):
                assert s.info("fv_variant") == v
                assert s.info("fv_tile_rows") == (128 if v <= 4 else 256)
                s.step(steps)
            ref = runs[0]
            ref_cd = ref.forces()[0]
            for s in runs[1:]:
                for g in grids(case):
                    for x, y in zip(ref.fields(g), s.fields(g)):
                        assert np.array_equal(x, y, equal_nan=True), (name, g)
                assert np.array_equal(ref_cd, s.forces()[0])
            groups.append((ref, ref_cd))
            for s in runs[1:]:
                s.close()
        (a, cda), (b, cdb) = groups
        for g in grids(case):
            (_, ax, ay), (_, bx, by) = a.fields(g), b.fields(g)
            assert rel_velocity_diff(ax, ay, bx, by) <= 1e-5, (name, g)
        assert np.abs(cda - cdb).max() <= 1e-5 * np.abs(cdb).max()
        a.close()
        b.close()
    # the autotuner times the 256-row tiles only where the 128-row tiles need
    # more than two waves of resident blocks: not on the 200 k-node mesh, on
    # the 1.5 M-node one
    t = H.Solver(make_case("hlbm_single"), precision="fp32")
    assert t.info("fv_variant") in range(1, 5) and t.info("fv_tile_rows") == 128
    assert all(t.info(f"fv_tune_us{v}") > 0 for v in range(1, 5))
    assert all(t.info(f"fv_tune_us{v}") == 0 for v in range(5, 9))
    t.close()
    t = H.Solver(make_case("hlbm_large_fv"), precision="fp32")
    assert all(t.info(f"fv_tune_us{v}") > 0 for v in range(1, 9))
    assert t.info("fv_tile_rows") == (128 if t.info("fv_variant") <= 4 else 256)
    t.close()


def test_wide_tiling_fp32_against_fp64(H):
    """The 256-row tiling of the FP32 sub-step against the FP64 path on the
    one-level airfoil case: velocity relative L2 within 1e-5 after 100
    coarse steps, mean C_D and C_L within 1e-3."""
    case = make_case("hlbm_small", aoa_deg=8.0)
    a = H.Solver(case, precision="fp32", fv_variant=6)
    b = H.Solver(case, precision="fp64")
    assert a.info("fv_tile_rows") == 256 and b.info("fv_tile_rows") == 128
    a.step(100)
    b.step(100)
    for g in grids(case):
        _, ux, uy = a.fields(g)
        _, vx, vy = b.fields(g)
        m = np.isfinite(vx)
        err = math.sqrt(((ux[m] - vx[m]) ** 2 + (uy[m] - vy[m]) ** 2).sum() / (vx[m] ** 2 + vy[m] ** 2).sum())
        assert err <= 1e-5, f"grid {g}: velocity relative L2 {err:.2e}"
    (cd, cl), (cd64, cl64) = a.forces(), b.forces()
    assert abs(cd.mean() - cd64.mean()) <= 1e-3 * abs(cd64.mean())
    assert abs(cl.mean() - cl64.mean()) <= 1e-3 * abs(cl64.mean())


@pytest.mark.parametrize("name", ["hlbm_small", "hlbm_mini2"])
def test_level0_mass_matches_oracle(H, orc, name):
    """The FP64 mass monitor: sum of rho over level 0's computed nodes against
    the oracle's level-0 density field; a healthy run drifts little."""
    case = make_case(name)
    sol = H.Solver(case, precision="fp64")
    sim = orc.Oracle(case)
    m0 = sol.info("mass")
    r0, _, _ = sim.fields(0)
    assert abs(m0 - np.nansum(r0)) <= 1e-12 * m0
    sol.step(20)
    sim.step(20)
    r, _, _ = sim.fields(0)
    m = sol.info("mass")
    assert abs(m - np.nansum(r)) <= 1e-12 * m
    assert 0 < sol.info("mass_drift") < 1e-3
    assert sol.info("mass_drift") == pytest.approx(abs(m - m0) / m0, rel=1e-9)


def test_checkpoint_resume_is_bitwise(H, tmp_path):
    """hlbm_save after 7 coarse steps, hlbm_load into a new context made from
    the same inputs, 5 more steps each: the same fields on every grid, force
    series and wall statistics, bit for bit; another precision is refused."""
    for name, prec, filt in (("hlbm_mini2", "fp32", 0.0), ("hlbm_small", "fp16s", 0.0), ("hlbm_mini2", "fp64", 0.0),
                             ("hlbm_small", "fp32", 0.01)):
        case = make_case(name, aoa_deg=4.0, fv_filter=filt)
        a = H.Solver(case, precision=prec, wall_stats=True)
        a.step(7)
        path = str(tmp_path / f"{name}_{prec}_{filt:g}.ckpt")
        a.save(path)
        b = H.Solver(case, precision=prec, wall_stats=True)
        b.load(path)
        a.step(5)
        b.step(5)
        for g in grids(case):
            for x, y in zip(a.fields(g), b.fields(g)):
                assert np.array_equal(x, y, equal_nan=True), (name, prec, g)
        fa, fb = a.forces(), b.forces()
        assert len(fa[0]) == len(fb[0]) == 12
        assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
        wa, wb = a.wall_stats(), b.wall_stats()
        assert wa[1] == wb[1] == 12 and np.array_equal(wa[0], wb[0])
    other = H.Solver(make_case("hlbm_mini2", aoa_deg=4.0), precision="fp32", wall_stats=True)
    with pytest.raises(H.HlbmError) as e:
        other.load(str(tmp_path / "hlbm_mini2_fp64_0.ckpt"))
    assert e.value.code == H.HLBM_EINVAL


@pytest.mark.parametrize("filt", [0.0, 0.02])
def test_graphs_and_plain_launches_agree_bitwise(H, filt):
    case = make_case("hlbm_mini2", fv_filter=filt)
    a = H.Solver(case, precision="fp64", use_graphs=True)
    b = H.Solver(case, precision="fp64", use_graphs=False)
    a.step(9)
    b.step(9)
    for g in grids(case):
        for x, y in zip(a.fields(g), b.fields(g)):
            assert np.array_equal(x, y, equal_nan=True)
    assert np.array_equal(a.forces()[0], b.forces()[0])


def test_step_graphs_with_health_checks_and_wall_stats_agree_bitwise(H):
    """FP32 on the refined airfoil case with wall statistics: graphs of one
    and two coarse steps (with the finite-volume branch and the forces kept on
    it inside a pair), cut where a health check falls (every 3 steps) and at
    odd call lengths, against plain launches of every step: the same fields,
    forces and wall sums, bit for bit."""
    case = make_case("hlbm_mini3", aoa_deg=6.0)
    a = H.Solver(case, precision="fp32", use_graphs=True, check_every=3, wall_stats=True)
    b = H.Solver(case, precision="fp32", use_graphs=False, wall_stats=True)
    a.step(4)
    a.step(7)
    b.step(11)
    for g in grids(case):
        for x, y in zip(a.fields(g), b.fields(g)):
            assert np.array_equal(x, y, equal_nan=True), g
    (ca, la), (cb, lb) = a.forces(), b.forces()
    assert len(ca) == 11 and np.array_equal(ca, cb) and np.array_equal(la, lb)
    (wa, na), (wb, nb) = a.wall_stats(), b.wall_stats()
    assert na == nb == 11 and np.array_equal(wa, wb)
    a.close()
    b.close()


def test_runs_are_deterministic(H):
    case = make_case("hlbm_small")
    res = []
    for _ in range(2):
        s = H.Solver(case, precision="fp32")
        s.step(25)
        res.append((s.fields(-1), s.fields(0), s.forces()))
    for x, y in zip(res[0][0] + res[0][1], res[1][0] + res[1][1]):
        assert np.array_equal(x, y, equal_nan=True)
    assert np.array_equal(res[0][2][0], res[1][2][0])


def test_hole_nodes_are_nan_and_the_rest_finite(H):
    case = make_case("hlbm_small")
    s = H.Solver(case, precision="fp64")
    s.step(3)
    r, _, _ = s.fields(0)
    nan = ~np.isfinite(r)
    n_interp = s.info("n_interp")
    assert nan.sum() > n_interp > 0
    y, x = np.divmod(np.arange(r.size), case.levels[0][0])
    cx, cy, a, b = case.hole
    inside = ((x - cx) / a) ** 2 + ((y - cy) / b) ** 2 < 1
    assert np.array_equal(nan, inside)


def test_force_ring_buffer_keeps_the_latest_samples(H):
    case = make_case("hlbm_mini2")
    s = H.Solver(case, precision="fp64", force_cap=8)
    s.step(5)
    cd1, _ = s.forces()
    assert len(cd1) == 5
    s.step(20)
    cd2, _ = s.forces()
    assert len(cd2) == 8  # older samples were overwritten
    ref = H.Solver(case, precision="fp64")
    ref.step(25)
    cd_all, _ = ref.forces()
    assert np.array_equal(cd1, cd_all[:5])
    assert np.array_equal(cd2, cd_all[-8:])


def test_health_flag_reports_instability(H):
    """An explicit finite-volume sub-step count far below the stability bound
    blows up; hlbm_step reports it through the NaN health flag."""
    case = make_case("hlbm_small")
    s = H.Solver(case, precision="fp64", n_sub=10, check_every=10)
    with pytest.raises(H.HlbmError) as e:
        s.step(400)
    assert e.value.code == H.HLBM_EUNSTABLE
