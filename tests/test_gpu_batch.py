"""Batched ensemble: cases advanced together by one graph launch per coarse
step give, case by case, bitwise the results of stepping each case alone."""
import numpy as np
import pytest

from workloads import ensemble_case, make_case

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


CASES = [("hlbm_small", 0.0, "fp32"), ("hlbm_small", 8.0, "fp16s"), ("hlbm_mini2", 3.0, "fp64"),
         ("hlbm_mini2", 0.0, "fp32")]


def grids(case):
    return list(range(case.n_levels)) + [-1]


def test_batch_matches_cases_stepped_alone(H):
    cases = [make_case(n, aoa_deg=a) for n, a, _ in CASES]
    alone = [H.Solver(c, precision=p) for c, (_, _, p) in zip(cases, CASES)]
    grouped = [H.Solver(c, precision=p) for c, (_, _, p) in zip(cases, CASES)]
    batch = H.Batch(grouped)
    for s in alone:
        s.step(5)
    batch.step(2)
    batch.step(3)  # odd then even phase start
    for case, a, b in zip(cases, alone, grouped):
        for g in grids(case):
            for x, y in zip(a.fields(g), b.fields(g)):
                assert np.array_equal(x, y, equal_nan=True)
        fa, fb = a.forces(), b.forces()
        assert len(fb[0]) == 5
        assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    batch.close()


def test_batch_refuses_a_case_stepped_outside_it(H):
    solvers = [H.Solver(make_case("hlbm_mini2"), precision="fp32") for _ in range(2)]
    batch = H.Batch(solvers)
    batch.step(1)
    solvers[1].step(1)
    with pytest.raises(H.HlbmError) as e:
        batch.step(1)
    assert e.value.code == H.HLBM_ESTATE
    batch.close()


def test_batched_fp64_cases_match_the_oracle(H, orc):
    """Two FP64 cases of different sizes and level counts (the one-level
    airfoil case at 5 degrees and the two-level case at 2 degrees) advanced
    only by batched graph launches, against the oracle run of each case:
    every field within 1e-12 of its scale and the force series within 1e-12,
    after 30 coarse steps."""
    cases = [make_case("hlbm_small", aoa_deg=5.0), make_case("hlbm_mini2", aoa_deg=2.0)]
    solvers = [H.Solver(c, precision="fp64") for c in cases]
    batch = H.Batch(solvers)
    batch.step(13)
    batch.step(17)
    batch.sync()
    for case, s in zip(cases, solvers):
        o = orc.Oracle(case)
        o.step(30)
        for g in grids(case):
            (ar, ax, ay), (br, bx, by) = s.fields(g), o.fields(g)
            m = np.isfinite(br)
            assert np.array_equal(np.isfinite(ar), m)
            assert np.abs(ar[m] - br[m]).max() <= 1e-12 * np.abs(br[m]).max()
            assert np.hypot(ax[m] - bx[m], ay[m] - by[m]).max() <= 1e-12 * np.hypot(bx[m], by[m]).max()
        (cd, cl), (ocd, ocl) = s.forces(), o.forces()
        assert len(cd) == 30
        assert np.abs(cd - ocd).max() <= 1e-12 * np.abs(ocd).max()
        assert np.abs(cl - ocl).max() <= 1e-12 * max(np.abs(ocl).max(), np.abs(ocd).max())
    batch.close()


def test_ensemble_cases_at_full_size_match_the_oracle(H, orc):
    """Two members of the batched ensemble at their full sizes, the largest
    (Re 5000 at 15 degrees: 2048 x 1024 lattice, 300 032-node mesh, 93
    sub-steps per step) and the smallest (Re 500 at 0 degrees: 512 x 256, 20 480
    nodes), FP64, advanced only by batched graph launches: every field within
    1e-12 of its scale and the force series within 1e-12 of the oracle's
    (OpenMP build) after two coarse steps."""
    cases = [ensemble_case(5000.0, 15.0), ensemble_case(500.0, 0.0)]
    solvers = [H.Solver(c, precision="fp64") for c in cases]
    batch = H.Batch(solvers)
    batch.step(2)
    batch.sync()
    for case, s in zip(cases, solvers):
        o = orc.Oracle(case, openmp=True)
        o.step(2)
        for g in grids(case):
            (ar, ax, ay), (br, bx, by) = s.fields(g), o.fields(g)
            m = np.isfinite(br)
            assert np.array_equal(np.isfinite(ar), m)
            assert np.abs(ar[m] - br[m]).max() <= 1e-12 * np.abs(br[m]).max(), (case.name, g)
            assert np.hypot(ax[m] - bx[m], ay[m] - by[m]).max() <= 1e-12 * np.hypot(bx[m], by[m]).max(), (case.name, g)
        (cd, cl), (ocd, ocl) = s.forces(), o.forces()
        assert len(cd) == 2
        assert np.abs(cd - ocd).max() <= 1e-12 * np.abs(ocd).max()
        assert np.abs(cl - ocl).max() <= 1e-12 * max(np.abs(ocl).max(), np.abs(ocd).max())
    batch.close()
