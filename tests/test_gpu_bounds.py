"""Bounds-checked library (HLBM_DEBUG): every table-driven or computed index
of the kernels is checked against its extent.  Runs of the parity workloads
through it meet no violation, and their results are those of the release
library (the checks change no arithmetic).  This stands in for a memory
checker: the checks redirect a bad access to index 0 and count it, so no run
can fault."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from workloads import make_case

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# (workload, angle of attack, precision, coarse steps, wall statistics,
# finite-volume variant: 0 autotuned, 2 and 8 on 128- and 256-row tiles)
RUNS = [("hlbm_mini2", 3.0, "fp64", 3, True, 0), ("hlbm_single", 0.0, "fp32", 2, False, 2),
        ("hlbm_small", 8.0, "fp16s", 3, True, 0), ("hlbm_single", 0.0, "fp32", 2, False, 8),
        ("hlbm_mini2", 3.0, "fp32", 3, True, 6)]

CHILD = r"""
import json, sys
import numpy as np
import paper_2006_10487_gb300 as H
from workloads import make_case
runs, out = json.loads(sys.argv[1]), sys.argv[2]
arrays, report = {}, {}
for j, (name, aoa, prec, steps, ws, var) in enumerate(runs):
    case = make_case(name, aoa_deg=aoa)
    s = H.Solver(case, precision=prec, wall_stats=ws, fv_variant=var)
    s.step(steps)
    for g in list(range(case.n_levels)) + [-1]:
        arrays[f"{j}_{g}"] = np.stack(s.fields(g))
    arrays[f"{j}_forces"] = np.stack(s.forces())
    if ws:
        arrays[f"{j}_wall"] = s.wall_stats()[0]
    report[j] = (s.info("bounds_violations"), s.info("bounds_sites"))
    s.close()
np.savez(out, **arrays)
print(json.dumps(report))
"""


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_10487_gb300 import build
    build.build()
    build.build(debug=True)
    import paper_2006_10487_gb300 as H
    return H


def test_parity_workloads_meet_no_bounds_violation(H, tmp_path):
    out = str(tmp_path / "debug.npz")
    env = dict(os.environ, HLBM_DEBUG="1", PYTHONPATH=ROOT)
    res = subprocess.run([sys.executable, "-c", CHILD, json.dumps(RUNS), out], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    report = json.loads(res.stdout.strip().splitlines()[-1])
    for j, (violations, sites) in report.items():
        assert violations == 0 and sites == 0, (RUNS[int(j)], violations, sites)
    dbg = np.load(out)
    for j, (name, aoa, prec, steps, ws, var) in enumerate(RUNS):
        case = make_case(name, aoa_deg=aoa)
        s = H.Solver(case, precision=prec, wall_stats=ws, fv_variant=var)
        s.step(steps)
        assert s.info("bounds_violations") == -1  # the release library has no checks
        tol = 1e-12 if prec == "fp64" else 1e-5
        for g in list(range(case.n_levels)) + [-1]:
            a, b = np.stack(s.fields(g)), dbg[f"{j}_{g}"]
            assert np.array_equal(np.isnan(a), np.isnan(b)), (name, g)
            m = ~np.isnan(a)
            assert np.linalg.norm(a[m] - b[m]) <= tol * np.linalg.norm(a[m]), (name, prec, g)
        np.testing.assert_allclose(np.stack(s.forces()), dbg[f"{j}_forces"], rtol=tol, atol=tol * 1e-2)
        if ws:
            np.testing.assert_allclose(s.wall_stats()[0], dbg[f"{j}_wall"], rtol=tol, atol=tol)
        s.close()
