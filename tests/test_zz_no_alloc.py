"""The allocation-free force entry point, checked against hlbm_forces.

Some callers cannot call cudaMalloc (their device memory belongs to another
framework's pool, or they evaluate forces in loops that must not allocate).
hlbm_wall_forces_static serves them: it keeps its reduction scratch in a fixed
device array.  This file runs last so that a failure here leaves every other
test already run; it also passes on its own in a fresh process.
"""
import ctypes as C
import math

import numpy as np
import pytest

from workloads import make_case

pytestmark = pytest.mark.gpu


def test_static_forces_match_the_solver_forces_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_10487_gb300 import build
    build.build()
    import paper_2006_10487_gb300 as H

    case = make_case("hlbm_small", aoa_deg=8.0)
    sol = H.Solver(case, precision="fp64")
    xy = torch.tensor(H.hlbm_inspect(case, "xy").reshape(-1, 2), dtype=torch.float64, device="cuda")
    we = H.hlbm_inspect(case, "wall_edges").astype(np.int32).reshape(-1, 2)
    ea = torch.tensor(we[:, 0].copy(), dtype=torch.int32, device="cuda")
    eb = torch.tensor(we[:, 1].copy(), dtype=torch.int32, device="cuda")
    u0 = case.Ma / math.sqrt(3)
    qdyn = 0.5 * u0 * u0 * case.chord
    stream = torch.cuda.current_stream().cuda_stream
    lib = H.lib()
    for steps in (20, 1):  # two calls in a row, on two different states
        sol.step(steps)
        cd, cl = sol.forces()
        f = torch.tensor(sol.populations(-1), dtype=torch.float64, device="cuda").contiguous()
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.hlbm_wall_forces_static(f.data_ptr(), case.n_nodes, xy.data_ptr(), ea.data_ptr(), eb.data_ptr(),
                                         int(ea.numel()), qdyn, out.data_ptr(), stream)
        assert rc == H.HLBM_OK, H.hlbm_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = max(abs(cd[-1]), abs(cl[-1]))
        assert abs(got[0] - cd[-1]) <= 1e-12 * scale
        assert abs(got[1] - cl[-1]) <= 1e-12 * scale


def _static_call(H, f, n_nodes, xy, ea, eb, qdyn):
    import torch
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    rc = H.lib().hlbm_wall_forces_static(f.data_ptr(), n_nodes, xy.data_ptr(), ea.data_ptr(), eb.data_ptr(),
                                         int(ea.numel()), qdyn, out.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    assert rc == H.HLBM_OK, H.hlbm_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_forces_at_the_edge_limit_and_with_a_bad_index():
    """131 072 edges (the wall list repeated: 1024 first-pass blocks, so the
    final pass strides over more partials than it has threads) give the
    repeat count times the single-copy force; an edge with an end point
    outside [0, n_nodes) is skipped unread and both outputs become NaN."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_10487_gb300 as H

    case = make_case("hlbm_small", aoa_deg=8.0)
    sol = H.Solver(case, precision="fp64")
    sol.step(10)
    f = torch.tensor(sol.populations(-1), dtype=torch.float64, device="cuda").contiguous()
    xy = torch.tensor(H.hlbm_inspect(case, "xy").reshape(-1, 2), dtype=torch.float64, device="cuda")
    we = H.hlbm_inspect(case, "wall_edges").astype(np.int32).reshape(-1, 2)
    u0 = case.Ma / math.sqrt(3)
    qdyn = 0.5 * u0 * u0 * case.chord
    limit = 131072
    reps = limit // we.shape[0]
    idx = np.resize(np.arange(we.shape[0]), limit)  # whole copies, then a partial one
    big = we[idx]
    ea = torch.tensor(big[:, 0].copy(), device="cuda")
    eb = torch.tensor(big[:, 1].copy(), device="cuda")
    one = _static_call(H, f, case.n_nodes, xy, torch.tensor(we[:, 0].copy(), device="cuda"),
                       torch.tensor(we[:, 1].copy(), device="cuda"), qdyn)
    rest = limit - reps * we.shape[0]
    part = _static_call(H, f, case.n_nodes, xy, torch.tensor(we[:rest, 0].copy(), device="cuda"),
                        torch.tensor(we[:rest, 1].copy(), device="cuda"), qdyn) if rest else np.zeros(2)
    got = _static_call(H, f, case.n_nodes, xy, ea, eb, qdyn)
    want = reps * one + part
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-12 * scale
    # one edge end point out of range, in the last block
    bad = big.copy()
    bad[-1, 1] = case.n_nodes
    got = _static_call(H, f, case.n_nodes, xy, torch.tensor(bad[:, 0].copy(), device="cuda"),
                       torch.tensor(bad[:, 1].copy(), device="cuda"), qdyn)
    assert np.isnan(got).all()
    bad = we.copy()
    bad[0, 0] = -1
    got = _static_call(H, f, case.n_nodes, xy, torch.tensor(bad[:, 0].copy(), device="cuda"),
                       torch.tensor(bad[:, 1].copy(), device="cuda"), qdyn)
    assert np.isnan(got).all()
    # and the next call with valid edges is unaffected by the flags left behind
    got = _static_call(H, f, case.n_nodes, xy, torch.tensor(we[:, 0].copy(), device="cuda"),
                       torch.tensor(we[:, 1].copy(), device="cuda"), qdyn)
    assert np.array_equal(got, one)


def test_static_forces_reject_inputs_beyond_the_scratch_limit():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_10487_gb300 as H
    lib = H.lib()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.hlbm_wall_forces_static(dummy.data_ptr(), 1, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                     131072 + 1, 1.0, dummy.data_ptr(), None)
    assert rc == H.HLBM_EINVAL
    assert "limit" in H.hlbm_last_error()
