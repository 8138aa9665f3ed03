"""C-ABI checks that need no GPU: the library loads, exports every declared
entry point, validates its inputs, and its host set-up (Eq. 3 operators,
Eq. 8 / Eq. 9 stencils, hole classification, wall edges, sub-step count)
matches the oracle's independent set-up."""
import os
import re

import numpy as np
import pytest

import paper_2006_10487_gb300 as H
from workloads import make_case

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2006_10487_gb300 import build
    build.build()
    return H.lib()


def test_every_declared_symbol_is_exported(built):
    hdr = open(os.path.join(ROOT, "include", "hlbm.h")).read()
    names = sorted(set(re.findall(r"\b(hlbm_[a-z_]+)\s*\(", hdr)))
    assert "hlbm_create" in names and "hlbm_step" in names
    for name in names:
        assert hasattr(built, name), name


INTEGER_TABLES = ["rowptr", "col", "is_node", "is_don", "ring", "ring_don", "wall_edges", "n_sub"]
REAL_TABLES = {"sx": 1e-12, "sy": 1e-12, "cc": 1e-14, "area": 1e-14, "xy": 0.0, "is_w": 1e-14, "ring_w": 1e-15}


@pytest.mark.parametrize("name,aoa", [("hlbm_small", 0.0), ("hlbm_small", 8.0), ("hlbm_mini2", 3.0),
                                      ("hlbm_single", 0.0)])
def test_host_setup_matches_the_oracle(built, orc, name, aoa):
    case = make_case(name, aoa_deg=aoa)
    o = orc.Oracle(case)
    for t in INTEGER_TABLES:
        a = np.array([o.n_sub]) if t == "n_sub" else o.table(t)
        b = H.hlbm_inspect(case, t)
        assert a.shape == b.shape and np.array_equal(a, b), t
    for lv in range(case.n_levels):
        typ = o.table(f"type{lv}")
        want = ((typ == 4) | (typ == 5)).astype(float)  # hole or interpolation node
        assert np.array_equal(H.hlbm_inspect(case, f"inactive{lv}"), want), f"inactive{lv}"
    for t, tol in REAL_TABLES.items():
        a, b = o.table(t), H.hlbm_inspect(case, t)
        assert a.shape == b.shape
        assert np.abs(a - b).max() <= tol * max(1.0, np.abs(a).max()), t


def test_rejects_bad_inputs(built):
    case = make_case("hlbm_small")
    with pytest.raises(H.HlbmError, match="n_levels"):
        case2 = make_case("hlbm_small")
        case2.levels = np.zeros((0, 4), np.int32)
        H.hlbm_inspect(case2, "n_sub")
    bad = make_case("hlbm_small")
    bad.tri = bad.tri[:, ::-1].copy()  # clockwise triangles
    with pytest.raises(H.HlbmError, match="inverted"):
        H.hlbm_inspect(bad, "n_sub")
    big_hole = make_case("hlbm_small")
    big_hole.hole = (70.0, 50.0, 90.0, 20.0)  # reaches the level boundary
    with pytest.raises(H.HlbmError, match="hole"):
        H.hlbm_inspect(big_hole, "n_sub")
    small_hole = make_case("hlbm_small")
    small_hole.hole = (70.0, 50.0, 3.0, 1.0)  # inside the airfoil, not covered by triangles
    with pytest.raises(H.HlbmError, match="outside the mesh"):
        H.hlbm_inspect(small_hole, "n_sub")
    lv = make_case("hlbm_mini2")
    lv.levels = np.array([[96, 48, 0, 0], [98, 65, 24, 8]], np.int32)  # even fine size
    with pytest.raises(H.HlbmError, match="odd"):
        H.hlbm_inspect(lv, "n_sub")
    with pytest.raises(H.HlbmError, match="positive"):
        H.hlbm_inspect(make_case("hlbm_small", Re=-1.0), "n_sub")
    with pytest.raises(H.HlbmError, match="unknown table"):
        H.hlbm_inspect(case, "nope")


def test_rejects_corrupt_and_non_finite_inputs(built):
    """Host-side fault injection: corrupted mesh arrays and non-finite or
    out-of-range parameters are refused by the set-up (no GPU involved)."""
    c = make_case("hlbm_small")
    c.xy = c.xy.copy()
    c.xy[17, 1] = np.nan
    with pytest.raises(H.HlbmError, match="finite"):
        H.hlbm_inspect(c, "n_sub")
    c = make_case("hlbm_small")
    c.tri = c.tri.copy()
    c.tri[5, 2] = c.n_nodes + 3
    with pytest.raises(H.HlbmError, match="out of range"):
        H.hlbm_inspect(c, "n_sub")
    c = make_case("hlbm_small")
    c.hole = (70.0, np.inf, 30.0, 20.0)
    with pytest.raises(H.HlbmError, match="finite"):
        H.hlbm_inspect(c, "n_sub")
    c = make_case("hlbm_small")
    c.tri = c.tri.copy()
    c.tri[9, [1, 2]] = c.tri[9, [2, 1]]  # one triangle turned clockwise
    with pytest.raises(H.HlbmError, match="manifold|inverted"):
        H.hlbm_inspect(c, "n_sub")
    c = make_case("hlbm_small")
    c.kind = c.kind.copy()
    c.kind[3] = 7
    with pytest.raises(H.HlbmError, match="kind"):
        H.hlbm_inspect(c, "n_sub")
    with pytest.raises(H.HlbmError, match="precision"):
        H.hlbm_inspect(make_case("hlbm_small"), "n_sub", precision=5)
    for kw in ({"Re": np.inf}, {"Ma": 1.5}, {"Ma": np.nan}, {"aoa_deg": np.nan}):
        with pytest.raises(H.HlbmError):
            H.hlbm_inspect(make_case("hlbm_small", **kw), "n_sub")
    assert H.hlbm_inspect(make_case("hlbm_small"), "n_sub")[0] > 0  # the unmodified case passes


def test_explicit_sub_steps_are_kept(built):
    case = make_case("hlbm_mini2")
    assert H.hlbm_inspect(case, "n_sub", n_sub=37)[0] == 37


def test_batch_create_rejects_bad_arguments(built):
    import ctypes as C
    import paper_2006_10487_gb300 as H
    L = H.lib()
    out = C.c_void_p()
    assert L.hlbm_batch_create(None, 0, None, C.byref(out)) == H.HLBM_EINVAL
    arr = (C.c_void_p * 2)(None, None)
    assert L.hlbm_batch_create(arr, 2, None, C.byref(out)) == H.HLBM_EINVAL
    assert out.value is None
    assert "NULL" in L.hlbm_batch_last_error(None).decode()


@pytest.mark.parametrize("aoa", [0.0, 8.0])
def test_wall_geometry_matches_oracle(built, orc, aoa):
    """Host set-up of the wall coefficients (chord position, side, |N_P|,
    normal, downstream tangent) against the oracle's."""
    import paper_2006_10487_gb300 as H
    case = make_case("hlbm_small", aoa_deg=aoa)
    geo = H.hlbm_inspect(case, "wall_geo").reshape(-1, 7)
    w = orc.Oracle(case).wall_coeffs()
    assert geo.shape[0] == w.shape[0]
    assert np.allclose(geo[:, 0], w[:, 0], atol=1e-12)
    off = np.abs(w[:, 1] - geo[:, 1]) > 0
    assert off.sum() <= 2  # leading / trailing edge lie on the chord line
    assert np.allclose(geo[:, 2:], w[:, 5:], rtol=1e-12, atol=1e-13)
