"""Host-side checks of the synthetic geometry helpers (no GPU)."""
import math

import numpy as np

from workloads import make_case, naca0012_half_thickness, thickness_modes


def test_thickness_modes_move_the_wall_by_the_bump_and_spare_the_interface():
    """Mode m moves wall node k by (0, +-C sin(m pi x_k)) (x_k its chord
    fraction; + upper, - lower surface), ring j of the same mesh line by that
    times 1 - j / n_layers, and the outer interface ring not at all."""
    case = make_case("hlbm_small")
    nt, nl = case.n_theta, case.n_layers
    modes = thickness_modes(case, 12)
    assert modes.shape == (12, case.n_nodes, 2)
    assert np.all(modes[:, :, 0] == 0.0)
    le_x, le_y = case.pivot[0] - 0.25 * case.chord, case.pivot[1]
    wall = case.xy[:nt]
    x = np.clip((wall[:, 0] - le_x) / case.chord, 0.0, 1.0)
    upper = wall[:, 1] >= le_y
    for m in (1, 5, 12):
        dy = modes[m - 1, :nt, 1]
        expect = np.where(upper, 1.0, -1.0) * case.chord * np.sin(m * math.pi * x)
        # leading and trailing edge sit on the chord line: either sign is fine there
        on_chord = np.abs(wall[:, 1] - le_y) < 1e-9
        assert np.allclose(dy[~on_chord], expect[~on_chord], atol=1e-12)
        assert np.allclose(np.abs(dy[on_chord]), np.abs(expect[on_chord]), atol=1e-12)
        assert np.all(modes[m - 1, nl * nt:, :] == 0.0)  # interface ring
        j = 10
        assert np.allclose(modes[m - 1, j * nt:(j + 1) * nt, 1], (1.0 - j / nl) * dy)


def test_first_thickness_mode_scales_the_section():
    """Adding A sin(pi x) to t(x) moves the upper wall up and the lower wall
    down: for small A the half thickness of the moved section at x grows by
    A C sin(pi x), measured on the displaced wall nodes."""
    case = make_case("hlbm_small")
    nt = case.n_theta
    A = 1e-3
    moved = case.xy[:nt] + A * thickness_modes(case, 1)[0, :nt]
    le_x, le_y = case.pivot[0] - 0.25 * case.chord, case.pivot[1]
    x = (case.xy[:nt, 0] - le_x) / case.chord
    half = np.abs(moved[:, 1] - le_y) / case.chord
    inner = (x > 0.05) & (x < 0.95)
    assert np.allclose(half[inner], naca0012_half_thickness(x[inner]) + A * np.sin(math.pi * x[inner]), atol=1e-9)


def test_moved_case_keeps_the_input_arrays():
    from paper_2006_10487_gb300.shape import _moved_case
    case = make_case("hlbm_mini2")
    modes = thickness_modes(case, 2)
    m = _moved_case(case, [0.01, -0.02], 4.0, modes)
    assert m.aoa_deg == 4.0 and case.aoa_deg == 0.0
    assert np.allclose(m.xy, case.xy + 0.01 * modes[0] - 0.02 * modes[1])
    assert m.tri is case.tri and m.kind is case.kind
