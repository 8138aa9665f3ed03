"""Host post-processing (Strouhal number, separation point, Eq. 14)."""
import numpy as np

from paper_2006_10487_gb300 import post


def test_strouhal_of_a_sampled_sinusoid():
    """A lift series oscillating at a frequency between two FFT bins, on a mean
    and with a slow drift: the refined peak recovers f to 0.5 %."""
    dt, chord, u0 = 4.0, 200.0, 0.1 / np.sqrt(3.0)
    st_true = 0.8345
    f = st_true * u0 / chord
    t = dt * np.arange(20000)  # about 19 periods
    cl = 0.3 + 0.05 * np.sin(2 * np.pi * f * t + 0.4) + 1e-6 * t / t[-1]
    st = post.strouhal(cl, dt, chord, u0)
    assert abs(st - st_true) <= 5e-3 * st_true
    assert post.strouhal(np.full(100, 0.2), dt, chord, u0) is None
    assert post.strouhal(np.where(t < t[-1] / 2, cl, np.nan), dt, chord, u0) is None
    assert post.strouhal(cl[:2000], dt, chord, u0) is None  # 1.9 periods: not resolved


def test_separation_point_from_skin_friction():
    """C_f = 0.3 - x on the upper surface changes sign at x/C = 0.3 (linear,
    so exactly); the lower surface stays attached; the stagnation region
    near the leading edge is ignored."""
    x = np.linspace(0.0, 1.0, 41)
    up = np.stack([x, np.ones_like(x), np.zeros_like(x), 0.3 - x], axis=1)
    up[0, 3] = -1.0                                   # stagnation point, x < x_min
    lo = np.stack([x, -np.ones_like(x), np.zeros_like(x), 0.1 + 0 * x], axis=1)
    w = np.concatenate([up, lo])[np.random.default_rng(0).permutation(82)]
    assert abs(post.separation_point(w, +1.0) - 0.3) <= 1e-12
    assert post.separation_point(w, -1.0) is None


def test_gain_model_with_the_papers_constants():
    """Section 6.3 of the paper: chi = 1.5e-4, n = 10, g = 1.6 and s' between
    3 and 5 give G of about 0.63."""
    for s_prime in (3.0, 4.0, 5.0):
        G = post.gain_model(1.5e-4, s_prime, 10, 1.6)
        assert 0.627 <= G <= 0.631
