"""Post-processing of HLBM results on the host (numpy): the Strouhal number of
the lift series, the separation point from the mean skin friction of Eq. 13,
and the gain indicator of Eq. 14.  These read results the CUDA path produced
(force series, hlbm_wall_stats); none of them is on the time-stepping path.
"""
from __future__ import annotations

import numpy as np


def strouhal(cl, dt, chord, u0, skip=0):
    """St = f C / u0 of the dominant frequency f of the lift series.

    cl: one sample every dt finest-level time units (a coarse step is
    2^(L-1) of them); chord, u0 in finest-level units.  The series after
    `skip` samples has its mean removed and a Hann window applied; the peak of
    the magnitude spectrum (bins 1..) is refined by a parabola through the log
    magnitudes of the peak bin and its two neighbours.  Returns None for a
    series with no oscillation."""
    x = np.asarray(cl, dtype=np.float64)[skip:]
    n = x.size
    if n < 8 or not np.all(np.isfinite(x)):
        return None
    m = x.mean()
    x = x - m
    if np.abs(x).max() <= 1e-12 * max(1.0, abs(m)):
        return None
    spec = np.abs(np.fft.rfft(x * np.hanning(n)))
    k = 1 + int(np.argmax(spec[1:]))
    if k < 3:  # fewer than three periods in the series: no frequency resolved
        return None
    delta = 0.0
    if 1 <= k < spec.size - 1 and spec[k - 1] > 0 and spec[k + 1] > 0:
        a, b, c = np.log(spec[k - 1]), np.log(spec[k]), np.log(spec[k + 1])
        den = a - 2 * b + c
        if den != 0:
            delta = 0.5 * (a - c) / den
    f = (k + delta) / (n * dt)
    return f * chord / u0


def separation_point(wall, side=1.0, x_min=0.02):
    """Chord position (x/C) where the mean skin friction on one surface first
    turns from positive to non-positive going downstream (zero with a negative
    gradient), linearly interpolated; None if it never does.

    wall: rows of hlbm_wall_stats / Solver.wall_stats (columns x/C, side, C_p,
    C_f, ...); side: +1 upper surface, -1 lower surface; rows with
    x/C < x_min (the stagnation region) are ignored; None also for non-finite
    input."""
    w = np.asarray(wall, dtype=np.float64)
    if not np.all(np.isfinite(w[:, :4])):
        return None
    w = w[(w[:, 1] == side) & (w[:, 0] >= x_min)]
    w = w[np.argsort(w[:, 0])]
    x, cf = w[:, 0], w[:, 3]
    for i in range(x.size - 1):
        if cf[i] > 0.0 >= cf[i + 1]:
            return float(x[i] + (x[i + 1] - x[i]) * cf[i] / (cf[i] - cf[i + 1]))
    return None


def gain_model(chi, s_prime, n_sub, g):
    """Eq. 14: G = T_h / T_eq = (1 + chi s' n) / g, with chi the ratio of
    unstructured to structured node updates per finest step, s' the time of
    one finite-volume node update over that of one lattice node update, n the
    finite-volume sub-steps per lattice step and g the ratio of the node count
    an equivalent uniform lattice needs to the structured node updates per
    finest step.  G < 1: the hybrid method is cheaper."""
    return (1.0 + chi * s_prime * n_sub) / g
