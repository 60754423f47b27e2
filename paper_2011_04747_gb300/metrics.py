"""Comparison measures of Section 3 for simulation outputs (host-side numpy).

Used by the accuracy comparison of the integration schemes (OST, OSTAR,
DAETI) on the 2D sheet:

* ``nrmse`` -- Eq. 4: root-mean-square difference of a field against the
  reference field, divided by the reference's range.
* ``conduction_velocity`` -- slope (cm/ms) of the least-squares line of
  position against activation time over the activated nodes of a line.
* ``aligned_max_dv`` -- largest voltage difference of two action potentials
  after moving the second in time so that both activate together (the
  comparison of aligned APs in Section 3.1).
* ``apd90`` -- action potential duration at 90 % repolarisation, from the
  instant of maximum upstroke velocity to the first time after the peak at
  which V falls below V_rest + 0.1 (V_peak - V_rest).
"""
from __future__ import annotations

import numpy as np


def nrmse(field, reference) -> float:
    """Eq. 4 with u = reference and u_hat = field (NaN for a constant reference)."""
    ref = np.asarray(reference, dtype=np.float64).ravel()
    got = np.asarray(field, dtype=np.float64).ravel()
    span = float(ref.max() - ref.min())
    if span <= 0.0:
        return float("nan")
    return float(np.sqrt(np.mean(np.square(got - ref))) / span)


def conduction_velocity(x, act) -> float:
    """d x / d t of the least-squares line through the activated (act >= 0) points."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(act, dtype=np.float64)
    keep = t >= 0.0
    if keep.sum() < 2:
        return float("nan")
    slope, _ = np.polyfit(t[keep], x[keep], 1)
    return float(slope)


def aligned_max_dv(t, v_a, v_b, act_a, act_b, after=None) -> float:
    """max over t of |v_a(t) - v_b(t + act_b - act_a)|, v_b linearly interpolated,
    over the times where the moved trace is defined (and, with `after`, from
    act_a + after on: the plateau and repolarisation without the upstroke,
    whose 0.1 ms samples interpolate poorly)."""
    t = np.asarray(t, dtype=np.float64)
    v_a = np.asarray(v_a, dtype=np.float64)
    v_b = np.asarray(v_b, dtype=np.float64)
    moved = t + (float(act_b) - float(act_a))
    inside = (moved >= t[0]) & (moved <= t[-1])
    if after is not None:
        inside &= t >= float(act_a) + float(after)
    if not inside.any():
        return float("nan")
    return float(np.abs(v_a[inside] - np.interp(moved[inside], t, v_b)).max())


def apd90(t, v) -> float:
    """APD90 of the first action potential of a trace (NaN if it never repolarises).

    The upstroke instant is that of the largest slope: the forward
    differences of V sit at the midpoints of the sample pairs, and the
    parabola through the largest one and its two neighbours places the
    maximum between samples (uniform sampling).  The rest level is the first
    sample, the peak the maximum after the upstroke; the end is the linearly
    interpolated first crossing of the 90 % repolarisation level after the peak.
    """
    t = np.asarray(t, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    if t.size < 3:
        return float("nan")
    rate = np.diff(v) / np.diff(t)
    j = int(np.argmax(rate))
    t_up = 0.5 * (t[j] + t[j + 1])
    if 0 < j < rate.size - 1:
        curv = rate[j - 1] - 2.0 * rate[j] + rate[j + 1]
        if curv < 0.0:
            shift = 0.5 * (rate[j - 1] - rate[j + 1]) / curv
            t_up += min(0.5, max(-0.5, shift)) * (t[j + 1] - t[j])
    rest = v[0]
    p = j + int(np.argmax(v[j:]))
    level = v[p] - 0.9 * (v[p] - rest)
    below = np.nonzero(v[p:] < level)[0]
    if below.size == 0:
        return float("nan")
    q = p + int(below[0])
    # v[q-1] >= level > v[q]
    t_end = t[q - 1] + (level - v[q - 1]) * (t[q] - t[q - 1]) / (v[q] - v[q - 1])
    return float(t_end - t_up)
