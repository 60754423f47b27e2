"""Error and propagation metrics (Section 3).

* ``nrmse``: Eq. 4, e_Z = sqrt(mean((u_hat - u)^2)) / (u_max - u_min), u the
  reference nodal values (OST in Section 3.3), u_hat the compared ones.
* ``conduction_velocity``: slope of activation time along a line of nodes
  (least squares of distance against activation time), cm/ms.
* ``aligned_max_dv``: largest |V_a - V_b| between two voltage traces after
  shifting one by the difference of their activation times (the comparison of
  "aligned APs" in Sections 3.1 and 3.2), by linear interpolation in time.
* ``apd90``: action potential duration at 90 % repolarisation measured from
  the instant of largest dV/dt (the APD90 of Section 3.1 and e_APD of
  Eq. 4, Section 3.3).
"""
from __future__ import annotations

import numpy as np


def nrmse(u_hat, u):
    u = np.asarray(u, dtype=np.float64)
    u_hat = np.asarray(u_hat, dtype=np.float64)
    rng = u.max() - u.min()
    return float(np.sqrt(np.mean((u_hat - u) ** 2)) / rng) if rng > 0 else float("nan")


def conduction_velocity(positions, act_times):
    x = np.asarray(positions, dtype=np.float64)
    t = np.asarray(act_times, dtype=np.float64)
    ok = t >= 0
    x, t = x[ok], t[ok]
    A = np.stack([t, np.ones_like(t)], axis=1)
    slope, _ = np.linalg.lstsq(A, x, rcond=None)[0]
    return float(slope)


def aligned_max_dv(times, va, vb, act_a, act_b):
    """max |va(t) - vb(t + (act_b - act_a))| over the overlap of the two traces."""
    times = np.asarray(times, dtype=np.float64)
    shift = float(act_b - act_a)
    tb = times + shift
    ok = (tb >= times[0]) & (tb <= times[-1])
    vb_shift = np.interp(tb[ok], times, vb)
    return float(np.max(np.abs(np.asarray(va)[ok] - vb_shift))) if ok.any() else float("nan")


def apd90(times, v):
    """APD90 of the first action potential in a uniformly sampled trace.

    Start: the midpoint of the sample interval with the largest rise of V
    (the maximum of dV/dt, resolved to the sampling).  End: the first time
    after the peak at which V has fallen by 90 % of its amplitude (peak minus
    the trace's first value), interpolated linearly between samples.  NaN if
    V does not come back down that far.
    """
    times = np.asarray(times, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    jump = v[1:] - v[:-1]
    j = int(np.argmax(jump))
    t_start = 0.5 * (times[j] + times[j + 1])
    k = j + int(np.argmax(v[j:]))
    v90 = v[k] - 0.9 * (v[k] - v[0])
    after = np.nonzero(v[k:] < v90)[0]
    if after.size == 0:
        return float("nan")
    m = k + int(after[0])
    frac = (v[m - 1] - v90) / (v[m - 1] - v[m])
    return float(times[m - 1] + frac * (times[m] - times[m - 1]) - t_start)
