"""Comparison measures of the package (Section 3: Eq. 4, CV, aligned APs,
APD90) against closed forms, and against the oracle's independent versions."""
import numpy as np
import pytest

from oracle import metrics as om
from paper_2011_04747_gb300 import metrics as pm


def _ap(t, t_up, v_rest=-85.0, v_peak=30.0, plateau=300.0):
    """Synthetic AP: 1 ms quadratic upstroke from t_up (steepest at its end),
    then a linear fall back to rest over `plateau` ms."""
    v = np.full_like(t, v_rest)
    up = (t >= t_up) & (t < t_up + 1.0)
    v[up] = v_rest + (t[up] - t_up) ** 2 * (v_peak - v_rest)
    down = (t >= t_up + 1.0) & (t < t_up + 1.0 + plateau)
    v[down] = v_peak - (t[down] - t_up - 1.0) / plateau * (v_peak - v_rest)
    return v


def test_nrmse_closed_form():
    ref = np.linspace(-3.0, 5.0, 101)
    assert pm.nrmse(ref + 0.4, ref) == pytest.approx(0.4 / 8.0, rel=1e-14)
    assert pm.nrmse(ref, ref) == 0.0
    assert np.isnan(pm.nrmse(ref, np.ones(7)[:1].repeat(101)))


def test_conduction_velocity_of_a_planar_front():
    x = np.linspace(0.0, 4.0, 81)
    act = 5.0 + x / 0.061
    act[:3] = -1.0                       # never activated: ignored
    assert pm.conduction_velocity(x, act) == pytest.approx(0.061, rel=1e-12)


def test_aligned_max_dv_removes_a_time_shift_but_not_an_offset():
    t = np.arange(5000) * 0.1
    a = _ap(t, 50.0)
    b = _ap(t, 73.4)
    assert pm.aligned_max_dv(t, a, b, 50.0, 73.4) < 1e-9
    assert pm.aligned_max_dv(t, a, b + 0.25, 50.0, 73.4) == pytest.approx(0.25, abs=1e-9)
    # unaligned, the same traces differ by most of the upstroke
    assert pm.aligned_max_dv(t, a, b, 50.0, 50.0) > 100.0
    # a 20 mV distortion of the upstroke only: seen over the whole trace, not
    # from 5 ms after activation on
    c = b.copy()
    c[(t >= 73.4) & (t < 74.4)] += 20.0
    assert pm.aligned_max_dv(t, a, c, 50.0, 73.4) == pytest.approx(20.0, abs=1e-9)
    assert pm.aligned_max_dv(t, a, c, 50.0, 73.4, after=5.0) < 1e-9


def _smooth_ap(t, t_mid, rest=-85.0, amp=115.0, width=0.1, hold=5.0, fall=300.0):
    """Logistic upstroke of steepest slope at t_mid, held for `hold` ms, then a
    linear fall of `amp` over `fall` ms: APD90 = hold + 0.9 fall (to e^-50)."""
    v = rest + amp / (1.0 + np.exp(-(t - t_mid) / width))
    late = t > t_mid + hold
    v[late] -= (t[late] - t_mid - hold) * amp / fall
    return v


def test_apd90_of_a_synthetic_ap():
    t = np.arange(12000) * 0.05
    for t_mid in (40.0, 40.0123, 40.031):
        # steepest slope between samples: found to a small part of the 0.05 ms step
        assert pm.apd90(t, _smooth_ap(t, t_mid)) == pytest.approx(5.0 + 0.9 * 300.0, abs=0.005)
    # with the 0.1 ms sampling of the probes
    t = np.arange(6000) * 0.1
    assert pm.apd90(t, _smooth_ap(t, 50.037)) == pytest.approx(275.0, abs=0.02)
    assert np.isnan(pm.apd90(t[:1000], _smooth_ap(t, 50.0)[:1000]))     # cut before repolarisation


def test_package_and_oracle_measures_agree():
    rng = np.random.default_rng(2011047)
    ref = rng.normal(size=500)
    got = ref + rng.normal(scale=0.1, size=500)
    assert pm.nrmse(got, ref) == pytest.approx(om.nrmse(got, ref), rel=1e-12)
    x = np.sort(rng.uniform(0, 3, 60))
    act = 2.0 + x / 0.05 + rng.normal(scale=0.2, size=60)
    assert pm.conduction_velocity(x, act) == pytest.approx(om.conduction_velocity(x, act), rel=1e-9)
    t = np.arange(0.0, 400.0, 0.1)
    a, b = _ap(t, 30.0), _ap(t, 42.0) + rng.normal(scale=0.01, size=t.size)
    assert pm.aligned_max_dv(t, a, b, 30.0, 41.9) == pytest.approx(om.aligned_max_dv(t, a, b, 30.0, 41.9),
                                                                   rel=1e-12)


def test_oracle_apd90_of_a_synthetic_ap():
    """The oracle's APD90 (start at the sample interval of largest rise, no
    sub-sample refinement) against the closed form of the synthetic AP: within
    half a sampling step, and exact when the steepest point is an interval
    midpoint."""
    for dt in (0.05, 0.1):
        t = np.arange(int(600 / dt)) * dt
        for t_mid in (40.0 + dt / 2, 40.0123, 40.031):
            got = om.apd90(t, _smooth_ap(t, t_mid))
            assert got == pytest.approx(275.0, abs=0.5 * dt + 0.005)
        assert om.apd90(t, _smooth_ap(t, 40.0 + dt / 2)) == pytest.approx(275.0, abs=0.005)
    t = np.arange(6000) * 0.1
    assert np.isnan(om.apd90(t[:1000], _smooth_ap(t, 50.0)[:1000]))
    # the package's refined value and the oracle's agree to the sampling step
    assert abs(om.apd90(t, _smooth_ap(t, 50.037)) - pm.apd90(t, _smooth_ap(t, 50.037))) <= 0.1
