"""Section 3's scheme comparison on the GPU: OST, OSTAR and DAETI on a 1 x 1 cm
sheet with the spacing and conductivities of Section 3.1 (TP06 in place of
O'Hara-Rudy), 400 ms, errors against OST.

Bounds: the paper reports for DAETI against OST a CV 6.4 % higher, equal
APD90 at the centre, aligned APs within 0.34 mV (2D) and e_LAT, e_APD of
order 1e-3 and 1e-4 (3D).  The checks allow the splitting error of a
different cell model while catching a wrong operator or schedule (a
diffusion or time-step error of tens of percent moves CV and e_LAT far past
them): CV within 10 %, APD90 within 1 ms at every probe (the paper's
three APD90 values agree to the ms; e_APD itself is not bounded: on a
homogeneous sheet APD90 spans only a few ms, so its normalisation magnifies
sub-0.5 ms differences), e_LAT < 0.05 (OSTAR, whose step differs from OST's
by 25 %: < 0.01), and aligned APs within 2 mV from 5 ms after activation on
(the FP32 tolerance)."""
import pytest

import inputs as I
from parity_util import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("precision", ["fp32_kahan", "fp64"])
def test_scheme_comparison_on_the_sheet(precision):
    from parity_util import ensure_lib
    from paper_2011_04747_gb300.compare import scheme_comparison

    binding = ensure_lib()
    wl = I.aniso_sheet_2d(n=101, length=1.0, t_end=400.0)
    runs = [("ost", dict(scheme="ost", dt=0.01, precision=precision)),
            ("ostar", dict(scheme="ostar", precision=precision)),
            ("daeti", dict(scheme="daeti", precision=precision))]
    per = scheme_comparison(binding, wl, runs, probes_per_side=6)
    ost, ostar, daeti = per["ost"], per["ostar"], per["daeti"]
    assert ost["dt_ms"] == 0.01 and ostar["dt_ms"] == pytest.approx(0.0125) and daeti["dt_ms"] == 0.1
    assert daeti["l"] == 3 and daeti["k_max"] == 10 and ost["k_max"] == 1
    for r in per.values():
        assert r["all_activated"]
        assert 250.0 < r["apd90_centre_ms"] < 340.0
        assert 0.05 < r["cv_cm_per_ms"] < 0.11
    for r in (ostar, daeti):
        assert abs(r["cv_cm_per_ms"] / ost["cv_cm_per_ms"] - 1.0) < 0.10
        assert r["max_abs_dapd90_ms"] < 1.0
        assert r["aligned_max_dv_mv_from_5ms"] < 2.0
    assert ostar["e_lat"] < 0.01
    assert daeti["e_lat"] < 0.05
