"""Force-wetting calibration (the angle -> kappa^w map of Sec. IV.A, method 1)
without a GPU: the shipped tables, the registration call of the C ABI and
the contact-angle measurement of the calibration script."""
import json

import numpy as np
import pytest

from paper_1904_06881_gb300 import tlb
from paper_1904_06881_gb300 import workloads as W


def _tables():
    with open(tlb.CALIBRATION_PATH) as fh:
        return {t["lattice"]: t for t in json.load(fh)["tables"]}


def test_shipped_tables_are_monotone_and_neutral_at_zero():
    tabs = _tables()
    assert set(tabs) == {W.D2Q9, W.D3Q27}
    for t in tabs.values():
        kw, th = np.array(t["kappa_w"]), np.array(t["theta_deg"])
        assert len(kw) >= 2 and np.all(np.diff(kw) > 0) and np.all(np.diff(th) < 0)
        # a wall without wetting force is neutral (Sec. IV.A: kappa^w = 0 gives 90 deg)
        assert 0.0 in t["kappa_w"]
        assert abs(th[list(kw).index(0.0)] - 90.0) < 2.5
        # attraction lowers the angle
        assert th[-1] < 80.0
        base = W.base_params()
        for k, v in t["params"].items():
            assert np.allclose(v, base[k]), k


def test_registration_rejects_bad_tables():
    p = tlb.make_params(W.D2Q9, 8, 8, 1, **W.base_params())
    for kw, th in (([0.0], [90.0]), ([0.0, 0.1], [90.0, 95.0]), ([0.1, 0.0], [80.0, 90.0]),
                   ([0.0, np.nan], [90.0, 80.0])):
        with pytest.raises(tlb.TlbError) as e:
            tlb.tlb_set_force_calibration(p, kw, th)
        assert e.value.code == -1


def test_angles_outside_the_table_are_uncalibrated():
    assert tlb.register_force_calibration() == 2
    lo = min(_tables()[W.D2Q9]["theta_deg"])
    p = tlb.make_params(W.D2Q9, 64, 64, 1, **W.base_params(wetting=W.WET_FORCE, theta_deg=(lo - 5.0, 90.0, 90.0)))
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_create_ex(p)
    assert e.value.code == -5
    # another parameter set has no table
    p = tlb.make_params(W.D2Q9, 64, 64, 1, **W.base_params(wetting=W.WET_FORCE, theta_deg=(80.0, 80.0, 90.0),
                                                           kappa=(0.02, 1.0, 1.0)))
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_create_ex(p)
    assert e.value.code == -5


@pytest.mark.parametrize("theta", [35.0, 60.0, 90.0, 115.0, 145.0])
def test_circle_fit_recovers_exact_caps(theta):
    from paper_1904_06881_gb300 import calibrate as C

    R, wall = 30.0, 0.5
    yc = wall - R * np.cos(np.radians(theta))
    y, x = np.mgrid[0:96, 0:128].astype(float)
    rho = 3.3 - 2.85 * np.tanh((np.hypot(x - 64, y - yc) - R) / 2.0)
    rho[0] = 0.0                       # the solid row
    assert abs(C.circle_angle(C.contour_points(rho, 3.3), wall) - theta) < 0.1
