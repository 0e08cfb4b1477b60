"""Force wetting from contact angles through the calibration tables: the
strengths a lattice receives and the angle a drop then takes (GPU)."""
import ctypes
import json

import numpy as np
import pytest

from paper_1904_06881_gb300 import tlb
from paper_1904_06881_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _table(lattice):
    with open(tlb.CALIBRATION_PATH) as fh:
        return next(t for t in json.load(fh)["tables"] if t["lattice"] == lattice)


def _kappa(t, theta):
    return float(np.interp(theta, t["theta_deg"][::-1], t["kappa_w"][::-1]))


def _params_of(lat):
    p = tlb.Params()
    assert tlb.lib().tlb_get_params(lat.h, ctypes.byref(p)) == 0
    return p


def test_strengths_from_the_two_liquid_gas_angles():
    t = _table(W.D3Q27)
    th21, th31 = 100.0, 70.0
    lat = tlb.Lattice(W.D3Q27, 32, 32, 16, **W.base_params(wetting=W.WET_FORCE, theta_deg=(th21, th31, 90.0)))
    p = _params_of(lat)
    s2, s3 = _kappa(t, th21), _kappa(t, th31)
    assert abs(p.kw_rho - 0.5 * (s2 + s3)) < 1e-12 and abs(p.kw_phi - 0.5 * (s2 - s3)) < 1e-12
    lat.close()
    # explicit strengths take precedence over the table
    lat = tlb.Lattice(W.D3Q27, 32, 32, 16, **W.base_params(wetting=W.WET_FORCE, theta_deg=(th21, th31, 90.0),
                                                         kw_rho=0.05))
    p = _params_of(lat)
    assert p.kw_rho == 0.05 and p.kw_phi == 0.0
    lat.close()


def test_drop_takes_the_requested_angle():
    from paper_1904_06881_gb300 import calibrate as C

    L, theta = 128, 80.0
    mask, rho, phi = W.sessile_drop_2d(L, L, L / 4.0, xc=L / 2.0, yc=0.5)
    wl = dict(lattice=W.D2Q9, nx=L, ny=L, nz=1, mask=mask, rho=rho, phi=phi,
              params=W.base_params(wetting=W.WET_FORCE, theta_deg=(theta, theta, 90.0)))
    lat = tlb.lattice_from_workload(wl)
    lat.step(30000)
    got = C.measure(lat, lat.derived, W.D2Q9)
    print("requested %.1f deg, measured %.2f deg" % (theta, got))
    assert abs(got - theta) < 1.5
    lat.close()
