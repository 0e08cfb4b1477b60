"""Washburn capillary filling at the paper's channel (Sec. V, Eqs. capforce,
viscousforce, Washburn, Washburnprefactor) on the GPU library.

A 2D channel of length L = 2000 and height H = 70 (solid slabs 12 nodes
thick) runs between a liquid-1 reservoir and a gas reservoir, 1024 nodes
each, on a D2Q9 lattice of 4096 x 94; geometric-interpolation wetting;
beta = 0.5, so nu = 1/6.  As in the paper, the analysis window is the last
10 % of the run: x(t) = K sqrt(t - t0) is fitted there, and K is compared
with sqrt(gamma <cos theta> H / (3 nu rho_l)), where gamma is the liquid-gas
tension measured by Laplace's law on the same library and <theta> is the mean
dynamic angle of the meniscus over the window (a circle through the
rho = (rho_l + rho_g)/2 crossings).

Pinned: K within 5 % of the prediction at theta = 60 and 80 deg with
geometric interpolation (measured 0.989 and 0.991) and at 80 deg with the
force method, kappa^w from the calibration (measured 0.977: the force method
deviates more, as the paper reports).  The 60 deg run stops at 1.05 M steps,
before the liquid reservoir (1024 x 94 nodes) has emptied into the channel.
"""
import numpy as np
import pytest

from helpers import meniscus_fit, record, washburn_fit

pytestmark = pytest.mark.gpu

NU = 1.0 / 6.0


@pytest.fixture(scope="module")
def gamma_lg():
    from paper_1904_06881_gb300 import tension as T

    res, _ = T.sweep([dict(lam=(0.6, 1.0, 1.0), kappa=(0.01, 1.0, 1.0))], L=96, R=24.0, steps=4000)
    return res[0]["gamma"]["12"]


@pytest.mark.parametrize("scheme,theta,steps", [("interpolation", 60.0, 1050000), ("interpolation", 80.0, 1500000),
                                                ("force", 80.0, 1500000)])
def test_washburn_prefactor_paper_channel(gamma_lg, scheme, theta, steps):
    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    nx, ny, wall, x_in, x_out, every = 4096, 94, 12, 1024, 3024, 15000
    wl = W.c1_capillary(nx=nx, ny=ny, wall=wall, x_in=x_in, x_out=x_out)
    if scheme == "force":
        # kappa^w from the force-wetting calibration (its D2Q9 range is 75-90 deg)
        wl["params"] = W.base_params(wetting=W.WET_FORCE, theta_deg=(theta, theta, 90.0))
    else:
        wl["params"] = W.base_params(wetting=W.WET_GEOM_INTERP, theta_deg=(theta, 60.0, 120.0))
    lat = tlb.lattice_from_workload(wl)
    d = lat.derived
    half = 0.5 * (d["rho_l"] + d["rho_g"])
    H = ny - 2 * wall
    ts, xs, cs = [], [], []
    try:
        for k in range(steps // every):
            lat.step(every)
            m = meniscus_fit(lat.fields()["rho"][0], half, wall, x_in, x_out)
            assert m is not None, "meniscus lost at step %d" % ((k + 1) * every)
            ts.append((k + 1) * every)
            xs.append(m[0])
            cs.append(m[1])
    finally:
        lat.close()
    K, t0 = washburn_fit(ts, xs)
    n = len(ts)
    cos_mean = float(np.mean(cs[int(round(0.9 * n)):]))
    K_pred = np.sqrt(gamma_lg * cos_mean * H / (3.0 * NU * d["rho_l"]))
    record("washburn_paper_channel_%s_%d" % (scheme, int(theta)), K=K, K_pred=K_pred, ratio=K / K_pred,
           theta_dyn=float(np.degrees(np.arccos(cos_mean))), x_end=xs[-1], gamma=gamma_lg)
    assert xs[-1] > 700.0
    assert abs(K / K_pred - 1.0) < 0.05, (K, K_pred, np.degrees(np.arccos(cos_mean)))
