"""Physics pins of the oracle: Laplace's law for the liquid-gas pairs and the
Washburn capillary-filling law (Sec. III bubble test, Sec. V).

- Laplace: a 2D drop in gas has dP = gamma / R; dP R agrees for R = 18 and 22
  within 3% and down to R = 14 within 5%, and a liquid-2 and a liquid-3 drop
  give the same gamma (set 1 is symmetric in the two liquids: gamma_12 =
  gamma_13).
- Washburn (Eqs. capforce, viscousforce, Washburn, Washburnprefactor): the
  capillary force 2 gamma cos(theta) balances Poiseuille friction.  At this
  density ratio (14) the gas column ahead of the meniscus also dissipates, so
  the balance reads d/dt[(rho_l - rho_g) x^2/2 + rho_g L x] = gamma cos(theta)
  H / (6 nu) (the paper's law when rho_g -> 0).  As in the paper, theta is the
  mean dynamic angle of the meniscus over the analysis window (the second
  half of the run).  Pinned: the rates for theta = 45 and 60 deg scale as
  their mean cos(theta) (within 5%), and the prefactor K (the square root of
  the rate ratio: x^2 grows as K^2 t) lies within 10% of the prediction
  (measured 0.92 and 0.93).  In this short channel (H = 24, x/H of 3 to 5
  in the window) the flow into the entrance and the diffuse meniscus add
  friction the law leaves out, a share that falls as the column grows; on
  the paper's channel (L = 2000, H = 70, run on the GPU library) K agrees
  within 5%.
"""
import numpy as np
import pytest

import oracle
from paper_1904_06881_gb300 import workloads as W


def _laplace(R, liquid, n=64, steps=6000):
    mask, rho, phi = W.sessile_drop_2d(n, n, R, xc=n / 2, yc=n / 2, walls=(), liquid=liquid)
    wl = dict(lattice=W.D2Q9, nx=n, ny=n, nz=1, params=W.base_params(), mask=mask, rho=rho, phi=phi)
    o = oracle.from_workload(wl)
    o.step(steps)
    p = o.aux("p0")[0]
    return (p[n // 2, n // 2] - p[0, 0]) * R


@pytest.fixture(scope="module")
def gamma_lg():
    return _laplace(18.0, 2)


@pytest.mark.slow
def test_laplace_liquid_gas_pairs(gamma_lg):
    """Laplace's law for the liquid-gas pairs: dP R constant across radii, to
    3 % between R = 18 and 22 (measured 0.3 %) and 5 % down to R = 14
    (2.9 %: the interface, about 4 nodes wide, is no longer thin against
    R); C2 and C3 bubbles alike (set 1 is symmetric)."""
    g22 = _laplace(22.0, 2, n=80)
    assert abs(g22 / gamma_lg - 1.0) < 0.03
    g14 = _laplace(14.0, 2)
    assert abs(g14 / gamma_lg - 1.0) < 0.05
    g14_3 = _laplace(14.0, 3)
    assert abs(g14_3 - g14) <= 1e-8 * abs(g14)


def _filling(theta, nx=384, ny=40, wall=8, x_in=96, x_out=352, steps=10000, every=500):
    wl = W.c1_capillary(nx=nx, ny=ny, wall=wall, x_in=x_in, x_out=x_out)
    wl["params"] = W.base_params(wetting=W.WET_GEOM_INTERP, theta_deg=(theta, 60.0, 120.0))
    o = oracle.from_workload(wl)
    d = o.derived
    half = 0.5 * (d["rho_l"] + d["rho_g"])
    H = ny - 2 * wall
    ts, xs, cs = [], [], []
    for k in range(steps // every):
        o.step(every)
        r = o.fields()["rho"][0]
        ys = np.arange(wall, ny - wall)
        fx = []
        for y in ys:                        # rho = (rho_l + rho_g)/2 along each row
            row = r[y]
            i = x_in + np.where(row[x_in:x_out] < half)[0][0]
            fx.append(i - 1 + (row[i - 1] - half) / (row[i - 1] - row[i]))
        fx, yy = np.array(fx), ys.astype(float)
        # circle through the meniscus; a circular meniscus spanning the channel
        # meets the walls at cos(theta) = (H/2)/R
        A = np.vstack([fx, yy, np.ones_like(fx)]).T
        Dc, Ec, Fc = np.linalg.lstsq(A, -(fx ** 2 + yy ** 2), rcond=None)[0]
        Rm = np.sqrt(Dc ** 2 / 4 + Ec ** 2 / 4 - Fc)
        ts.append((k + 1) * every)
        xs.append(fx[len(fx) // 2] - x_in)
        cs.append(min(1.0, 0.5 * H / Rm))
    ts, xs, cs = np.array(ts, float), np.array(xs), np.array(cs)
    sel = ts >= ts[-1] / 2
    rl, rg = d["rho_l"], d["rho_g"]
    s = (rl - rg) * xs ** 2 / 2 + rg * (x_out - x_in) * xs
    rate = np.polyfit(ts[sel], s[sel], 1)[0]
    return rate, cs[sel].mean(), H


@pytest.mark.slow
def test_washburn_filling_rate(gamma_lg):
    nu = 1.0 / 6.0
    r45, c45, H = _filling(45.0)
    r60, c60, _ = _filling(60.0)
    assert abs((r45 / r60) / (c45 / c60) - 1.0) < 0.05
    for rate, c in ((r45, c45), (r60, c60)):
        pred = gamma_lg * c * H / (6.0 * nu)
        assert 0.90 < np.sqrt(rate / pred) < 1.05, (rate, pred)
