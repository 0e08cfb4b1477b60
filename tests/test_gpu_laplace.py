"""Laplace's law on the GPU library at the radii the oracle cannot reach in
test time (Sec. III bubble test): for set 1, dP R of each interface pair is
the same at R = 20, 30 and 40 within 3 %, gamma_12 = gamma_13 within 1 % (the
two liquids are symmetric in set 1), and gamma_23 lies within 5 % of the
closed form alpha_23 (lambda_2 + lambda_3) / 6 (Eqs. liquidliquidalpha,
tension23).  The library's fields are held to the FP64 oracle by the parity
tests; this checks the method itself at larger sizes, and in 3D: a D3Q27
liquid-1 drop has dP = 2 gamma / R with the gamma of the D2Q9 bubbles, within
3 % (the pair's tension does not depend on the lattice).  40 000 steps: the
liquid-liquid bubble reaches its pressure jump through the Cahn-Hilliard
diffusion of phi, over a time of order L^2 / M (M = 0.5), and 8 000 steps
leave gamma_23 at R = 20, 30, 40 reading 0.326, 0.313, 0.362."""
import pytest

from helpers import record

pytestmark = pytest.mark.gpu

SET1 = dict(lam=(0.6, 1.0, 1.0), kappa=(0.01, 1.0, 1.0))


def test_laplace_across_radii():
    from paper_1904_06881_gb300 import tension as T

    gam = {}
    for R, L in ((20.0, 96), (30.0, 128), (40.0, 176)):
        res, _ = T.sweep([SET1], L=L, R=R, steps=40000)
        gam[R] = res[0]["gamma"]
        record("laplace R=%g" % R, **{"gamma_" + k: v for k, v in gam[R].items()})
    for pair in ("12", "13", "23"):
        g = [gam[R][pair] for R in gam]
        assert max(g) / min(g) - 1.0 < 0.03, (pair, g)
    for R in gam:
        assert abs(gam[R]["12"] / gam[R]["13"] - 1.0) < 0.01, gam[R]
    closed = 1.0 * (1.0 + 1.0) / 6.0            # alpha_23 = sqrt((1 + 1) / (1 + 1)) = 1
    for R in gam:
        assert abs(gam[R]["23"] / closed - 1.0) < 0.05, gam[R]


def test_laplace_3d_drop_matches_the_2d_tension():
    import math

    import numpy as np

    from paper_1904_06881_gb300 import tension as T
    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    # both at 8000 steps: the liquid-gas tension of this state drifts slowly
    # with the gas density (2D: 0.2135 at R = 20 after 8000 steps, 0.2077
    # after 40 000)
    res, _ = T.sweep([SET1], L=128, R=30.0, steps=8000)
    g2 = res[0]["gamma"]["12"]
    out = {}
    for R, n in ((20.0, 80), (28.0, 112)):
        wl = W.big_periodic_drop_3d(n, R=R)
        lat = tlb.lattice_from_workload(wl)
        lat.step(8000)
        p0 = lat.aux("p0")
        C2 = lat.fields()["C"][1]
        lat.close()
        dP = float(p0[n // 2, n // 2, n // 2] - p0[0, 0, 0])
        Rm = (3.0 * float(C2.sum()) / (4.0 * math.pi)) ** (1.0 / 3.0)
        out[R] = dP * Rm / 2.0
    record("laplace 3D drop", gamma_2d=g2, **{"gamma_3d_R%d" % int(R): v for R, v in out.items()})
    for R, g3 in out.items():
        assert abs(g3 / g2 - 1.0) < 0.03, (R, g3, g2)
