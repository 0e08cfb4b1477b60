"""Pins against values the paper prints (fixtures under tests/golden/).

- Table 1: the Neumann angles printed beside each parameter set follow from the
  printed surface tensions through the oracle's cosine relations (Eqs.
  theta1fromtension-theta3fromtension), within the printing precision; set 4
  forms no triangle.  The oracle's liquid-liquid bubble test gives the printed
  gamma_23 of sets 1 and 2.  The parameter set the workloads use is set 1.
- Sec. IV.B, geometric interpolation in 2D: each printed exact case satisfies
  tan(theta - 90 deg) = offset, and the oracle's ghost (Eq. interp2D) at that
  angle is the stored value c_{i+offset,k+1} on a field that is not linear.
- Table 2: the subspace definitions of the surface-tension sweep are the
  printed ones; on subspace 4 the oracle's gamma_23 follows Eq. tension23
  with no gas in the liquid-liquid interface, as Sec. III states.
"""
import itertools
import math
import os
import re

import numpy as np
import pytest

import oracle
import oracle.tension as OT
from paper_1904_06881_gb300 import tension as T
from paper_1904_06881_gb300 import workloads as W

from test_oracle_thermo import _mk

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def _table1():
    out = {}
    for r in _rows("table1_parameter_sets.txt"):
        v = [float(x) for x in r[1:]]
        out[int(r[0])] = dict(lam=tuple(v[0:3]), kappa=tuple(v[3:6]), gamma=tuple(v[6:9]), theta=tuple(v[9:12]))
    return out


@pytest.mark.parametrize("k", [1, 2, 3])
def test_table1_neumann_angles_follow_from_the_printed_tensions(k):
    """Each printed angle lies inside the range the oracle's Neumann angles
    take over the box gamma +- 0.0005 (three printed decimals), widened by
    0.05 deg (one printed decimal).  Over so small a box each angle is
    monotone in each tension, so the corners bound it.  Set 2 has three
    different tensions, so an exchanged pair in any relation fails it."""
    s = _table1()[k]
    corners = [OT.neumann(*(g + d for g, d in zip(s["gamma"], ds)))
               for ds in itertools.product((-5e-4, 5e-4), repeat=3)]
    centre = OT.neumann(*s["gamma"])
    for j in range(3):
        lo = min(c[j] for c in corners) - 0.05
        hi = max(c[j] for c in corners) + 0.05
        assert lo <= s["theta"][j] <= hi, (k, j, s["theta"][j], centre[j], lo, hi)
    assert abs(sum(centre) - 360.0) < 1e-9


def test_table1_set4_forms_no_triangle():
    """Set 4 prints no angles: gamma_12 > gamma_13 + gamma_23, so every cosine
    of the Neumann relations leaves [-1, 1]."""
    s = _table1()[4]
    assert all(math.isnan(t) for t in s["theta"])
    assert all(math.isnan(t) for t in OT.neumann(*s["gamma"]))
    g12, g13, g23 = s["gamma"]
    assert g12 > g13 + g23


def _gamma23_laplace(s, R_):
    """gamma_23 = dP R of a C2 disc of radius R in C3 (both liquids at
    rho_l, tanh edge of width 2), 64^2 or 80^2 periodic, by the oracle."""
    n, steps = (64, 4000) if R_ <= 16 else (80, 6000)
    o = _mk(n, n, lam=s["lam"], kappa=s["kappa"])
    rl = o.derived["rho_l"]
    y, x = np.mgrid[0:n, 0:n].astype(float)
    C2 = 0.5 * (1 - np.tanh((np.hypot(x - n / 2, y - n / 2) - R_) / 2))
    o.init_fields(np.full((1, n, n), rl), (5.0 * (2 * C2 - 1))[None])
    o.step(steps)
    p = o.aux("p0")[0]
    return (p[n // 2, n // 2] - p[0, 0]) * R_


@pytest.mark.slow
@pytest.mark.parametrize("k,R_", [(1, 16.0), (2, 16.0), (2, 20.0)])
def test_table1_gamma23_from_a_liquid_liquid_bubble(k, R_):
    """The liquid-liquid tension of Table 1 barely depends on the density
    ratio (both liquids sit at rho_l), so the oracle's bubble test reproduces
    the printed gamma_23 of sets 1 and 2 (0.323, 0.259) within 1.5 % at this
    ratio (measured +0.6 % and 0.0 %, -0.2 % at R = 20).  Set 2 has kappa_2 !=
    kappa_3, which makes the rho-phi gradient coupling kappa' of Eq.
    InterfEnergy nonzero: the derived kappa' = (kappa_2 - kappa_3) / (4 chi
    (rho_l - rho_g)) gives 0.259, the opposite sign 0.251 and 0.249 (-3.2 %,
    -3.9 %)."""
    s = _table1()[k]
    g = _gamma23_laplace(s, R_)
    assert abs(g / s["gamma"][2] - 1.0) < 0.015, (k, R_, g)


@pytest.mark.slow
@pytest.mark.parametrize("X,Y", [(0.6, 1.0), (1.0, 0.4), (1.4, 0.8)])
def test_subspace4_gamma23_follows_the_closed_form(X, Y):
    """Sec. III on subspace 4 of Table 2 (lambda = kappa = (0.01, X, Y)):
    gamma_23 follows Eq. tension23, here (X + Y) / 6, and the density field
    does not vary across the liquid-liquid interface.  The oracle's bubble
    (R = 16) reads 0.967-0.973 of the closed form (Table 1's printed values
    of sets 1-3 lie 3 % below theirs) with at most 0.8 % gas in the
    interface.  X != Y makes kappa' nonzero: its opposite sign reads
    0.912-0.950 and lets 4-5 % gas into the interface."""
    p = T.subspace_params(4, X, Y)
    n, R_ = 64, 16.0
    o = _mk(n, n, lam=p["lam"], kappa=p["kappa"])
    rl = o.derived["rho_l"]
    y, x = np.mgrid[0:n, 0:n].astype(float)
    C2 = 0.5 * (1 - np.tanh((np.hypot(x - n / 2, y - n / 2) - R_) / 2))
    o.init_fields(np.full((1, n, n), rl), (5.0 * (2 * C2 - 1))[None])
    o.step(4000)
    pr = o.aux("p0")[0]
    g = (pr[n // 2, n // 2] - pr[0, 0]) * R_
    assert 0.955 < g / ((X + Y) / 6.0) < 0.985, (X, Y, g)
    assert o.fields()["C"][0].max() < 0.02


@pytest.mark.slow
def test_subspace4_liquid_gas_tensions_follow_their_own_liquid():
    """Sec. III on subspace 4: gamma_12 depends mainly on X = lambda_2 and
    gamma_13 on Y = lambda_3.  The oracle's bubbles (64^2, R = 16, 4000
    steps): doubling X raises gamma_12 from 0.124 to 0.227 and doubling Y
    moves it by 4e-4; exchanging the liquids (X <-> Y, C2 <-> C3) maps
    gamma_12 onto gamma_13 (set 1's phi -> -phi symmetry, here with kappa_2 !=
    kappa_3)."""
    def g(pair, X, Y):
        return OT.laplace(OT.bubble(pair, 64, 16.0, 4000, **T.subspace_params(4, X, Y)), pair)

    g0, gx, gy = g("12", 0.6, 0.6), g("12", 1.2, 0.6), g("12", 0.6, 1.2)
    assert gx - g0 > 0.5 * g0
    assert abs(gy - g0) < 0.02 * (gx - g0)
    assert abs(g("13", 1.2, 0.6) / gy - 1.0) < 1e-6


def test_workloads_use_table1_set1():
    s = _table1()[1]
    assert W.SET1["lam"] == s["lam"] and W.SET1["kappa"] == s["kappa"]
    p = W.base_params()
    assert tuple(p["lam"]) == s["lam"] and tuple(p["kappa"]) == s["kappa"]


def _interp_cases():
    """(printed theta, offset, theta read) for each printed exact case.  The
    row printed "45" with offset +1 reads 135."""
    out = []
    for th, off in _rows("interp2d_exact_cases.txt"):
        th, off = float(th), int(off)
        exact = 90.0 + math.degrees(math.atan(off))
        out.append((th, off, 135.0 if (off == 1 and th == 45.0) else th, exact))
    return out


def test_interp2d_printed_angles_meet_lattice_nodes():
    """tan(theta - 90 deg) = offset: the printed approximate angles are the
    exact ones cut to two decimals; the duplicated 45 is the typo for 135."""
    cases = _interp_cases()
    assert [c[1] for c in cases] == [-3, -2, -1, 0, 1, 2, 3]
    for printed, off, read, exact in cases:
        assert abs(read - exact) < 0.01, (printed, off, exact)
    typo = [c for c in cases if c[1] == 1][0]
    assert typo[0] == 45.0 and abs(typo[3] - 135.0) < 1e-12


def _wall_row_case(theta):
    """2D lattice, solid row 0, first fluid row 1.  rho falls along +x in
    seeded random steps (so the liquid, the phase where rho is high, lies at
    lower x and the field is not linear); phi = 0 (interface pair 1-2, c =
    rho, angle theta_21)."""
    nx, ny = 40, 8
    o = _mk(nx, ny, wetting=W.WET_GEOM_INTERP, theta_deg=(theta, 70.0, 110.0))
    d = o.derived
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, 0, :] = 1
    o.set_solid(mask)
    steps = np.random.default_rng(19040).uniform(0.01, 0.05, nx)
    line = 0.5 * (d["rho_l"] + d["rho_g"]) + 0.5 * steps.sum() - np.cumsum(steps)
    rho = np.tile(line, (1, ny, 1))
    o.init_fields(rho, np.zeros_like(rho))
    return o, line


@pytest.mark.parametrize("case", range(7))
def test_interp2d_exact_cases_take_the_stored_node(case):
    """At the exact angle the ghost is c_{i+offset,k+1} to rounding; at the
    printed (cut) angle it is within |l_par - offset| |c_{i+l1} - c_{i+l0}| of
    it, l_par = tan(theta - 90 deg) (Eq. interp2D)."""
    printed, off, read, exact = _interp_cases()[case]
    xs = np.arange(8, 32)
    o, line = _wall_row_case(exact)
    g = o.aux("rho_ghost")[0, 0, xs]
    assert np.abs(g - line[xs + off]).max() < 1e-12, (exact, off)
    o, line = _wall_row_case(read)
    g = o.aux("rho_ghost")[0, 0, xs]
    l_par = math.tan(math.radians(read - 90.0))
    dmax = np.abs(np.diff(line)).max()
    assert np.abs(g - line[xs + off]).max() <= abs(l_par - off) * dmax + 1e-12, (read, off)
    if off != 0:
        assert np.abs(g - line[xs]).min() > 0.005        # the shift is taken, not a copy


def _linear(expr, X, Y):
    total = 0.0
    for term in re.findall(r"[+-]?[^+-]+", expr):
        sign = -1.0 if term.startswith("-") else 1.0
        term = term.lstrip("+-")
        if term[-1] in "XY":
            coef = float(term[:-1]) if term[:-1] else 1.0
            total += sign * coef * (X if term[-1] == "X" else Y)
        else:
            total += sign * float(term)
    return total


@pytest.mark.parametrize("k", range(1, 9))
def test_table2_subspaces_match_the_sweep(k):
    row = [r for r in _rows("table2_subspaces.txt") if int(r[0]) == k][0]
    for X, Y in ((0.3, 0.7), (1.25, 0.45), (0.8, 1.9)):
        p = T.subspace_params(k, X, Y)
        want = [_linear(e, X, Y) for e in row[1:]]
        assert np.allclose(p["lam"] + p["kappa"], want, rtol=0, atol=1e-15), (k, X, Y)
