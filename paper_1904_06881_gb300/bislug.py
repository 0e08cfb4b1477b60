"""Self-propelled bi-slug (Sec. VI): a train of a C2 and a C3 slug in a
periodic channel, driven by the wetting imbalance of the geometric
interpolation method, advanced by the library.

  * centroid: the x centre of mass of the liquid (C2 + C3) in the channel
    rows, as a circular mean on the periodic ring, unwrapped over time;
  * run: steps a lattice and samples the centroid every `every` steps; the
    velocity is its finite difference;
  * theory: the long-train law of Eqs. capillaryforce-bislugrelaxation,
    Delta gamma = gamma_23 cos theta_23 - gamma_13 cos theta_31 + gamma_12 cos
    theta_21, v_inf = H Delta gamma / (6 rho_l nu L), tau_rel = H^2 / (12 nu);
    with rho_g > 0 the gas columns (total length L_g) add their Poiseuille
    friction, v_inf = H Delta gamma / (6 nu (rho_l L + rho_g L_g)) (the
    paper's law when rho_g -> 0).

    python -m paper_1904_06881_gb300.bislug [--H 39 --L 1500 --gas 400 --steps 20000]
"""
import argparse
import math
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    __package__ = "paper_1904_06881_gb300"

from . import tlb  # noqa: E402
from . import workloads as W  # noqa: E402


def centroid(C, prev=None):
    """Liquid centre of mass along x of concentrations C (3, ny, nx) of a
    channel with solid rows 0 and ny - 1: circular mean on the ring of nx
    nodes, taken nearest to `prev` (unwrapping) when given, else in [0, nx)."""
    liq = (C[1, 1:-1] + C[2, 1:-1]).sum(axis=0)
    nx = liq.shape[0]
    ang = 2.0 * np.pi * np.arange(nx) / nx
    xc = (math.atan2(float((liq * np.sin(ang)).sum()), float((liq * np.cos(ang)).sum())) / (2.0 * np.pi)) * nx
    if prev is not None:
        xc += nx * round((prev - xc) / nx)
    else:
        xc %= nx                              # first sample in [0, nx)
    return xc


def run(wl, steps, every=500, lat=None):
    """(t, x_cm) sampled every `every` steps (t = 0 included)."""
    own = lat is None
    lat = tlb.lattice_from_workload(wl) if own else lat
    ts, xs = [0], [centroid(lat.fields()["C"][:, 0])]
    for k in range(steps // every):
        lat.step(every)
        ts.append((k + 1) * every)
        xs.append(centroid(lat.fields()["C"][:, 0], xs[-1]))
    if own:
        lat.close()
    return np.array(ts, float), np.array(xs)


def theory(H, L, gammas, thetas, rho_l, rho_g=0.0, L_gas=0.0, nu=1.0 / 6.0):
    """v_inf and tau_rel of the long-train law; gammas = (g12, g13, g23),
    thetas = (theta_21, theta_31, theta_23) in degrees."""
    g12, g13, g23 = gammas
    t21, t31, t23 = (math.radians(t) for t in thetas)
    dg = g23 * math.cos(t23) - g13 * math.cos(t31) + g12 * math.cos(t21)
    v = H * dg / (6.0 * nu * (rho_l * L + rho_g * L_gas))
    return dict(delta_gamma=dg, v_inf=v, tau_rel=H * H / (12.0 * nu))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--H", type=int, default=39)
    ap.add_argument("--L", type=int, default=1500)
    ap.add_argument("--gas", type=int, default=400)
    ap.add_argument("--theta", type=float, default=60.0)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=1000)
    a = ap.parse_args(argv)
    wl = W.bislug_2d(H=a.H, L1=a.L // 2, L2=a.L - a.L // 2, gas=a.gas, theta=a.theta)
    t0 = time.perf_counter()
    ts, xs = run(wl, a.steps, a.every)
    secs = time.perf_counter() - t0
    v = np.diff(xs) / np.diff(ts)
    print("bi-slug %dx%d (H %d, L %d, gas %d), theta %.0f deg: %d steps in %.2f s" % (
        wl["nx"], wl["ny"], a.H, a.L, a.gas, a.theta, a.steps, secs))
    for t, x, vv in zip(ts[1:], xs[1:], v):
        print("  t %7d  x_cm %10.3f  v %.6f" % (t, x, vv))


if __name__ == "__main__":
    main()
