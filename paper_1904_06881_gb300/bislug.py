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
    paper's law when rho_g -> 0);
  * dynamic_angles: the apparent angle of each of the three interfaces of a
    moving train (rear gas | C2, C2 | C3, front C3 | gas), from a circle
    fitted to the interface inside the channel (Sec. VI: angles measured by
    circle fits), in the convention of Sec. IV (theta_21 in liquid C2,
    theta_23 in C2, theta_31 in C3);
  * cox_f, cox_g, slip_length: Cox's viscous bending, Eqs. Coxapparent and
    Coxlful: g(theta, lambda) - g(theta_w, lambda) = Ca ln(L_c / L_s) with
    g(theta, lambda) = int_0^theta dphi / f(phi, lambda); the slope
    m = dg/dCa over a set of speeds gives L_s = L_c exp(-m).

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


def _row_crossings(v, level):
    """Sub-node positions where v crosses `level` along a row (linear
    interpolation), with the sign of the crossing (+1 upward)."""
    d = v - level
    i = np.where(d[:-1] * d[1:] < 0)[0]
    pos = i + d[i] / (d[i] - d[i + 1])
    return pos, np.sign(d[i + 1] - d[i])


def _circle(px, py):
    A = np.column_stack([px, py, np.ones_like(px)])
    k = np.linalg.lstsq(A, -(px ** 2 + py ** 2), rcond=None)[0]
    xc, yc = -k[0] / 2.0, -k[1] / 2.0
    return xc, yc, math.sqrt(max(xc * xc + yc * yc - k[2], 0.0))


def _wall_angle_left(xc, yc, R, yw, xguess):
    """Angle between the wall y = yw and a circular interface, measured in
    the phase on the left (smaller x) of the interface near the wall."""
    h = yw - yc
    dx = math.sqrt(max(R * R - h * h, 0.0))
    xs = xc + dx if abs(xc + dx - xguess) < abs(xc - dx - xguess) else xc - dx
    # tangent (dx/dy, 1) of the circle at (xs, yw), pointing away from the wall
    # when yw is the bottom wall; the left phase lies along -x
    slope = -(yw - yc) / (xs - xc) if xs != xc else 0.0
    return math.degrees(math.acos(max(-1.0, min(1.0, -slope / math.sqrt(1.0 + slope * slope)))))


def dynamic_angles(fields, rho_l, rho_g, skip=3):
    """Apparent angles (deg) of the three interfaces of a bi-slug whose slugs
    sit in a channel with solid rows 0 and ny - 1 (fields of one lattice: C
    (3, 1, ny, nx), rho, phi): theta_21 at the rear gas | C2 interface (in
    C2), theta_23 at the C2 | C3 interface (in C2), theta_31 at the front
    C3 | gas interface (in C3).  Each interface is the level rho = (rho_l +
    rho_g)/2 (liquid-gas) or C2 = C3 (liquid-liquid) in the channel rows at
    least `skip` rows from the walls; a circle fitted to it is intersected
    with the wall planes (half a node inside the solid rows), and the angles
    at the two walls are averaged (the bottom one as is, the top one
    mirrored).  The lattice is rolled so that the liquid train does not
    wrap."""
    C = fields["C"][:, 0]
    rho = fields["rho"][0]
    ny, nx = rho.shape
    # roll the gas column's circular centre of mass to x = 0: the train then
    # lies inside [0, nx) without wrapping
    gas = C[0, 1:-1].sum(axis=0)
    ang = 2.0 * np.pi * np.arange(nx) / nx
    xg = math.atan2(float((gas * np.sin(ang)).sum()), float((gas * np.cos(ang)).sum())) / (2.0 * np.pi) * nx
    shift = -int(round(xg))
    rho = np.roll(rho, shift, axis=1)
    C = np.roll(C, shift, axis=2)
    mid = 0.5 * (rho_l + rho_g)
    rows = np.arange(1 + skip, ny - 1 - skip)
    pts = {"rear": ([], []), "ll": ([], []), "front": ([], [])}
    for y in rows:
        pos, sg = _row_crossings(rho[y], mid)
        up, dn = pos[sg > 0], pos[sg < 0]
        if len(up) == 0 or len(dn) == 0:
            continue
        xr, xf = up.min(), dn.max()
        pts["rear"][0].append(xr), pts["rear"][1].append(y)
        pts["front"][0].append(xf), pts["front"][1].append(y)
        d23 = C[1, y] - C[2, y]
        lp, lsg = _row_crossings(d23, 0.0)
        inside = (lp > xr) & (lp < xf) & (lsg < 0)
        if inside.any():
            pts["ll"][0].append(lp[inside][0]), pts["ll"][1].append(y)
    out = {}
    walls = (0.5, ny - 1.5)
    for key, (px, py) in pts.items():
        px, py = np.array(px, float), np.array(py, float)
        xc, yc, R = _circle(px, py)
        ang = []
        for k, yw in enumerate(walls):
            # the top wall is the bottom wall of the mirrored channel
            ycm = yc if k == 0 else (ny - 1) - yc
            ywm = walls[0]
            guess = px[np.argmin(py)] if k == 0 else px[np.argmax(py)]
            ang.append(_wall_angle_left(xc, ycm, R, ywm, guess))
        left = 0.5 * (ang[0] + ang[1])
        out[key] = left
    # the convention of Sec. IV: theta_21 in C2 (the right phase of the rear
    # interface), theta_23 in C2 (left of the liquid-liquid one), theta_31 in
    # C3 (left of the front one)
    return {"theta_21": 180.0 - out["rear"], "theta_23": out["ll"], "theta_31": out["front"]}


def cox_f(theta, lam):
    """f(theta, lambda) of Eq. Coxlful (theta in radians, lambda the ratio of
    the advancing to the receding fluid's dynamic viscosity)."""
    s, c = math.sin(theta), math.cos(theta)
    pt = math.pi - theta
    num = 2.0 * s * (lam * lam * (theta * theta - s * s) + 2.0 * lam * (theta * pt + s * s) + (pt * pt - s * s))
    den = lam * (theta * theta - s * s) * (pt + s * c) + (pt * pt - s * s) * (theta - s * c)
    return num / den


def cox_g(theta, lam, n=2000):
    """g(theta, lambda) = int_0^theta dphi / f(phi, lambda) (Eq. Coxapparent),
    theta in radians; composite Simpson rule on n intervals (1/f ~ phi^2/3
    near 0, smooth on (0, pi))."""
    if theta <= 0.0:
        return 0.0
    n += n % 2
    h = theta / n
    acc = 0.0
    for k in range(n + 1):
        phi = k * h
        v = 0.0 if phi == 0.0 else 1.0 / cox_f(phi, lam)
        acc += v * (1 if k in (0, n) else (4 if k % 2 else 2))
    return acc * h / 3.0


def slip_length(thetas_deg, cas, theta_w_deg, lam, Lc):
    """Slip length of Sec. VI: the slope m of g(theta, lambda) - g(theta_w,
    lambda) against Ca (least squares through the origin) is ln(L_c / L_s),
    so L_s = L_c exp(-m).  Returns (L_s, m)."""
    g0 = cox_g(math.radians(theta_w_deg), lam)
    dg = np.array([cox_g(math.radians(t), lam) - g0 for t in thetas_deg])
    ca = np.asarray(cas, float)
    m = float((ca * dg).sum() / (ca * ca).sum())
    return Lc * math.exp(-m), m


# the three interfaces of a train moving towards +x: the angle key (Sec. IV
# convention), the phase it is measured in, and the advancing and receding
# components (0 gas, 1 C2, 2 C3)
INTERFACES = (("theta_21", "rear gas | C2", 0, 1), ("theta_23", "C2 | C3", 1, 2), ("theta_31", "front C3 | gas", 2, 0))


def cox_slip(runs, gammas, rho, nu=1.0 / 6.0, Lc=39.0):
    """Slip lengths of Sec. VI from steady trains of one angle set at several
    speeds.  runs: [(v_inf, dynamic_angles dict)], gammas = (g12, g13, g23),
    rho = (rho_gas, rho_C2, rho_C3).  Per interface: the static angle theta_w
    is the intercept at zero speed of a straight line through theta(v) (Sec.
    VI: the angles vary linearly with the speed); Cox's relation is taken in
    the form that is invariant under relabelling the two fluids (the
    exchange symmetry of f): theta measured in the advancing fluid, Ca = mu_adv
    v / gamma, lambda = mu_rec / mu_adv (mu = rho nu); the slope of g(theta,
    lambda) - g(theta_w, lambda) against Ca gives L_s = L_c exp(-m).
    Returns {key: dict(theta_w, slope_deg_per_v, L_s, m, lam)}."""
    gam = {"theta_21": gammas[0], "theta_23": gammas[2], "theta_31": gammas[1]}
    out = {}
    v = np.array([r[0] for r in runs], float)
    for key, _, adv, rec in INTERFACES:
        th = np.array([r[1][key] for r in runs], float)
        # the angle in the advancing fluid: theta_21 is measured in C2, which
        # recedes at the rear interface, so the gas's angle is its supplement
        th_adv = 180.0 - th if key == "theta_21" else th
        k, th0 = np.polyfit(v, th_adv, 1)
        lam = rho[rec] / rho[adv]
        ca = rho[adv] * nu * v / gam[key]
        Ls, m = slip_length(th_adv, ca, th0, lam, Lc)
        out[key] = dict(theta_w=float(th0), slope_deg_per_v=float(k), L_s=float(Ls), m=float(m), lam=float(lam))
    return out


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
