"""Self-propelled bi-slug (Sec. VI) on the CPU: the oracle's trajectories
pinned to the symmetries and the sign of the capillary drive, and the
package's long-train law against the oracle's.

Pins of the oracle (oracle/bislug.py), on a 240 x 21 channel (H = 19, two
slugs of 60 nodes, set 1 of Table 1, geometric interpolation):
  * reflection: the mirror image x -> -x of the initial state follows the
    mirror image of the trajectory (to 1e-8: the scheme is symmetric and the
    centroid exact);
  * no drive at theta = 90 deg: with set 1 (liquids alike) and theta_21 =
    theta_31, reflecting and exchanging the liquids maps the state onto
    itself when theta_23 = 90 deg, so the centroid stays put (Delta gamma =
    0 in Eq. capillaryforce);
  * the sign of the drive: all angles 60 deg (Delta gamma = gamma_23 cos 60 >
    0) move the train towards +x, all angles 110 deg towards -x.
The magnitude of the long-train law is not pinned: at this density ratio
(14) and train length (L/H ~ 6) the measured velocity is a fraction of it.
"""
import math

import numpy as np

import oracle.bislug as OB
from paper_1904_06881_gb300 import bislug as B
from paper_1904_06881_gb300 import workloads as W

STEPS, EVERY = 2000, 500


def test_oracle_mirror_image_follows_mirror_trajectory():
    wl = W.bislug_2d(theta=60.0)
    m = dict(wl, rho=wl["rho"][:, :, ::-1].copy(), phi=wl["phi"][:, :, ::-1].copy())
    _, xa = OB.trajectory(wl, STEPS, EVERY)
    _, xb = OB.trajectory(m, STEPS, EVERY)
    nx = wl["nx"]
    for a, b in zip(xa, xb):
        assert abs(a + b - (nx - 1)) < 1e-8, (a, b)      # node x mirrors to nx - 1 - x
    assert xa[-1] - xa[0] > 1.0


def test_oracle_no_drive_at_90_degrees_and_sign_of_drive():
    _, x90 = OB.trajectory(W.bislug_2d(theta=90.0), STEPS, EVERY)
    assert max(abs(x - x90[0]) for x in x90) < 1e-9, x90
    _, x60 = OB.trajectory(W.bislug_2d(theta=60.0), STEPS, EVERY)
    _, x110 = OB.trajectory(W.bislug_2d(theta=110.0), STEPS, EVERY)
    assert x60[-1] - x60[0] > 1.0 and x110[-1] - x110[0] < -0.5, (x60, x110)


def test_package_law_matches_oracle():
    for gam, th in (((0.3, 0.3, 0.32), (60.0, 60.0, 60.0)), ((0.2, 0.25, 0.3), (50.0, 70.0, 110.0))):
        t = B.theory(39, 1500, gam, th, W.RHO_L, W.RHO_G, 400)
        assert abs(t["v_inf"] - OB.steady_velocity(39, 1500, gam, th, W.RHO_L, W.RHO_G, 400)) < 1e-15
        assert t["tau_rel"] == 39 * 39 / 2.0


def test_package_centroid_unwraps():
    """The package centroid of a hand-made liquid blob across the periodic seam."""
    C = np.zeros((3, 5, 100))
    C[1, 1:-1, 95:] = 1.0
    C[2, 1:-1, :5] = 1.0
    assert abs(B.centroid(C) - 99.5) < 1e-9
    assert abs(B.centroid(C, prev=-0.4) - (-0.5)) < 1e-9


def _arc_side(x, y, x0, ymid, H, theta_left):
    """Indicator (tanh edge of width 4) of the side left of a circular arc
    that crosses the channel centre line at x0 and meets both walls at
    theta_left, measured in the left phase."""
    R = (H / 2.0) / abs(math.cos(math.radians(theta_left)))
    if theta_left < 90.0:
        xc = x0 + R                                       # centre on the right: left side outside
        d = np.hypot(x - xc, y - ymid) - R
        return np.where(x < xc, 0.5 * (1.0 + np.tanh(d / 2.0)), 0.0)
    xc = x0 - R                                           # centre on the left: left side inside
    d = np.hypot(x - xc, y - ymid) - R
    return np.where(x > xc, 0.5 * (1.0 - np.tanh(d / 2.0)), 1.0)


def test_dynamic_angles_of_synthetic_train():
    """Three circular interfaces of known angles (rear gas | C2 at theta_21 =
    70 deg in C2, C2 | C3 at theta_23 = 100 deg in C2, front C3 | gas at
    theta_31 = 55 deg in C3) in a channel of height 39 are measured within
    0.3 deg, wherever the train sits on the periodic ring."""
    H, nx = 39, 420
    ny = H + 2
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    ymid = (ny - 1) / 2.0
    La = _arc_side(x, y, 150.0, ymid, H, 180.0 - 70.0)
    Lb = _arc_side(x, y, 230.0, ymid, H, 100.0)
    Lc = _arc_side(x, y, 310.0, ymid, H, 55.0)
    C2, C3 = np.clip(Lb - La, 0, 1), np.clip(Lc - Lb, 0, 1)
    rl, rg = 6.0, 0.4
    for shift in (0, 250):
        c2, c3 = np.roll(C2, shift, 1), np.roll(C3, shift, 1)
        C1 = 1.0 - c2 - c3
        rho = rl + C1 * (rg - rl)
        f = dict(C=np.stack([C1, c2, c3])[:, None], rho=rho[None])
        a = B.dynamic_angles(f, rl, rg)
        assert abs(a["theta_21"] - 70.0) < 0.3, a
        assert abs(a["theta_23"] - 100.0) < 0.3, a
        assert abs(a["theta_31"] - 55.0) < 0.3, a


def test_cox_function_limits_and_symmetry():
    """Eq. Coxlful: exchanging the two fluids (theta -> pi - theta, lambda ->
    1/lambda) scales f by 1/lambda exactly; for an inviscid receding fluid
    (lambda -> 0... the advancing one alone, Voinov's limit) g(theta) ->
    theta^3 / 9 at small angles; g increases with theta."""
    for th in (0.3, 1.0, 2.0, 2.8):
        for lam in (0.5, 2.0, 14.0):
            assert math.isclose(lam * B.cox_f(math.pi - th, 1.0 / lam), B.cox_f(th, lam), rel_tol=1e-12)
    assert math.isclose(B.cox_g(0.05, 0.0), 0.05 ** 3 / 9.0, rel_tol=1e-3)
    gs = [B.cox_g(math.radians(t), 14.0) for t in (30, 60, 90, 120, 150)]
    assert all(b > a for a, b in zip(gs, gs[1:]))


def test_slip_length_recovers_a_planted_slope():
    """Dynamic angles built from Eq. Coxapparent with a known L_s give it back."""
    from scipy.optimize import brentq

    lam, tw, Lc, Ls = 14.0, 60.0, 39.0, 2.5
    m = math.log(Lc / Ls)
    g0 = B.cox_g(math.radians(tw), lam)
    cas = [1e-3, 2e-3, 4e-3]
    ths = [math.degrees(brentq(lambda t: B.cox_g(t, lam) - g0 - ca * m, 1e-3, math.pi - 1e-3)) for ca in cas]
    ls, mm = B.slip_length(ths, cas, tw, lam, Lc)
    assert math.isclose(ls, Ls, rel_tol=1e-4) and math.isclose(mm, m, rel_tol=1e-5)


def test_cox_slip_recovers_planted_slip_lengths():
    """cox_slip on angles built from Cox's relation (R25 form) for each
    interface of a train at three speeds, with a known static angle and slip
    length per interface, returns them (the static angle as the zero-speed
    intercept of the angle-speed line, within the line's curvature)."""
    from scipy.optimize import brentq

    gam = (0.2, 0.21, 0.33)                       # g12, g13, g23
    rho = (0.43, 6.14, 6.14)                      # gas, C2, C3
    nu, Lc = 1.0 / 6.0, 39.0
    planted = {"theta_21": (70.0, 3.0), "theta_23": (75.0, 6.0), "theta_31": (60.0, 2.0)}
    gmap = {"theta_21": gam[0], "theta_23": gam[2], "theta_31": gam[1]}
    runs = []
    for v in (2e-4, 4e-4, 8e-4):
        ang = {}
        for key, _, adv, rec in B.INTERFACES:
            tw, Ls = planted[key]
            lam = rho[rec] / rho[adv]
            ca = rho[adv] * nu * v / gmap[key]
            tw_adv = 180.0 - tw if key == "theta_21" else tw
            target = B.cox_g(math.radians(tw_adv), lam) + ca * math.log(Lc / Ls)
            th_adv = math.degrees(brentq(lambda t: B.cox_g(t, lam) - target, 1e-3, math.pi - 1e-3))
            ang[key] = 180.0 - th_adv if key == "theta_21" else th_adv
        runs.append((v, ang))
    out = B.cox_slip(runs, gam, rho, nu=nu, Lc=Lc)
    for key, (tw, Ls) in planted.items():
        tw_adv = 180.0 - tw if key == "theta_21" else tw
        assert abs(out[key]["theta_w"] - tw_adv) < 0.05, (key, out[key])
        assert abs(out[key]["L_s"] / Ls - 1.0) < 0.05, (key, out[key])
