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
