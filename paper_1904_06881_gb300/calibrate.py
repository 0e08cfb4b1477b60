"""Force-wetting calibration: contact angle against wall strength.

The wetting force of Eq. forceBC (Sec. IV.A, method 1) is set by strengths
kappa^w, not by an angle.  Sec. IV.A maps strengths to angles by
equilibrating 2D sessile drops and fitting circular profiles (Fig.
force_angles), and the map is specific to the free-energy parameter set.
This script does that measurement with the library itself, for the
parameter set of the workloads, and writes the tables that
tlb_set_force_calibration takes (the Python binding registers them when it
loads the library):

  * a drop of liquid 2 (radius L/4, liquid 3 absent, gas around it) on the
    bottom wall of a box, kappa_phi^w = 0, for a range of kappa_rho^w, all
    advanced together by tlb_step_batch;
  * its angle from the iso-line rho = (rho_l + rho_g)/2: a least-squares
    circle through the contour points at least 3 nodes above the wall, and
    cos(theta) = (y_wall - y_centre) / R with the wall plane half a node above
    the solid row (halfway bounce-back); in 3D the same in the x-z plane
    through the drop's centre;
  * converged when the angle moves by less than 0.3 deg over the last
    `check` steps; points that did not converge, diverged, left the wall or
    are not monotone are left out (and listed in the table).  At the density
    ratio of the workloads the 2D drops are stable over 80 000 steps only for
    0 <= kappa_rho^w <= 0.2 (repelling walls detach them, stronger attraction
    diverges), so the D2Q9 table is narrow; the 3D drops converge over the
    whole sweep.

    python -m paper_1904_06881_gb300.calibrate [--out PATH]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    __package__ = "paper_1904_06881_gb300"

from . import tlb  # noqa: E402
from . import workloads as W  # noqa: E402

# thermodynamic parameter set of the tables: the workloads' set 1 (Table 1),
# Carnahan-Starling EOS at the density ratio of the workloads
PARAM_KEYS = ("lam", "kappa", "chi", "a", "b", "R", "rho_l", "rho_g")
KAPPAS = (-0.5, -0.4, -0.3, -0.2, -0.1, 0.0, 0.1, 0.2, 0.3, 0.35, 0.4)


def circle_angle(pts, wall):
    """Contact angle (deg) of the circle through pts (N x 2: tangential,
    normal coordinate) fitted by least squares, against a wall at normal
    coordinate `wall`."""
    x, y = pts[:, 0], pts[:, 1]
    A = np.column_stack([x, y, np.ones_like(x)])
    c = np.linalg.lstsq(A, -(x * x + y * y), rcond=None)[0]
    xc, yc = -0.5 * c[0], -0.5 * c[1]
    R = np.sqrt(max(xc * xc + yc * yc - c[2], 0.0))
    return float(np.degrees(np.arccos(np.clip((wall - yc) / R, -1.0, 1.0))))


def contour_points(rho2d, half, skip=3):
    """Points of the iso-line rho = half of a drop on the wall row 0 of a 2D
    cut (rows = normal direction), by linear interpolation along columns and
    along rows, rows 1 + skip and above only."""
    ny, nx = rho2d.shape
    pts = []
    for x in range(nx):
        col = rho2d[:, x]
        for y in range(1 + skip, ny - 2):
            a, b = col[y], col[y + 1]
            if (a - half) * (b - half) < 0:
                pts.append((x, y + (a - half) / (a - b)))
    for y in range(1 + skip, ny - 2):
        row = rho2d[y]
        for x in range(nx - 1):
            a, b = row[x], row[x + 1]
            if (a - half) * (b - half) < 0:
                pts.append((x + (a - half) / (a - b), y))
    return np.array(pts, float)


def drop_case(lattice, kw, L):
    p = W.base_params(wetting=W.WET_FORCE, kw_rho=float(kw), kw_phi=0.0)
    if lattice == W.D2Q9:
        mask, rho, phi = W.sessile_drop_2d(L, L, L / 4.0, xc=L / 2.0, yc=0.5)
        return dict(lattice=W.D2Q9, nx=L, ny=L, nz=1, params=p, mask=mask, rho=rho, phi=phi)
    nz = L
    z, y, x = np.mgrid[0:nz, 0:L, 0:L].astype(np.float64)
    C2 = 0.5 * (1.0 - np.tanh((np.sqrt((x - L / 2) ** 2 + (y - L / 2) ** 2 + (z - 0.5) ** 2) - L / 4.0) / 2.0))
    rho, phi = W.phase_fields(C2, np.zeros_like(C2))
    mask = np.zeros((nz, L, L), np.uint8)
    mask[0] = 1
    mask[nz - 1] = 1
    return dict(lattice=W.D3Q27, nx=L, ny=L, nz=nz, params=p, mask=mask, rho=rho, phi=phi)


def measure(lat, d, lattice):
    try:
        rho = lat.fields()["rho"]
    except tlb.TlbError:              # a strength too large for the scheme: diverged
        return float("nan")
    half = 0.5 * (d["rho_l"] + d["rho_g"])
    cut = rho[0] if lattice == W.D2Q9 else rho[:, rho.shape[1] // 2, :]
    pts = contour_points(cut, half)
    return circle_angle(pts, 0.5) if len(pts) >= 6 else float("nan")


def sweep(lattice, L, steps, check, kappas=KAPPAS, log=print):
    lats = [tlb.lattice_from_workload(drop_case(lattice, kw, L)) for kw in kappas]
    d = lats[0].derived
    tlb.tlb_step_batch([x.h for x in lats], steps - check)
    first = [measure(x, d, lattice) for x in lats]
    tlb.tlb_step_batch([x.h for x in lats], check)
    last = [measure(x, d, lattice) for x in lats]
    kw, th, dropped = [], [], []
    for k, a, b in zip(kappas, first, last):
        # a drop that left the wall (180 deg) or spread to a film (0 deg) has no contact angle
        ok = np.isfinite(a) and np.isfinite(b) and abs(a - b) < 0.3 and 1.0 < b < 179.0
        log("  kappa_rho^w %+.3f: theta %.2f deg (%.2f deg %d steps before)%s" % (k, b, a, check, "" if ok else "  [left out]"))
        if ok:
            kw.append(float(k))
            th.append(float(b))
        else:
            dropped.append(float(k))
    for x in lats:
        x.close()
    # keep the monotone part (theta decreasing in kappa^w)
    keep_k, keep_t = [], []
    for k, t in zip(kw, th):
        if keep_t and not t < keep_t[-1]:
            dropped.append(k)
            continue
        keep_k.append(k)
        keep_t.append(t)
    return keep_k, keep_t, dropped, d


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=tlb.CALIBRATION_PATH)
    args = ap.parse_args(argv)
    base = W.base_params()
    tables = []
    for lattice, L, steps, check in ((W.D2Q9, 128, 80000, 10000), (W.D3Q27, 64, 24000, 4000)):
        name = "D2Q9" if lattice == W.D2Q9 else "D3Q27"
        print("%s: drops of radius %d, %d steps" % (name, L // 4, steps), flush=True)
        t0 = time.time()
        kw, th, dropped, d = sweep(lattice, L, steps, check)
        tables.append(dict(lattice=lattice, lattice_name=name, params={k: base[k] for k in PARAM_KEYS},
                           kappa_w=kw, theta_deg=th, left_out=dropped,
                           geometry="box %d^%d, drop of liquid 2 radius %d on the wall, gas around" % (L, 2 if lattice == W.D2Q9 else 3, L // 4),
                           steps=steps, density_ratio=d["rho_l"] / d["rho_g"]))
        print("  %.1f s" % (time.time() - t0), flush=True)
    out = dict(note="force-wetting calibration written by paper_1904_06881_gb300/calibrate.py: contact angle of a "
                    "sessile drop of liquid 2 against kappa_rho^w (kappa_phi^w = 0)", tables=tables)
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
