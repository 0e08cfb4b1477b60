"""GPU (CUDA, sm_103a) vs FP64 oracle on measured physical quantities, through
the C ABI: contact angles of sessile drops for the three wetting schemes
(within 0.5 deg), the meniscus track of the capillary channel (within 0.5
lattice units), and the entropic alpha away from equilibrium, where the CUDA
path leaves its series root for Halley's method (max_i |x_i| > 0.1,
x_i = (f^eq_i(u) - f_i) / f'_i; Eqs. EntropyEquation, mirror_state)."""
import numpy as np
import pytest

import oracle
from paper_1904_06881_gb300 import workloads as W

from helpers import (circle_fit_angle, gpu_from_workload, match_directions, meniscus_x, oracle_from_workload,
                     record)

pytestmark = pytest.mark.gpu

ANGLE_TOL = 0.5          # deg
MENISCUS_TOL = 0.5       # lattice units


def _drop(wet, theta=90.0, kw=0.0, n=64, R=16.0):
    mask, rho, phi = W.sessile_drop_2d(n, n, R, xc=n / 2 + 0.3, yc=0.5)
    return dict(name="drop", lattice=W.D2Q9, nx=n, ny=n, nz=1, mask=mask, rho=rho, phi=phi,
                params=W.base_params(wetting=wet, theta_deg=(theta, theta, 90.0), kw_rho=kw))


@pytest.mark.parametrize("wet,theta,kw", [(W.WET_FORCE, 90.0, 0.1), (W.WET_GEOM_EXTRAP, 60.0, 0.0),
                                          (W.WET_GEOM_INTERP, 120.0, 0.0)])
def test_contact_angle_matches_oracle(wet, theta, kw):
    """A liquid-1 drop (radius 16) on the bottom wall after 4000 steps: the
    angle of the circle fitted to the rho = (rho_l + rho_g)/2 contour is
    measured the same way on both fields."""
    wl = _drop(wet, theta, kw)
    g, o = gpu_from_workload(wl), oracle_from_workload(wl)
    g.step(4000)
    o.step(4000)
    d = o.derived
    tg = circle_fit_angle(g.fields()["rho"][0], d["rho_l"], d["rho_g"])
    to = circle_fit_angle(o.fields()["rho"][0], d["rho_l"], d["rho_g"])
    record("contact angle, wetting %d, prescribed %g deg, kappa_w %g" % (wet, theta, kw), gpu_deg=tg,
           oracle_deg=to, diff_deg=abs(tg - to), bound=ANGLE_TOL)
    assert abs(tg - to) <= ANGLE_TOL, (tg, to)


def test_capillary_meniscus_track_matches_oracle():
    """The full 1024 x 64 channel (geometric interpolation, 30/60/120 deg):
    the meniscus position inside the channel every 500 steps up to 6000."""
    wl = W.c1_capillary()
    ch = wl["channel"]
    g, o = gpu_from_workload(wl), oracle_from_workload(wl)
    d = o.derived
    y0, y1 = ch["wall"], wl["ny"] - ch["wall"]
    track = []
    for k in range(12):
        g.step(500)
        o.step(500)
        xg = meniscus_x(g.fields()["rho"][0], d["rho_l"], d["rho_g"], ch["x_in"] - 8, ch["x_out"], y0, y1)
        xo = meniscus_x(o.fields()["rho"][0], d["rho_l"], d["rho_g"], ch["x_in"] - 8, ch["x_out"], y0, y1)
        track.append((500 * (k + 1), xg, xo))
    diff = max(abs(a - b) for _, a, b in track)
    record("c1 meniscus track, 6000 steps", max_diff=diff, x_start=track[0][2], x_end=track[-1][2],
           bound=MENISCUS_TOL)
    assert track[-1][2] > track[0][2] + 2.0          # the liquid advances into the channel
    assert diff <= MENISCUS_TOL, track


def _halley_nodes(o, f, lattice):
    """Fluid nodes whose collision takes Halley's method on the GPU: max_i
    |x_i| > 0.1, computed on the host from the populations (oracle order)
    and the oracle's force of the same state."""
    c, w = oracle.lattice(lattice)
    D = 2 if lattice == W.D2Q9 else 3
    F = [o.aux(k).reshape(-1) for k in ("Fx", "Fy", "Fz")[:D]]
    rho = f.sum(0)
    idx = []
    for n in range(f.shape[1]):
        if not rho[n] > 0:
            continue
        u = (f[:, n, None] * c[:, :D]).sum(0) / rho[n]
        du = np.array([F[a][n] for a in range(D)]) / rho[n]
        ue, ud = np.zeros(3), np.zeros(3)
        ue[:D], ud[:D] = u, u + du
        fe, fd = oracle.feq(lattice, rho[n], ue), oracle.feq(lattice, rho[n], ud)
        fp = f[:, n] + fd - fe
        if np.abs((fe - f[:, n]) / fp).max() > 0.1:
            idx.append(n)
    return np.array(idx, dtype=np.int64)


def test_alpha_away_from_equilibrium_matches_oracle():
    """Every seventh fluid node of a drop is moved away from equilibrium
    (each population scaled by 1 + U[-0.15, 0.15]); one step from the same
    state on both sides.  The collisions at those nodes take Halley's method
    on the GPU (counted on the host), and the post-step populations match
    the oracle's exact root to FP32 rounding everywhere."""
    wl = _drop(W.WET_GEOM_INTERP, 60.0)
    g, o = gpu_from_workload(wl), oracle_from_workload(wl)
    g.step(300)
    perm = match_directions(wl["lattice"])
    fg, gg = g.populations()
    f, gq = fg[perm], gg[perm]
    fl = np.where(wl["mask"].reshape(-1) == 0)[0]
    o.set_populations(f, gq)
    natural = len(_halley_nodes(o, f, wl["lattice"]))
    rng = np.random.default_rng(7)
    sel = fl[::7]
    f = f.copy()
    f[:, sel] *= 1.0 + rng.uniform(-0.15, 0.15, (f.shape[0], len(sel)))
    inv = np.argsort(perm)
    g.set_populations(f[inv], gq[inv])
    o.set_populations(f, gq)
    hal = _halley_nodes(o, f, wl["lattice"])
    clipped0 = o.alpha_clipped
    g.step(1)
    o.step(1)
    assert o.alpha_clipped == clipped0            # every root lies below the positivity bound
    fg2, _ = g.populations()
    fo2, _ = o.populations()
    err = np.abs(fg2[perm][:, fl] - fo2[:, fl]).max() / np.abs(fo2[:, fl]).max()
    record("alpha on the Halley branch, one step", halley_nodes=len(hal), halley_nodes_unperturbed=natural,
           fluid_nodes=len(fl), max_rel_population_err=err, bound=3e-6)
    assert len(hal) >= 100, len(hal)
    assert err <= 3e-6, err
