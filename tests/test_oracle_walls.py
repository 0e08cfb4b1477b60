"""Pins of the oracle's solid boundaries and wetting schemes (Sec. IV).

- halfway bounce-back conserves mass exactly; a uniform fluid at rest next to
  flat walls feels no force (wall rule for grad P);
- geometric extrapolation (Eqs. geomamgle, geomding) and interpolation
  (Eqs. interp2D, interp3D) both give c_ghost = c_1 + cot(theta)|grad_par c|
  on a field that is linear along the wall, in 2D and in 3D;
- the interface-identification rules of Sec. IV.B pick theta_21, theta_31 or
  theta_23;
- the force method's wall force (Eq. forceBC) on a uniform fluid: -n/6 times
  the phase's strength, on the second fluid layer only;
- contact angles: a neutral wall holds 90 deg, geometric angles below and
  above 90 deg spread and bead the drop, the force strength kappa^w > 0
  spreads it.
"""
import numpy as np
import pytest

import oracle
from paper_1904_06881_gb300 import workloads as W

from test_oracle_thermo import _mk


@pytest.mark.parametrize("wet,th", [(W.WET_FORCE, (90, 90, 90)), (W.WET_GEOM_EXTRAP, (45, 60, 120)),
                                    (W.WET_GEOM_INTERP, (60, 60, 120))])
def test_mass_conserved_with_walls(wet, th):
    c = W.c0_sessile_drop()
    o = _mk(64, 64, wetting=wet, theta_deg=th, kw_rho=0.01 if wet == W.WET_FORCE else 0.0)
    o.set_solid(c["mask"])
    o.init_fields(c["rho"], c["phi"])
    d0 = o.diagnostics()
    o.step(300)
    d1 = o.diagnostics()
    for k in ("mass_rho", "mass_phi", "C1", "C2", "C3"):
        assert abs(d1[k] - d0[k]) <= 1e-12 * max(abs(d0["mass_rho"]), 1.0), k


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
@pytest.mark.parametrize("wet", [W.WET_FORCE, W.WET_GEOM_EXTRAP, W.WET_GEOM_INTERP])
def test_uniform_fluid_at_rest_between_walls(lat, wet):
    if lat == oracle.D2Q9:
        shape, o = (1, 10, 12), _mk(12, 10, wetting=wet, theta_deg=(60, 70, 120))
    else:
        shape, o = (8, 6, 6), _mk(6, 6, 8, lat=lat, wetting=wet, theta_deg=(60, 70, 120))
    mask = np.zeros(shape, np.uint8)
    if lat == oracle.D2Q9:
        mask[0, 0, :] = mask[0, -1, :] = 1
    else:
        mask[0] = mask[-1] = 1
    o.set_solid(mask)
    rl = o.derived["rho_l"]
    o.init_fields(np.full(shape, rl), np.full(shape, 5.0))
    for k in ("Fx", "Fy", "Fz"):
        assert np.abs(o.aux(k)).max() < 1e-13
    o.step(100)
    f = o.fields()
    fl = mask == 0
    assert np.abs(f["rho"][fl] - rl).max() < 1e-12 and np.abs(f["u"]).max() < 1e-14


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
@pytest.mark.parametrize("phase", ["liquid2", "liquid3", "gas"])
def test_force_wetting_closed_form(lat, phase):
    """Eq. forceBC on flat walls with a uniform fluid at rest: the bulk force
    vanishes (wall rule), and on the second fluid layer alone F_s =
    rho_rel (kappa_rho^w + phi_rel kappa_phi^w) sum_i w_i s(x + c_i) c_i, where
    the lattice sum over the first-layer neighbours is -n/6 in D2Q9 and in
    D3Q27 (n the wall normal into the fluid).  Liquid 2 (phi = chi) takes
    kappa_rho^w + kappa_phi^w, liquid 3 (phi = -chi) kappa_rho^w -
    kappa_phi^w, the gas (rho_rel = 0) none."""
    kr, kp = 0.03, 0.07
    if lat == oracle.D2Q9:
        shape, o = (1, 10, 6), _mk(6, 10, wetting=W.WET_FORCE, kw_rho=kr, kw_phi=kp)
    else:
        shape, o = (8, 5, 5), _mk(5, 5, 8, lat=lat, wetting=W.WET_FORCE, kw_rho=kr, kw_phi=kp)
    mask = np.zeros(shape, np.uint8)
    if lat == oracle.D2Q9:
        mask[0, 0, :] = mask[0, -1, :] = 1
    else:
        mask[0] = mask[-1] = 1
    o.set_solid(mask)
    d = o.derived
    rho, phi, amp = {"liquid2": (d["rho_l"], 5.0, kr + kp), "liquid3": (d["rho_l"], -5.0, kr - kp),
                     "gas": (d["rho_g"], 0.0, 0.0)}[phase]
    o.init_fields(np.full(shape, rho), np.full(shape, phi))
    axis = "Fy" if lat == oracle.D2Q9 else "Fz"
    Fn = o.aux(axis)
    Fn = Fn[0] if lat == oracle.D2Q9 else Fn          # wall-normal axis first
    layers = Fn.reshape(Fn.shape[0], -1)
    want = np.zeros(layers.shape[0])
    want[2], want[-3] = -amp / 6.0, amp / 6.0        # second layer above the lower and below the upper wall
    fl = slice(1, layers.shape[0] - 1)
    assert np.abs(layers[fl] - want[fl, None]).max() < 1e-13, (phase, layers[:, 0])
    for k in ("Fx", "Fy", "Fz"):
        if k != axis:
            assert np.abs(o.aux(k)[mask == 0]).max() < 1e-13


def _ghost_case_2d(wet, theta, slope, rho_mid=None, phi_of=None, nx=40):
    o = _mk(nx, 8, wetting=wet, theta_deg=theta)
    d = o.derived
    rl, rg = d["rho_l"], d["rho_g"]
    mask = np.zeros((1, 8, nx), np.uint8)
    mask[0, 0, :] = 1
    o.set_solid(mask)
    x = np.arange(nx, dtype=float)
    mid = 0.5 * (rl + rg) if rho_mid is None else rho_mid
    rho = np.tile(mid + slope * (x - nx / 2), (1, 8, 1))
    phi = 5.0 * (rho - rg) / (rl - rg) if phi_of is None else phi_of(rho, x)
    o.init_fields(rho, np.broadcast_to(phi, rho.shape).copy())
    return o, rho, phi


@pytest.mark.parametrize("wet", [W.WET_GEOM_EXTRAP, W.WET_GEOM_INTERP])
@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0, 150.0])
@pytest.mark.parametrize("slope", [0.05, -0.05])
def test_ghost_linear_field_2d(wet, theta, slope):
    """Along a wall with grad c parallel to it, both geometric schemes give the
    ghost c_1 + cot(theta) |grad_par c| (theta measured in the phase where c is
    high): extrapolation by Eq. geomding, interpolation exactly on linear data."""
    o, rho, phi = _ghost_case_2d(wet, (theta, 70.0, 110.0), slope)
    g = o.aux("rho_ghost")[0, 0]
    xs = np.arange(8, 32)
    expect = rho[0, 1, xs] + abs(slope) / np.tan(np.radians(theta))
    assert np.abs(g[xs] - expect).max() < 1e-12


def test_interface_identification_rules():
    th = (50.0, 70.0, 115.0)
    cot = 1 / np.tan(np.radians(th))
    xs = np.arange(8, 32)
    # 1-2: rho and phi rise together
    o, rho, phi = _ghost_case_2d(W.WET_GEOM_EXTRAP, th, 0.05)
    assert np.allclose(o.aux("rho_ghost")[0, 0, xs] - rho[0, 1, xs], 0.05 * cot[0], atol=1e-12)
    # 1-3: phi falls where rho rises
    o, rho, phi = _ghost_case_2d(W.WET_GEOM_EXTRAP, th, 0.05,
                                 phi_of=lambda r, x: -5.0 * (r - 0.43446462473239633) / (6.143914427184784 - 0.43446462473239633))
    assert np.allclose(o.aux("rho_ghost")[0, 0, xs] - rho[0, 1, xs], 0.05 * cot[1], atol=1e-12)
    # 2-3: rho flat in the liquid, phi varies; c = phi and theta_23
    rl = o.derived["rho_l"]
    o, rho, phi = _ghost_case_2d(W.WET_GEOM_EXTRAP, th, 0.0, rho_mid=rl,
                                 phi_of=lambda r, x: 0.1 * (x - 20.0))
    assert np.allclose(o.aux("phi_ghost")[0, 0, xs] - 0.1 * (xs - 20.0), 0.1 * cot[2], atol=1e-12)
    # bulk liquid 3 overrides the gradient sign: rho > rho_l/2 and phi < -0.95 chi -> 1-3
    o, rho, phi = _ghost_case_2d(W.WET_GEOM_EXTRAP, th, 1e-3, rho_mid=rl - 0.05,
                                 phi_of=lambda r, x: -4.9 + 1e-3 * (x - 20.0))
    assert np.allclose(o.aux("rho_ghost")[0, 0, xs] - rho[0, 1, xs], 1e-3 * cot[1], atol=1e-12)


@pytest.mark.parametrize("wet", [W.WET_GEOM_EXTRAP, W.WET_GEOM_INTERP])
@pytest.mark.parametrize("theta", [35.0, 75.0, 130.0])
@pytest.mark.parametrize("direction", [(1.0, 0.0), (0.6, 0.8), (-0.28, 0.96), (-0.8, -0.6)])
def test_ghost_linear_field_3d(wet, theta, direction):
    """3D: |grad_par c| is the in-plane norm; the plane through three of the four
    surrounding nodes (Eq. interp3D) reproduces a linear field."""
    n, nz = 24, 6
    o = _mk(n, n, nz, lat=oracle.D3Q27, wetting=wet, theta_deg=(theta, 70.0, 110.0))
    d = o.derived
    rl, rg = d["rho_l"], d["rho_g"]
    mask = np.zeros((nz, n, n), np.uint8)
    mask[0] = 1
    o.set_solid(mask)
    z, y, x = np.mgrid[0:nz, 0:n, 0:n].astype(float)
    s = 0.04
    rho = 0.5 * (rl + rg) + s * (direction[0] * (x - n / 2) + direction[1] * (y - n / 2))
    phi = 5.0 * (rho - rg) / (rl - rg)
    o.init_fields(rho, phi)
    g = o.aux("rho_ghost")[0]
    sl = (slice(6, 18), slice(6, 18))
    expect = rho[1][sl] + s / np.tan(np.radians(theta))
    assert np.abs(g[sl] - expect).max() < 1e-12


@pytest.mark.parametrize("corner", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_interp3d_support_drops_the_nearest_corner(corner):
    """Eq. interp3D takes the plane through the three of the four corners of
    the cell holding (l_x, l_y) that lie furthest from (i, j).  At cot(theta) =
    2.5 along the unit direction (0.985, 0.171), (l_x, l_y) = (2.46, 0.43) lies
    in the cell [2, 3] x [0, 1], whose corner nearest (i, j) is (2, 0).  A spike
    on the first fluid layer at that corner leaves the ghost at (i, j) on the
    linear field's value; a spike at a kept corner moves it by its barycentric
    weight in the triangle (3, 0), (2, 1), (3, 1).  The spikes sit two or more
    nodes from (i, j), outside the in-plane gradient's stencil."""
    n, nz, s, spike = 24, 6, 0.04, 0.3
    theta = np.degrees(np.arctan(1.0 / 2.5))
    o = _mk(n, n, nz, lat=oracle.D3Q27, wetting=W.WET_GEOM_INTERP, theta_deg=(theta, 70.0, 110.0))
    d = o.derived
    rl, rg = d["rho_l"], d["rho_g"]
    mask = np.zeros((nz, n, n), np.uint8)
    mask[0] = mask[-1] = 1            # the ghost at z = 0 then faces fluid on one side only
    o.set_solid(mask)
    u = np.array([0.92, 0.16]) / np.hypot(0.92, 0.16)
    z, y, x = np.mgrid[0:nz, 0:n, 0:n].astype(float)
    rho = 0.5 * (rl + rg) + s * (u[0] * (x - n / 2) + u[1] * (y - n / 2))
    i, j = 8, 10
    rho[1, j + corner[1], i + corner[0]] += spike
    phi = 5.0 * (rho - rg) / (rl - rg)
    o.init_fields(rho, phi)
    g = o.aux("rho_ghost")[0, j, i]
    linear = 0.5 * (rl + rg) + s * (u[0] * (i - n / 2) + u[1] * (j - n / 2)) + s * 2.5
    lx, ly = 2.5 * u
    b = 3.0 - lx                      # weight of (2, 1): x = 3 a + 2 b + 3 c with a + b + c = 1
    c = ly - b                        # weight of (3, 1): y = b + c
    weight = {(2, 0): 0.0, (3, 0): 1.0 - b - c, (2, 1): b, (3, 1): c}[corner]
    assert abs(g - (linear + weight * spike)) < 1e-12, (corner, g - linear, weight * spike)


@pytest.mark.parametrize("wet", [W.WET_GEOM_EXTRAP, W.WET_GEOM_INTERP])
def test_corner_ghosts_keep_the_diagonal_mirror_symmetry(wet):
    """A solid square block in a periodic box, a drop centred on the
    diagonal: the problem is symmetric under x <-> y, which maps a corner
    ghost's two fluid-facing axes onto each other.  Averaging the single-axis
    ghost values over the fluid-facing axes keeps the symmetry, at the block's
    off-diagonal corners too (taking either axis alone breaks it there), and
    the step keeps it: the fields stay mirror-symmetric to rounding over 200
    steps."""
    n = 32
    o = _mk(n, n, wetting=wet, theta_deg=(60.0, 70.0, 110.0))
    mask = np.zeros((1, n, n), np.uint8)
    mask[0, 12:18, 12:18] = 1
    o.set_solid(mask)
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    C2 = 0.5 * (1 - np.tanh((np.hypot(xx - 10.0, yy - 10.0) - 6.0) / 2.0))
    rho, phi = W.phase_fields(C2, np.zeros_like(C2))
    rho, phi = rho.reshape(1, n, n), phi.reshape(1, n, n)
    o.init_fields(rho, phi)
    g = o.aux("rho_ghost")[0]
    ring = mask[0].astype(bool)
    assert np.abs(g - g.T)[ring].max() < 1e-13
    # the two single-axis values differ at the off-diagonal corners, so the rule is exercised there
    assert abs(g[12, 17] - rho[0, 12, 18]) > 1e-4 and abs(g[12, 17] - rho[0, 11, 17]) > 1e-4
    o.step(200)
    r = o.fields()["rho"][0]
    assert np.abs(r - r.T).max() < 1e-10


def _contact_angle(rho, rl, rg, wall_plane=0.5):
    """Circular-cap angle from the base half-width a (at one node above the
    wall) and the apex height h of the rho = (rho_l + rho_g)/2 contour:
    tan(theta/2) = h/a."""
    half = 0.5 * (rl + rg)
    col = rho[:, rho.shape[1] // 2]
    ys = np.where(col > half)[0]
    top = ys.max()
    h = top + (col[top] - half) / (col[top] - col[top + 1]) - wall_plane
    row = rho[1]
    xs = np.where(row > half)[0]
    left, right = xs.min(), xs.max()
    xl = left - (row[left] - half) / (row[left] - row[left - 1])
    xr = right + (row[right] - half) / (row[right] - row[right + 1])
    a = 0.5 * (xr - xl)
    # account for the first row lying half a node above the wall plane
    R_ = (a * a + (h) ** 2) / (2 * h)
    yc = h - R_
    a0 = np.sqrt(max(R_ ** 2 - yc ** 2, 0.0))
    return np.degrees(2 * np.arctan2(h, a0))


def _sessile(wet, theta, kw=0.0, n=64, steps=6000):
    o = _mk(n, n, wetting=wet, theta_deg=(theta, theta, 90.0), kw_rho=kw)
    mask, rho, phi = W.sessile_drop_2d(n, n, 16.0, xc=n / 2, yc=0.5)
    o.set_solid(mask)
    o.init_fields(rho, phi)
    o.step(steps)
    d = o.derived
    return _contact_angle(o.fields()["rho"][0], d["rho_l"], d["rho_g"])


def _circle_fit_angle(rho, rl, rg, skip=3):
    """Contact angle of a least-squares circle through the rho = (rho_l +
    rho_g)/2 contour (linear interpolation along rows and columns, rows 1 +
    skip and above), against the wall plane half a node above the solid row."""
    half = 0.5 * (rl + rg)
    ny, nx = rho.shape
    pts = []
    for y in range(1 + skip, ny - 2):
        for x in range(nx):
            a, b = rho[y, x], rho[y + 1, x]
            if (a - half) * (b - half) < 0:
                pts.append((x, y + (a - half) / (a - b)))
            if x + 1 < nx:
                c = rho[y, x + 1]
                if (a - half) * (c - half) < 0:
                    pts.append((x + (a - half) / (a - c), y))
    p = np.array(pts)
    A = np.column_stack([p[:, 0], p[:, 1], np.ones(len(p))])
    k = np.linalg.lstsq(A, -(p[:, 0] ** 2 + p[:, 1] ** 2), rcond=None)[0]
    xc, yc = -k[0] / 2, -k[1] / 2
    R_ = np.sqrt(xc * xc + yc * yc - k[2])
    return np.degrees(np.arccos((0.5 - yc) / R_))


@pytest.mark.slow
@pytest.mark.parametrize("wet", [W.WET_FORCE, W.WET_GEOM_EXTRAP, W.WET_GEOM_INTERP])
def test_neutral_wall_gives_ninety_degrees(wet):
    """A neutral wall (force method with kappa^w = 0; geometric schemes at
    theta = 90 deg, whose ghost layer then mirrors the first fluid layer)
    leaves the drop at 90 deg: 88.6 deg measured for every scheme at radius 16
    (88.9 at radius 24: the gap closes with resolution)."""
    n = 64
    o = _mk(n, n, wetting=wet, theta_deg=(90.0, 90.0, 90.0))
    mask, rho, phi = W.sessile_drop_2d(n, n, 16.0, xc=n / 2, yc=0.5)
    o.set_solid(mask)
    o.init_fields(rho, phi)
    o.step(6000)
    d = o.derived
    assert abs(_circle_fit_angle(o.fields()["rho"][0], d["rho_l"], d["rho_g"]) - 90.0) < 2.0


@pytest.mark.slow
def test_geometric_angle_sign_and_value():
    a45 = _sessile(W.WET_GEOM_INTERP, 60.0)
    a135 = _sessile(W.WET_GEOM_INTERP, 120.0)
    assert a45 < 80.0 and a135 > 100.0
    # measured 63.0 and 126.5 deg at this size (radius 16, ratio 14)
    assert abs(a45 - 60.0) < 5.0 and abs(a135 - 120.0) < 8.0


@pytest.mark.slow
def test_force_strength_sign():
    # measured 76.0 and 102.3 deg for kappa^w = +-0.2 (radius 16, ratio 14)
    assert _sessile(W.WET_FORCE, 90.0, kw=0.2, steps=4000) < 85.0
    assert _sessile(W.WET_FORCE, 90.0, kw=-0.2, steps=4000) > 95.0


@pytest.mark.slow
def test_force_method_satisfies_girifalco_good():
    """Sec. IV.A: on the force method's ideal wall the three angles obey the
    Girifalco-Good relation (Eq. GirifalcoGood).  Young's law at each contact
    line, with theta_23 measured in C2 as the stated convention has it, makes
    the consistent combination gamma_12 cos theta_21 - gamma_13 cos theta_31 -
    gamma_23 cos theta_23 = 0 (the printed + sign on the gamma_23 term
    corresponds to theta_23 measured in C3).  Three sessile drops (C2 in gas,
    C3 in gas, C2 in C3; radius 16, 6000 steps) with kappa_rho^w = 0.05,
    kappa_phi^w = -0.1, and the three Laplace tensions (bubbles of radius 16,
    4000 steps): |Delta gamma| below 3 % of gamma_max (measured 1.9 %), where
    the printed-sign combination is 25 % of it."""
    import oracle.tension as OT

    n, R, kr, kp = 64, 16.0, 0.05, -0.1

    def drop(kind):
        y, x = np.mgrid[0:n, 0:n].astype(float)
        inside = 0.5 * (1 - np.tanh((np.hypot(x - n / 2, y - 0.5) - R) / 2.0))
        z = np.zeros_like(inside)
        C2, C3 = {"21": (inside, z), "31": (z, inside), "23": (inside, 1 - inside)}[kind]
        rho, phi = W.phase_fields(C2, C3)
        o = _mk(n, n, wetting=W.WET_FORCE, kw_rho=kr, kw_phi=kp)
        mask = np.zeros((n, n), np.uint8)
        mask[0] = 1
        mask[n - 1] = 1
        o.set_solid(mask)
        o.init_fields(rho, phi)
        o.step(6000)
        f, d = o.fields(), o.derived
        if kind == "23":
            return _circle_fit_angle(f["phi"][0], 5.0, -5.0)     # the level C2 = C3
        return _circle_fit_angle(f["rho"][0], d["rho_l"], d["rho_g"])

    th = {k: np.radians(drop(k)) for k in ("21", "31", "23")}
    g = {pair: OT.laplace(OT.bubble(pair, 64, 16.0, 4000), pair) for pair in ("12", "13", "23")}
    young = g["12"] * np.cos(th["21"]) - g["13"] * np.cos(th["31"]) - g["23"] * np.cos(th["23"])
    printed = g["23"] * np.cos(th["23"]) - g["13"] * np.cos(th["31"]) + g["12"] * np.cos(th["21"])
    gmax = max(g.values())
    assert abs(young) < 0.03 * gmax, (young, printed, th, g)
    assert abs(printed) > 0.1 * gmax
