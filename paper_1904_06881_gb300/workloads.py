"""Seeded synthetic inputs: solid masks, initial density/phase fields and
parameter sets shaped like the tests of arXiv:1904.06881.

This module holds geometry and random numbers only -- none of the method's
arithmetic.  Both the CUDA library and the CPU oracle are fed from it.

Physical parameters
-------------------
Free-energy parameters are Table 1, set 1 (lambda = 0.6, 1, 1; kappa = 0.01,
1, 1; chi = 5), which gives the liquid-liquid profile tanh(x/2), i.e. an
interface of width 4 (Sec. III, Eqs. liquidliquidalpha, profile).  The
Carnahan-Starling constants are the printed a = 0.037, b = 0.2, R = 1
(Sec. II.A).  The temperature is T = 0.8 T_c; the coexistence densities of
that EOS are the numbers RHO_L, RHO_G below (liquid/gas ratio 14.1).  The
step with the paper's pressure-form force and exact-difference forcing is
not stable from a tanh initial state at lower temperatures (higher ratios)
on these lattices, so every workload uses this temperature.

Fields are numpy arrays shaped (nz, ny, nx) with x fastest; masks are uint8
with 1 = solid.  Phases: C1 gas, C2 liquid with phi = +chi ("liquid 1"),
C3 liquid with phi = -chi ("liquid 2", the lubricant).
"""
import numpy as np

D2Q9, D3Q27 = 0, 1
WET_FORCE, WET_GEOM_EXTRAP, WET_GEOM_INTERP = 0, 1, 2

SET1 = dict(lam=(0.6, 1.0, 1.0), kappa=(0.01, 1.0, 1.0), chi=5.0)
CS_EOS = dict(a=0.037, b=0.2, R=1.0)
# Coexistence densities of the Carnahan-Starling EOS above at T = 0.8 T_c.
RHO_L = 6.143914427184784
RHO_G = 0.43446462473239633
KINETIC = dict(beta=0.5, tau_g=1.0, Gamma=1.0)   # tau = 1 for f and g, nu = 1/6


def base_params(**over):
    p = dict(SET1)
    p.update(CS_EOS)
    p.update(KINETIC)
    p.update(rho_l=RHO_L, rho_g=RHO_G, wetting=WET_FORCE, theta_deg=(90.0, 90.0, 90.0),
             kw_rho=0.0, kw_phi=0.0)
    p.update(over)
    return p


def phase_fields(C2, C3, rho_l=RHO_L, rho_g=RHO_G, chi=5.0):
    """(rho, phi) from liquid concentrations: C1 = 1 - C2 - C3 (Eq. definitionCsum),
    rho = rho_l + C1 (rho_g - rho_l) (Eq. definitionC1), phi = chi (C2 - C3)."""
    C1 = 1.0 - C2 - C3
    rho = rho_l + C1 * (rho_g - rho_l)
    phi = chi * (C2 - C3)
    return rho, phi


def _blob(dist, R, width):
    """Indicator of 'inside' with a tanh edge: 1 inside (dist < R), 0 outside."""
    return 0.5 * (1.0 - np.tanh((dist - R) / width))


def _noise(shape, seed, amp):
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, shape), rng.uniform(-amp, amp, shape)


def sessile_drop_2d(nx, ny, R, xc=None, yc=0.5, liquid=2, width=2.0, walls=("bottom", "top"),
                    noise=0.0, seed=0, rho_l=RHO_L, rho_g=RHO_G, chi=5.0):
    """2D drop of liquid C2 (liquid=2) or C3 (liquid=3) centred at (xc, yc) in
    gas; solid rows y=0 (bottom) and y=ny-1 (top).  The wall plane of the
    bottom wall lies at y = 0.5 (halfway bounce-back)."""
    xc = nx / 2.0 if xc is None else xc
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    inside = _blob(np.hypot(x - xc, y - yc), R, width)
    C2 = inside if liquid == 2 else np.zeros_like(inside)
    C3 = inside if liquid == 3 else np.zeros_like(inside)
    if noise:
        n2, n3 = _noise(C2.shape, seed, noise)
        C2, C3 = C2 + n2, C3 + n3
    rho, phi = phase_fields(C2, C3, rho_l, rho_g, chi)
    mask = np.zeros((ny, nx), np.uint8)
    if "bottom" in walls:
        mask[0, :] = 1
    if "top" in walls:
        mask[ny - 1, :] = 1
    return mask[None], rho[None], phi[None]


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
def c0_sessile_drop(seed=0):
    """D2Q9 64x64, periodic in x, solid rows at y=0 and y=63; liquid-1 cap of
    radius 16 on the bottom wall (centre (32, 0.5)) in gas; tanh edge of
    width 4; force wetting with kappa^w = 0 (theta = 90 deg); +-1e-3 uniform
    noise on C2 and C3; 1000 steps."""
    mask, rho, phi = sessile_drop_2d(64, 64, 16.0, xc=32.0, yc=0.5, noise=1e-3, seed=seed)
    return dict(name="c0_sessile_drop_d2q9_64x64", lattice=D2Q9, nx=64, ny=64, nz=1,
                params=base_params(wetting=WET_FORCE), mask=mask, rho=rho, phi=phi, steps=1000)


def c1_capillary(wetting=WET_GEOM_INTERP, nx=1024, ny=64, wall=12, x_in=256, x_out=960):
    """D2Q9 1024x64 capillary filling: solid slabs y<12 and y>=52 for
    x in [256, 960) leave a channel of height 40 between a liquid-1 reservoir
    (x < 256, full height) and a gas reservoir (x >= 960).  Geometric wetting
    with theta_21 = 30, theta_31 = 60, theta_23 = 120 deg.  50 000 steps."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    mask = np.zeros((ny, nx), np.uint8)
    slab = (x >= x_in) & (x < x_out) & ((y < wall) | (y >= ny - wall))
    mask[slab] = 1
    # liquid slab x in [0, x_in) on the periodic ring, tanh edges of width 4
    centre = 0.5 * (x_in - 1)
    xp = np.mod(x - centre + nx / 2, nx) - nx / 2
    C2 = _blob(np.abs(xp), 0.5 * x_in, 2.0)
    C3 = np.zeros_like(C2)
    rho, phi = phase_fields(C2, C3)
    params = base_params(wetting=wetting, theta_deg=(30.0, 60.0, 120.0))
    return dict(name="c1_capillary_d2q9_%dx%d" % (nx, ny), lattice=D2Q9, nx=nx, ny=ny, nz=1,
                params=params, mask=mask[None], rho=rho[None], phi=phi[None], steps=50000,
                channel=dict(x_in=x_in, x_out=x_out, wall=wall, H=ny - 2 * wall))


def c2_lubricated(nx=192, ny=192, nz=128, R=32.0, lub=6, gap=4, kw_rho=0.0):
    """D3Q27 192x192x128 lubricated substrate: solid planes z=0 and z=nz-1, a
    liquid-2 (C3) lubricant film z in [1, lub], a liquid-1 (C2) sphere of
    radius R whose bottom lies `gap` nodes above the film, gas elsewhere.
    Force wetting.  10 000 steps."""
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    zc = lub + gap + R
    C2 = _blob(np.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - zc) ** 2), R, 2.0)
    C3 = 0.5 * (1.0 - np.tanh((z - (lub + 0.5)) / 2.0)) * (1.0 - C2)
    rho, phi = phase_fields(C2, C3)
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[0] = 1
    mask[nz - 1] = 1
    params = base_params(wetting=WET_FORCE, theta_deg=(90.0, 20.0, 90.0), kw_rho=kw_rho)
    return dict(name="c2_lubricated_d3q27_%dx%dx%d" % (nx, ny, nz), lattice=D3Q27, nx=nx, ny=ny,
                nz=nz, params=params, mask=mask, rho=rho, phi=phi, steps=10000)


# Largest contact angle drawn for geometric wetting: a sessile drop of radius
# L/4 prescribed 129 deg (interpolation) drains the gas at its contact line to
# non-positive populations within 5000 steps for L >= 256 (within 250 steps in
# the FP64 oracle at L = 256); 125 deg runs 5000 steps at L = 64 to 512.
THETA_MAX = 125.0


def c3_sweep(seed=3, n=256, sizes=(64, 128, 256, 512)):
    """Batched D2Q9 contact-angle sweep: n draws of L from `sizes`, a sessile
    drop of radius L/4 on the bottom wall, theta_21 ~ U[30, THETA_MAX] deg; each
    draw runs with force and geometric-interpolation wetting (2n lattices).
    5000 steps."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(sizes, size=n)
    th = rng.uniform(30.0, THETA_MAX, size=n)
    out = []
    for k in range(n):
        L = int(Ls[k])
        for wet in (WET_FORCE, WET_GEOM_INTERP):
            out.append(dict(L=L, theta=float(th[k]), wetting=wet, seed=seed * 100003 + k))
    return out


def provisional_kw(theta_deg):
    """Force-method strength for a target angle from a linear fit of sessile
    drops run with the FP64 oracle (radius 16, 64x64: kappa^w = +0.2 gives
    76 deg, -0.2 gives 102 deg), clipped to |kappa^w| <= 0.25 (a radius-16
    drop started as a half disc leaves non-positive populations within 625
    steps at kappa^w = 0.3, and runs 5000 steps at 0.25).  Not a calibration:
    used only to give every force-wetting lattice of a sweep a strength of the
    right sign and size."""
    return float(np.clip((90.0 - theta_deg) / 65.0, -0.25, 0.25))


def c3_lattice(item):
    L = item["L"]
    mask, rho, phi = sessile_drop_2d(L, L, L / 4.0, xc=L / 2.0, yc=0.5)
    th = (item["theta"], item["theta"], 90.0)
    if item["wetting"] == WET_FORCE:
        params = base_params(wetting=WET_FORCE, kw_rho=provisional_kw(item["theta"]))
        return dict(name="c3_drop_%d" % L, lattice=D2Q9, nx=L, ny=L, nz=1, params=params,
                    mask=mask, rho=rho, phi=phi, steps=5000)
    params = base_params(wetting=item["wetting"], theta_deg=th)
    return dict(name="c3_drop_%d" % L, lattice=D2Q9, nx=L, ny=L, nz=1, params=params,
                mask=mask, rho=rho, phi=phi, steps=5000)


def big_periodic_drop_2d(n=4096, R=None):
    """Large D2Q9 periodic lattice with one liquid-1 drop (no walls)."""
    R = n / 4.0 if R is None else R
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    C2 = _blob(np.hypot(x - n / 2, y - n / 2), R, 2.0)
    rho, phi = phase_fields(C2, np.zeros_like(C2))
    return dict(name="big_d2q9_%d" % n, lattice=D2Q9, nx=n, ny=n, nz=1, params=base_params(),
                mask=np.zeros((1, n, n), np.uint8), rho=rho[None], phi=phi[None], steps=1000)


def big_periodic_drop_3d(n=256, R=None):
    """Large D3Q27 periodic lattice with one liquid-1 drop (no walls)."""
    R = n / 4.0 if R is None else R
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float32)
    d = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2).astype(np.float64)
    del x, y, z
    C2 = _blob(d, R, 2.0)
    rho, phi = phase_fields(C2, np.zeros_like(C2))
    return dict(name="big_d3q27_%d" % n, lattice=D3Q27, nx=n, ny=n, nz=n, params=base_params(),
                mask=np.zeros((n, n, n), np.uint8), rho=rho, phi=phi, steps=1000)


def bubble_2d(pair, L, R, **params):
    """Bubble test of Sec. III for one interface pair in a periodic L x L box:
    a disc of radius R (tanh edge of width 4) at the box centre.  pair "12":
    C2 (liquid 1) in C1 (gas); "13": C3 (liquid 2) in C1; "23": C3 in C2.
    params override base_params (lam, kappa, ...)."""
    y, x = np.mgrid[0:L, 0:L].astype(np.float64)
    inside = _blob(np.hypot(x - L / 2.0, y - L / 2.0), R, 2.0)
    zero = np.zeros_like(inside)
    C2, C3 = {"12": (inside, zero), "13": (zero, inside), "23": (1.0 - inside, inside)}[pair]
    p = base_params(**params)
    rho, phi = phase_fields(C2, C3, rho_l=p["rho_l"], rho_g=p["rho_g"], chi=p["chi"])
    return dict(name="bubble_%s_%d" % (pair, L), lattice=D2Q9, nx=L, ny=L, nz=1, params=p,
                mask=np.zeros((1, L, L), np.uint8), rho=rho[None], phi=phi[None])


def bislug_2d(H=19, L1=60, L2=60, gas=120, theta=60.0, x0=None, wetting=WET_GEOM_INTERP):
    """Self-propelled bi-slug of Sec. VI: a periodic channel of height H
    (solid rows y = 0 and y = H + 1, wall planes half a node inside) holding
    a slug of C2 (length L1) followed along +x by a slug of C3 (length L2),
    gas elsewhere (gas columns of total length `gas`); tanh edges of width 4.
    Geometric wetting with theta_21 = theta_31 = theta_23 = theta."""
    nx, ny = L1 + L2 + gas, H + 2
    x0 = gas / 2.0 if x0 is None else x0
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    left = 0.5 * (1.0 + np.tanh((x - x0) / 2.0))
    mid = 0.5 * (1.0 + np.tanh((x - x0 - L1) / 2.0))
    right = 0.5 * (1.0 + np.tanh((x - x0 - L1 - L2) / 2.0))
    C2, C3 = left - mid, mid - right
    rho, phi = phase_fields(C2, C3)
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = 1
    mask[ny - 1, :] = 1
    params = base_params(wetting=wetting, theta_deg=(theta, theta, theta))
    return dict(name="bislug_%dx%d" % (nx, ny), lattice=D2Q9, nx=nx, ny=ny, nz=1, params=params,
                mask=mask[None], rho=rho[None], phi=phi[None], steps=20000,
                slug=dict(H=H, L1=L1, L2=L2, gas=gas, x0=x0))


def lens_2d(L, R=None, ratio=None, theta=None, seed=0):
    """2D liquid lens (Sec. III, Neumann angles): a liquid-1 (C2) disc of
    radius R centred on the flat interface between a liquid-2 (C3) layer
    (lower half) and gas (upper half) of a periodic L x L box."""
    R = L / 6.0 if R is None else R
    y, x = np.mgrid[0:L, 0:L].astype(np.float64)
    disc = _blob(np.hypot(x - L / 2.0, y - L / 2.0), R, 2.0)
    below = 0.5 * (1.0 - np.tanh((y - L / 2.0) / 2.0))
    C2 = disc
    C3 = below * (1.0 - disc)
    rho_l, rho_g = RHO_L, (RHO_L / ratio if ratio else RHO_G)
    rho, phi = phase_fields(C2, C3, rho_l, rho_g)
    p = base_params(rho_l=rho_l, rho_g=rho_g)
    return dict(name="lens_%d" % L, lattice=D2Q9, nx=L, ny=L, nz=1, params=p,
                mask=np.zeros((1, L, L), np.uint8), rho=rho[None], phi=phi[None])


def drop_train_2d(nx, ny=64, ndrop=4, ratio=None, theta=60.0):
    """A train of `ndrop` liquid-1 drops (radius ny/5) alternating with
    liquid-2 drops, resting on the bottom wall of a periodic channel (solid
    rows y = 0 and y = ny - 1); geometric interpolation at `theta`."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    R = ny / 5.0
    C2 = np.zeros_like(x)
    C3 = np.zeros_like(x)
    for k in range(ndrop):
        xc = (k + 0.5) * nx / ndrop
        blob = _blob(np.hypot(x - xc, y - 0.5), R, 2.0)
        if k % 2 == 0:
            C2 = np.maximum(C2, blob)
        else:
            C3 = np.maximum(C3, blob)
    rho_l, rho_g = RHO_L, (RHO_L / ratio if ratio else RHO_G)
    rho, phi = phase_fields(C2, C3, rho_l, rho_g)
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = 1
    mask[ny - 1, :] = 1
    p = base_params(wetting=WET_GEOM_INTERP, theta_deg=(theta, theta, 90.0), rho_l=rho_l, rho_g=rho_g)
    return dict(name="drop_train_%dx%d" % (nx, ny), lattice=D2Q9, nx=nx, ny=ny, nz=1, params=p,
                mask=mask[None], rho=rho[None], phi=phi[None])


def _liquid_liquid(wl):
    """The same geometry with the gas replaced by liquid 2 (C3): a
    liquid-liquid request (density ratio 1)."""
    rho_l = wl["params"]["rho_l"]
    C1 = (wl["rho"] - rho_l) / (wl["params"]["rho_g"] - rho_l)
    C2 = 0.5 * (1.0 + wl["phi"] / wl["params"]["chi"] - C1)
    C3 = 1.0 - C2
    rho, phi = phase_fields(C2, C3, rho_l, wl["params"]["rho_g"], wl["params"]["chi"])
    out = dict(wl)
    out["rho"], out["phi"] = rho, phi
    out["name"] = wl["name"] + "_ll"
    return out


def c4_requests(seed=4, n=256, rate=20.0, sizes_2d=(64, 128, 256, 512, 1024), sizes_3d=(96, 128, 160, 192)):
    """Served mix: Poisson arrivals (mean `rate` per second) of n requests:
    sessile drops (L^2, L in sizes_2d), capillary channels (nx x 64,
    nx in 256-1024), lubricated substrates (D3Q27 n^3, n in sizes_3d), liquid
    lenses and drop trains (2D); uniform random angles in [30, THETA_MAX]
    deg; the liquid-gas density ratio log-uniform between 4 and the
    workloads' 14.1 (the gas density rho_l / ratio), or a liquid-liquid
    request (ratio 1: the gas replaced by liquid 2) in one request of eight.
    (Below a ratio of about 3.5 the density jump is so small that the lambda_2,
    lambda_3 wells, whose weight in mu_rho grows as 1/drho^2, give the liquid
    a sound speed above the lattice's, and the step diverges.)
    Steps: 2D 1000-5000, 3D 500-2000.  Returns a list of (arrival_s,
    workload dict, steps)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    ratio_max = RHO_L / RHO_G
    out = []
    for k in range(n):
        kind = rng.choice(["drop", "channel", "lubricated", "lens", "train"], p=[0.35, 0.2, 0.1, 0.15, 0.2])
        th = float(rng.uniform(30.0, THETA_MAX))
        ll = rng.uniform() < 0.125
        ratio = float(np.exp(rng.uniform(np.log(4.0), np.log(ratio_max))))
        if ll:
            ratio = ratio_max        # no gas: the EOS of the workloads
        if kind == "drop":
            L = int(rng.choice(sizes_2d))
            mask, rho, phi = sessile_drop_2d(L, L, L / 4.0, xc=L / 2.0, yc=0.5, rho_g=RHO_L / ratio)
            wl = dict(name="drop_%d" % L, lattice=D2Q9, nx=L, ny=L, nz=1, mask=mask, rho=rho, phi=phi,
                      params=base_params(wetting=WET_GEOM_INTERP, theta_deg=(th, th, 90.0), rho_g=RHO_L / ratio))
            steps = int(rng.integers(1000, 5001))
        elif kind == "channel":
            nx = int(rng.choice([256, 512, 1024]))
            wl = c1_capillary(nx=nx, ny=64, x_in=nx // 4, x_out=nx - nx // 16)
            wl["params"] = base_params(wetting=WET_GEOM_INTERP, theta_deg=(th, 60.0, 120.0))
            steps = int(rng.integers(1000, 5001))
        elif kind == "lens":
            wl = lens_2d(int(rng.choice(sizes_2d[:4])), ratio=ratio)
            steps = int(rng.integers(1000, 5001))
        elif kind == "train":
            wl = drop_train_2d(int(rng.choice([256, 512, 1024])), 64, ndrop=int(rng.integers(2, 7)), ratio=ratio,
                               theta=th)
            steps = int(rng.integers(1000, 5001))
        else:
            n3 = int(rng.choice(sizes_3d))
            wl = c2_lubricated(nx=n3, ny=n3, nz=n3, R=n3 / 6.0, lub=3, gap=2, kw_rho=0.02)
            steps = int(rng.integers(500, 2001))
            ll = False
        if ll:
            wl = _liquid_liquid(wl)
        out.append((float(t[k]), wl, steps))
    return out
