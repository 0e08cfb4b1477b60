"""Shared helpers of the GPU parity tests: the same seeded workload fed to the
CUDA library (through the C ABI) and to the FP64 oracle; the achieved errors
of every parity case are recorded (printed at the end of the session and
written as JSON to the path in TLB_PARITY_RECORD, when set)."""
import numpy as np

import oracle

RECORDS = []


def record(case, **values):
    """Keep one parity case's achieved figures for the session summary."""
    out = {"case": case}
    for k, v in values.items():
        if isinstance(v, dict):
            v = {kk: float(vv) for kk, vv in v.items()}
        elif isinstance(v, (np.floating, float, int, np.integer)):
            v = float(v)
        out[k] = v
    RECORDS.append(out)


def oracle_from_workload(wl, **over):
    return oracle.from_workload(wl, **over)


def gpu_from_workload(wl, **over):
    from paper_1904_06881_gb300 import tlb

    return tlb.lattice_from_workload(wl, **over)


def normwise(fg, fo, derived, chi=5.0, mask=None):
    """Normwise field errors (densities over rho_l - rho_g, phi over chi,
    concentrations absolute) on fluid nodes."""
    fl = np.ones(fg["rho"].shape, bool) if mask is None else (mask == 0)
    drho = derived["rho_l"] - derived["rho_g"]
    return dict(rho=np.abs(fg["rho"] - fo["rho"])[fl].max() / drho,
                phi=np.abs(fg["phi"] - fo["phi"])[fl].max() / chi,
                C=max(np.abs(fg["C"][k] - fo["C"][k])[fl].max() for k in range(3)))


def pointwise_rho(fg, fo, mask=None):
    """Largest pointwise relative density error |rho_gpu - rho_ora| / rho_ora
    on fluid nodes, gas nodes included (reported beside the normwise bar)."""
    fl = np.ones(fg["rho"].shape, bool) if mask is None else (mask == 0)
    return float((np.abs(fg["rho"][fl] - fo["rho"][fl]) / np.abs(fo["rho"][fl])).max())


def circle_fit_angle(rho, rl, rg, skip=3, wall_row=0):
    """Contact angle (deg) of a 2D sessile drop on the solid row `wall_row`:
    a least-squares circle through the rho = (rho_l + rho_g)/2 contour
    (linear interpolation along rows and columns, from `skip` rows above the
    first fluid row), measured against the wall plane half a node above the
    solid row."""
    half = 0.5 * (rl + rg)
    ny, nx = rho.shape
    pts = []
    for y in range(wall_row + 1 + skip, ny - 2):
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
    return float(np.degrees(np.arccos((wall_row + 0.5 - yc) / R_)))


def meniscus_x(rho, rl, rg, x_in, x_out, y0, y1):
    """Mean position along x of the rho = (rho_l + rho_g)/2 crossing inside a
    channel (rows y0..y1-1, searched from x_in towards x_out)."""
    half = 0.5 * (rl + rg)
    xs = []
    for y in range(y0, y1):
        row = rho[y]
        below = np.where(row[x_in:x_out] < half)[0]
        if len(below) == 0:
            xs.append(float(x_out))
            continue
        i = x_in + below[0]
        xs.append(i - 1 + (row[i - 1] - half) / (row[i - 1] - row[i]))
    return float(np.mean(xs))


def match_directions(lattice):
    """Permutation p with gpu_direction[p[i]] == oracle_direction[i]."""
    from paper_1904_06881_gb300 import tlb

    cg, _ = tlb.tlb_lattice_directions(lattice)
    co, _ = oracle.lattice(lattice)
    return np.array([int(np.where((cg == co[i]).all(1))[0][0]) for i in range(len(co))])


def meniscus_fit(rho, half, wall, x_in, x_out):
    """Meniscus of a liquid column filling a 2D channel (fluid rows wall ..
    ny - wall - 1, liquid entering at x_in): the rho = half crossing of every
    row (first one from x_in, linear interpolation), the centre row's crossing
    relative to x_in, and cos(theta) of the circle through the crossings (a
    circular meniscus spanning the channel meets the walls at
    cos(theta) = (H/2)/R).  None when a row has no crossing."""
    ny = rho.shape[0]
    ys = np.arange(wall, ny - wall)
    fx = []
    for y in ys:
        row = rho[y]
        below = np.where(row[x_in:x_out] < half)[0]
        if len(below) == 0:
            return None
        i = x_in + below[0]
        fx.append(i - 1 + (row[i - 1] - half) / (row[i - 1] - row[i]))
    fx, yy = np.array(fx), ys.astype(float)
    A = np.vstack([fx, yy, np.ones_like(fx)]).T
    Dc, Ec, Fc = np.linalg.lstsq(A, -(fx ** 2 + yy ** 2), rcond=None)[0]
    R = np.sqrt(Dc ** 2 / 4 + Ec ** 2 / 4 - Fc)
    return float(fx[len(fx) // 2] - x_in), float(min(1.0, 0.5 * len(ys) / R))


def washburn_fit(ts, xs, window=0.1):
    """Fit x = K sqrt(t - t0) over the last `window` of the samples (least
    squares on x^2 = K^2 (t - t0)); returns (K, t0)."""
    ts, xs = np.asarray(ts, float), np.asarray(xs, float)
    w = slice(int(round((1.0 - window) * len(ts))), len(ts))
    A = np.vstack([ts[w], np.ones(len(ts[w]))]).T
    K2, c = np.linalg.lstsq(A, xs[w] ** 2, rcond=None)[0]
    return float(np.sqrt(K2)), float(-c / K2)
