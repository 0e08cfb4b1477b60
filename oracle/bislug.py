"""Oracle of the bi-slug measurements of Sec. VI.  TEST INFRASTRUCTURE ONLY:
used by the test-suite to check the library's bi-slug runs; written
separately from the package (no shared code), pinned in tests/test_bislug_cpu.py.

  * trajectory(wl, steps, every): an FP64 oracle lattice of the workload,
    stepped, with the liquid (C2 + C3) centre of mass along x sampled every
    `every` steps: the circular mean over the channel rows 1 .. ny - 2, the
    first sample in [0, nx), each later one unwrapped to lie nearest the
    previous one;
  * steady_velocity(H, L, gammas, thetas, rho_l, rho_g, L_gas, nu): Eqs.
    capillaryforce and bislugvelocity, with the gas columns' Poiseuille
    friction added (the paper's law when rho_g -> 0).
"""
import math

from . import from_workload


def _centre(C, prev):
    ny, nx = C.shape[2], C.shape[3]
    s = c = 0.0
    for x in range(nx):
        m = 0.0
        for y in range(1, ny - 1):
            m += C[1, 0, y, x] + C[2, 0, y, x]
        s += m * math.sin(2.0 * math.pi * x / nx)
        c += m * math.cos(2.0 * math.pi * x / nx)
    xc = math.atan2(s, c) * nx / (2.0 * math.pi)
    if prev is None:
        return xc + nx if xc < 0.0 else xc
    else:
        while xc - prev > nx / 2.0:
            xc -= nx
        while prev - xc > nx / 2.0:
            xc += nx
    return xc


def trajectory(wl, steps, every):
    o = from_workload(wl)
    ts, xs = [0], [_centre(o.fields()["C"], None)]
    t = 0
    while t + every <= steps:
        o.step(every)
        t += every
        ts.append(t)
        xs.append(_centre(o.fields()["C"], xs[-1]))
    return ts, xs


def steady_velocity(H, L, gammas, thetas, rho_l, rho_g=0.0, L_gas=0.0, nu=1.0 / 6.0):
    g12, g13, g23 = gammas
    t21, t31, t23 = thetas
    dg = (g23 * math.cos(math.radians(t23)) - g13 * math.cos(math.radians(t31))
          + g12 * math.cos(math.radians(t21)))
    return 2.0 * dg * H / (12.0 * nu * (rho_l * L + rho_g * L_gas))
