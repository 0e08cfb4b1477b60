"""GPU (CUDA, sm_103a) library on the wall cases that pin the oracle's
boundary rules, through the C ABI.

- Eq. forceBC on flat walls with a uniform fluid at rest: the force is -n/6
  times the phase's wetting strength on the second fluid layer and zero
  elsewhere, in D2Q9 and D3Q27, for liquid 2, liquid 3 and the gas.
- Eq. interp3D: a spike on the corner of the interpolation cell nearest (i, j)
  leaves the ghost on the linear value, a spike on a kept corner moves it by
  that corner's barycentric weight.
- Corner ghosts (the average over fluid-facing axes): on a block in a periodic
  box with a drop on the diagonal, the ghost layer matches the oracle and is
  mirror-symmetric; the step keeps the fields symmetric to FP32 rounding.

FP32 bounds: values are O(1-6), so single-precision rounding of the ghost and
force arithmetic stays below 1e-5 absolute; the planted effects are 1e-2 and
larger.
"""
import numpy as np
import pytest

from paper_1904_06881_gb300 import workloads as W

from helpers import gpu_from_workload, oracle_from_workload, record

pytestmark = pytest.mark.gpu


def _wl(lat, nx, ny, nz, mask, rho, phi, **params):
    return dict(lattice=lat, nx=nx, ny=ny, nz=nz, mask=mask, rho=rho, phi=phi, params=W.base_params(**params))


@pytest.mark.parametrize("lat", [W.D2Q9, W.D3Q27])
@pytest.mark.parametrize("phase", ["liquid2", "liquid3", "gas"])
def test_force_wetting_closed_form(lat, phase):
    kr, kp = 0.03, 0.07
    shape = (1, 10, 6) if lat == W.D2Q9 else (8, 5, 5)
    mask = np.zeros(shape, np.uint8)
    if lat == W.D2Q9:
        mask[0, 0, :] = mask[0, -1, :] = 1
    else:
        mask[0] = mask[-1] = 1
    rl, rg = W.RHO_L, W.RHO_G
    rho, phi, amp = {"liquid2": (rl, 5.0, kr + kp), "liquid3": (rl, -5.0, kr - kp), "gas": (rg, 0.0, 0.0)}[phase]
    wl = _wl(lat, shape[2], shape[1], shape[0], mask, np.full(shape, rho), np.full(shape, phi),
             wetting=W.WET_FORCE, kw_rho=kr, kw_phi=kp)
    g = gpu_from_workload(wl)
    axis = "Fy" if lat == W.D2Q9 else "Fz"
    Fn = g.aux(axis)
    Fn = Fn[0] if lat == W.D2Q9 else Fn
    layers = Fn.reshape(Fn.shape[0], -1)
    want = np.zeros(layers.shape[0])
    want[2], want[-3] = -amp / 6.0, amp / 6.0
    fl = slice(1, layers.shape[0] - 1)
    err = np.abs(layers[fl] - want[fl, None]).max()
    record("force wetting closed form %s %s" % ("d2q9" if lat == W.D2Q9 else "d3q27", phase), abs_err=err)
    assert err < 1e-6, (phase, layers[:, 0])
    for k in ("Fx", "Fy", "Fz")[:2 if lat == W.D2Q9 else 3]:
        if k != axis:
            assert np.abs(g.aux(k)[mask == 0]).max() < 1e-6


@pytest.mark.parametrize("corner", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_interp3d_support_drops_the_nearest_corner(corner):
    n, nz, s, spike = 24, 6, 0.04, 0.3
    theta = float(np.degrees(np.arctan(1.0 / 2.5)))
    mask = np.zeros((nz, n, n), np.uint8)
    mask[0] = mask[-1] = 1
    rl, rg = W.RHO_L, W.RHO_G
    u = np.array([0.92, 0.16]) / np.hypot(0.92, 0.16)
    z, y, x = np.mgrid[0:nz, 0:n, 0:n].astype(float)
    rho = 0.5 * (rl + rg) + s * (u[0] * (x - n / 2) + u[1] * (y - n / 2))
    i, j = 8, 10
    rho[1, j + corner[1], i + corner[0]] += spike
    phi = 5.0 * (rho - rg) / (rl - rg)
    wl = _wl(W.D3Q27, n, n, nz, mask, rho, phi, wetting=W.WET_GEOM_INTERP, theta_deg=(theta, 70.0, 110.0))
    g = gpu_from_workload(wl)
    o = oracle_from_workload(wl)
    gg = g.aux("rho_ghost")[0, j, i]
    go = o.aux("rho_ghost")[0, j, i]
    linear = 0.5 * (rl + rg) + s * (u[0] * (i - n / 2) + u[1] * (j - n / 2)) + s * 2.5
    lx, ly = 2.5 * u
    b = 3.0 - lx
    c = ly - b
    weight = {(2, 0): 0.0, (3, 0): 1.0 - b - c, (2, 1): b, (3, 1): c}[corner]
    record("interp3d support corner %s" % (corner,), gpu_minus_expected=gg - (linear + weight * spike),
           gpu_minus_oracle=gg - go)
    assert abs(gg - (linear + weight * spike)) < 1e-5, (corner, gg - linear, weight * spike)
    assert abs(gg - go) < 1e-5


@pytest.mark.parametrize("wet", [W.WET_GEOM_EXTRAP, W.WET_GEOM_INTERP])
def test_corner_ghosts_match_and_keep_the_mirror_symmetry(wet):
    n = 32
    mask = np.zeros((1, n, n), np.uint8)
    mask[0, 12:18, 12:18] = 1
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    C2 = 0.5 * (1 - np.tanh((np.hypot(xx - 10.0, yy - 10.0) - 6.0) / 2.0))
    rho, phi = W.phase_fields(C2, np.zeros_like(C2))
    wl = _wl(W.D2Q9, n, n, 1, mask, rho.reshape(1, n, n), phi.reshape(1, n, n), wetting=wet,
             theta_deg=(60.0, 70.0, 110.0))
    g = gpu_from_workload(wl)
    o = oracle_from_workload(wl)
    ring = mask[0] == 1
    dr = g.derived["rho_l"] - g.derived["rho_g"]
    gg, go = g.aux("rho_ghost")[0], o.aux("rho_ghost")[0]
    vs_oracle = np.abs(gg - go)[ring].max() / dr
    asym0 = np.abs(gg - gg.T)[ring].max() / dr
    g.step(200)
    r = g.fields()["rho"][0]
    asym = np.abs(r - r.T).max() / dr
    record("corner ghosts, block in a periodic box, wetting %d" % wet, ghost_vs_oracle=vs_oracle,
           ghost_asymmetry=asym0, asymmetry_after_200=asym)
    assert vs_oracle < 2e-6 and asym0 < 2e-6
    # measured 4e-7 and 3e-7; a one-axis corner rule gives 0.3 (oracle)
    assert asym < 1e-4
