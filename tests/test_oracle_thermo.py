"""Pins of the oracle's thermodynamics (Sec. II.A-B, Sec. III).

- the printed Psi_eos is the Carnahan-Starling free energy: p = rho Psi' - Psi
  equals the textbook CS pressure, and the printed dPsi/drho is the derivative;
- T_c is the CS critical point (0.3773 a/(bR); the printed 0.3373 is a typo);
- coexistence: equal textbook pressure, equal chemical potential, Maxwell's
  equal-area rule;
- the three bulk minima are stationary states;
- stencils exact on quadratics (Laplacian) and products of linear fields
  (pressure tensor off-diagonal);
- phi -> -phi mirror symmetry of set 1 (fixes the sign of the lambda_2 term
  in mu_rho, derived from Eq. BulkEnergy);
- flat liquid-liquid interface: the tanh profile of Eq. profile with alpha_23
  of Eq. liquidliquidalpha;
- gamma_23 from the Laplace jump against Eq. tension23.
"""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq, curve_fit

import oracle
from paper_1904_06881_gb300 import workloads as W

A, B, R = 0.037, 0.2, 1.0


def cs_pressure(rho, a, b, R_, T):
    eta = b * rho / 4.0
    return rho * R_ * T * (1 + eta + eta ** 2 - eta ** 3) / (1 - eta) ** 3 - a * rho ** 2


def test_psi_is_carnahan_starling_and_derivative_matches():
    T = 0.05
    for rho in (0.01, 0.3, 2.0, 7.5, 12.0):
        psi = oracle.eos_psi(rho, A, B, R, T, 0.0)
        dpsi = oracle.eos_dpsi(rho, A, B, R, T, 0.0)
        assert np.isclose(rho * dpsi - psi, cs_pressure(rho, A, B, R, T), rtol=1e-12)
        h = 1e-6 * rho
        num = (oracle.eos_psi(rho + h, A, B, R, T, 0.0) - oracle.eos_psi(rho - h, A, B, R, T, 0.0)) / (2 * h)
        assert np.isclose(num, dpsi, rtol=1e-7)


def test_critical_temperature_is_cs_critical_point():
    # textbook CS critical point: dp/drho = d2p/drho2 = 0
    def dp(rho, T, k):
        h = 1e-4 * rho
        if k == 1:
            return (cs_pressure(rho + h, A, B, R, T) - cs_pressure(rho - h, A, B, R, T)) / (2 * h)
        return (cs_pressure(rho + h, A, B, R, T) - 2 * cs_pressure(rho, A, B, R, T)
                + cs_pressure(rho - h, A, B, R, T)) / h ** 2

    def min_dp(T):
        rs = np.linspace(0.05, 19.0, 4000)
        return min(dp(r, T, 1) for r in rs)

    Tc_ref = brentq(min_dp, 0.03, 0.1, xtol=1e-10)
    Tc = oracle.eos_critical_T(A, B, R)
    assert np.isclose(Tc, Tc_ref, rtol=1e-4)
    assert np.isclose(Tc * B * R / A, 0.3773, atol=2e-4)


@pytest.mark.parametrize("tred", [0.61, 0.8, 0.95])
def test_coexistence_equal_pressure_mu_and_area(tred):
    Tc = oracle.eos_critical_T(A, B, R)
    T = tred * Tc
    co = oracle.eos_coexistence(A, B, R, T)
    rg, rl = co["rho_g"], co["rho_l"]
    pg, pl = cs_pressure(rg, A, B, R, T), cs_pressure(rl, A, B, R, T)
    assert np.isclose(pg, pl, rtol=1e-9)

    # textbook CS chemical potential (up to a constant):
    def mu(r):
        eta = B * r / 4
        return R * T * (np.log(r) + (8 * eta - 9 * eta ** 2 + 3 * eta ** 3) / (1 - eta) ** 3) - 2 * A * r

    assert np.isclose(mu(rg), mu(rl), rtol=1e-9, atol=1e-12)
    # Maxwell equal area in the (1/rho, p) plane
    area = quad(lambda v: cs_pressure(1 / v, A, B, R, T) - pg, 1 / rl, 1 / rg, limit=400)[0]
    assert abs(area) < 1e-8 * pg * (1 / rg - 1 / rl)
    # C makes dPsi/drho vanish at both phases, Psi(rho_g) = Psi(rho_l) = Psi0
    for r in (rg, rl):
        assert abs(oracle.eos_dpsi(r, A, B, R, T, co["C"])) < 1e-10
        assert np.isclose(oracle.eos_psi(r, A, B, R, T, co["C"]), co["Psi0"], rtol=1e-9, atol=1e-12)


def _mk(nx, ny, nz=1, lat=oracle.D2Q9, **over):
    p = W.base_params(**over)
    return oracle.Oracle(lattice=lat, nx=nx, ny=ny, nz=nz, lam=p["lam"], kappa=p["kappa"],
                         chi=p["chi"], a=p["a"], b=p["b"], R=p["R"], rho_l=p["rho_l"],
                         rho_g=p["rho_g"], beta=p["beta"], tau_g=p["tau_g"], Gamma=p["Gamma"],
                         wetting=p["wetting"], theta_deg=p["theta_deg"], kw_rho=p["kw_rho"],
                         kw_phi=p["kw_phi"])


def test_rescaled_densities_hit_targets():
    o = _mk(8, 8, rho_l=1.0, rho_g=1e-3)
    d = o.derived
    assert np.isclose(d["rho_l"], 1.0, rtol=1e-9) and np.isclose(d["rho_g"], 1e-3, rtol=1e-7)
    assert np.isclose(d["a"] / d["b"], A / B, rtol=1e-12)       # T_c unchanged
    o = _mk(8, 8)
    assert np.isclose(o.derived["a"], A, rtol=1e-9) and np.isclose(o.derived["b"], B, rtol=1e-9)


@pytest.mark.parametrize("state", ["gas", "liq2", "liq3"])
def test_bulk_minima_are_stationary(state):
    o = _mk(8, 6)
    d = o.derived
    rho = {"gas": d["rho_g"], "liq2": d["rho_l"], "liq3": d["rho_l"]}[state]
    phi = {"gas": 0.0, "liq2": 5.0, "liq3": -5.0}[state]
    o.init_fields(np.full((1, 6, 8), rho), np.full((1, 6, 8), phi))
    for name in ("mu_rho", "mu_phi", "p0", "Fx", "Fy"):
        assert np.abs(o.aux(name)).max() < 1e-12, name
    o.step(50)
    f = o.fields()
    assert np.abs(f["rho"] - rho).max() < 1e-12 * rho and np.abs(f["phi"] - phi).max() < 1e-12


def test_laplacian_stencil_exact_on_quadratic():
    """mu_rho at a node differs between a quadratic field and a uniform field of
    the same value there only through -kappa_rr lap(rho) (Sec. II.B)."""
    nx = ny = 16
    o1, o2 = _mk(nx, ny), _mk(nx, ny)
    rho0, eps = 3.0, 1e-3
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    q = (x - 8) ** 2 + 2 * (y - 8) ** 2          # lap q = 6
    phi = np.full((1, ny, nx), 2.0)
    o1.init_fields((rho0 + eps * q)[None], phi)
    o2.init_fields(np.full((1, ny, nx), rho0), phi)
    dmu = o1.aux("mu_rho")[0, 8, 8] - o2.aux("mu_rho")[0, 8, 8]
    assert np.isclose(dmu, -o1.derived["kappa_rr"] * eps * 6.0, rtol=1e-9)


def test_pressure_tensor_offdiagonal_exact_on_linear_field():
    nx = ny = 16
    o = _mk(nx, ny)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    sx, sy = 0.01, -0.02
    rho = 3.0 + sx * (x - 8) + sy * (y - 8)
    o.init_fields(rho[None], np.full((1, ny, nx), 1.0))
    pxy = o.aux("Pxy")[0, 8, 8]
    assert np.isclose(pxy, o.derived["kappa_rr"] * sx * sy, rtol=1e-9)


def test_phi_mirror_symmetry_of_set1():
    """Set 1 is symmetric under phi -> -phi (C2 <-> C3); a liquid-2 drop and the
    mirrored liquid-3 drop evolve into mirrored fields."""
    nx = ny = 32
    mask, rho, phi = W.sessile_drop_2d(nx, ny, 8.0, yc=ny / 2, walls=(), liquid=2)
    _, rho3, phi3 = W.sessile_drop_2d(nx, ny, 8.0, yc=ny / 2, walls=(), liquid=3)
    assert np.allclose(rho, rho3) and np.allclose(phi, -phi3)
    o2, o3 = _mk(nx, ny), _mk(nx, ny)
    o2.init_fields(rho, phi)
    o3.init_fields(rho3, phi3)
    o2.step(200)
    o3.step(200)
    f2, f3 = o2.fields(), o3.fields()
    assert np.abs(f2["rho"] - f3["rho"]).max() < 1e-10
    assert np.abs(f2["phi"] + f3["phi"]).max() < 1e-10
    assert np.abs(f2["phi"]).max() > 1.0


def _ll_slab(nx, lam, kappa, steps):
    o = _mk(nx, 3, lam=lam, kappa=kappa)
    rl = o.derived["rho_l"]
    x = np.arange(nx, dtype=float)
    prof = np.tanh((x - nx / 4) / 3.0) * np.tanh((3 * nx / 4 - x) / 3.0)   # liquid 2 in the middle
    o.init_fields(np.full((1, 3, nx), rl), np.tile(5.0 * prof, (1, 3, 1)))
    o.step(steps)
    return o, o.fields()["C"][1, 0, 1]


@pytest.mark.parametrize("lam23,kap23", [((1.0, 1.0), (1.0, 1.0)), ((0.5, 0.5), (1.0, 1.0)),
                                         ((1.5, 1.5), (1.5, 1.5))])
def test_flat_liquid_liquid_tanh_profile(lam23, kap23):
    nx = 96
    o, C2 = _ll_slab(nx, (0.6,) + lam23, (0.01,) + kap23, 3000)
    alpha23 = np.sqrt(sum(kap23) / sum(lam23))
    x = np.arange(nx, dtype=float)
    sel = slice(nx // 4 - 12, nx // 4 + 12)
    popt, _ = curve_fit(lambda xx, x0, al: 0.5 * (1 + np.tanh((xx - x0) / (2 * al))), x[sel], C2[sel],
                        p0=(nx / 4, 1.0))
    assert abs(popt[1] / alpha23 - 1) < 0.03


def _laplace_ll(R_, n=64, steps=4000):
    o = _mk(n, n)
    rl = o.derived["rho_l"]
    y, x = np.mgrid[0:n, 0:n].astype(float)
    C2 = 0.5 * (1 - np.tanh((np.hypot(x - n / 2, y - n / 2) - R_) / 2))
    o.init_fields(np.full((1, n, n), rl), (5.0 * (2 * C2 - 1))[None])
    o.step(steps)
    p = o.aux("p0")[0]
    return p[n // 2, n // 2] - p[0, 0]


@pytest.mark.slow
def test_gamma23_laplace_closed_form():
    """gamma_23 = dP R for two radii agrees with alpha_23 (lambda2+lambda3)/6 = 1/3
    (Eq. tension23) within 5 % (measured 1.0 % and 2.6 % below; the paper's
    own bubble tests read 3 % below it)."""
    g = [_laplace_ll(R_) * R_ for R_ in (12.0, 16.0)]
    assert abs(g[0] / g[1] - 1) < 0.05
    for gi in g:
        assert 0.95 < gi / (1.0 / 3.0) < 1.05


def _gamma12_straight_path(T, s=1.0, lam=(0.6, 1.0, 1.0), kap=(0.01, 1.0, 1.0)):
    """Liquid-gas tension along the interface path with no third component
    (C3 = 0, so phi = chi C2 and C2 = (rho - rho_g)/drho, Sec. III): from
    Eqs. BulkEnergy and InterfEnergy, gamma = int sqrt(2 kappa_eff W) drho
    with kappa_eff = kappa_1 + kappa_2/drho^2 and W the bulk free energy
    above the common tangent (horizontal: dPsi/drho = 0 at both phases).
    The minimising path bends away from this line, so this is an upper bound
    of the model's gamma_12.  a, b scaled by s (s = 1: the printed values)."""
    a, b = A * s, B * s
    co = oracle.eos_coexistence(a, b, R, T)
    rg, rl = co["rho_g"], co["rho_l"]
    dr = rl - rg
    keff = kap[0] + kap[1] / dr ** 2

    def W_(r):
        c2 = (r - rg) / dr
        return 0.5 * lam[0] * (oracle.eos_psi(r, a, b, R, T, co["C"]) - co["Psi0"]) + \
            0.5 * lam[1] * c2 ** 2 * (1 - c2) ** 2

    return quad(lambda r: np.sqrt(max(2.0 * keff * W_(r), 0.0)), rg, rl, limit=200)[0], rl / rg


def test_table1_gamma12_fixes_the_density_scale():
    """Table 1, set 1: gamma_12 = 0.414 at a density ratio of about 10^3
    (Sec. III).  With the printed a = 0.037, b = 0.2 the straight-path bound
    rises with the ratio (0.22 at ratio 14, 0.33 at 115) and reaches the
    printed value between ratios 700 and 1000 (0.418 and 0.432): the paper's
    runs used these constants unscaled.  Scaling a and b to put rho_l at 1
    (same ratio) would give 0.19, half the printed tension."""
    Tc = oracle.eos_critical_T(A, B, R)
    g14, r14 = _gamma12_straight_path(0.8 * Tc)
    g1000, r1000 = _gamma12_straight_path(0.485 * Tc)
    assert abs(r1000 - 1000.0) < 5.0 and abs(r14 - 14.14) < 0.01
    assert g14 < 0.6 * 0.414
    assert 0.414 <= g1000 <= 1.05 * 0.414
    s = oracle.eos_coexistence(A, B, R, 0.485 * Tc)["rho_l"]
    g_scaled, _ = _gamma12_straight_path(0.485 * Tc, s=s)
    assert g_scaled < 0.5 * 0.414


def _vdw_p(rho, a, b, R_, T):
    return rho * R_ * T / (1.0 - b * rho) - a * rho ** 2


def _pr_p(rho, a, b, R_, T, omega=0.344):
    k = 0.37464 + 1.54226 * omega - 0.26992 * omega ** 2
    Tc = (0.07780 / 0.45724) * a / (b * R_)
    aA = a * (1.0 + k * (1.0 - np.sqrt(T / Tc))) ** 2
    return rho * R_ * T / (1.0 - b * rho) - aA * rho ** 2 / (1.0 + 2.0 * b * rho - (b * rho) ** 2)


@pytest.mark.parametrize("kind,pfun,tc", [(oracle.EOS_VDW, _vdw_p, 8.0 / 27.0), (oracle.EOS_PR, _pr_p, 0.07780 / 0.45724)])
def test_alternative_eos_free_energy_and_critical_point(kind, pfun, tc):
    """Van der Waals and Peng-Robinson (Sec. II.A: EOS the model hosts): the
    oracle's Psi_eos gives the textbook pressure through p = rho Psi' - Psi,
    its dPsi/drho is the derivative of Psi, and the critical temperature
    is the textbook one, 8a/(27bR) (vdW, exact) and 0.07780/0.45724 a/(bR)
    (PR, whose constants place the critical point there to their rounding)."""
    e = oracle.eos_k(kind)
    a, b = 0.05, 0.1
    Tc = e["critical_T"](a, b, R)
    assert np.isclose(Tc * b * R / a, tc, rtol=(1e-5 if kind == oracle.EOS_VDW else 2e-4))
    T = 0.8 * Tc
    for rho in (0.05, 0.8, 3.0, 6.0, 8.5):
        psi, dpsi = e["psi"](rho, a, b, R, T, 0.1), e["dpsi"](rho, a, b, R, T, 0.1)
        assert np.isclose(rho * dpsi - psi, pfun(rho, a, b, R, T), rtol=1e-11, atol=1e-14)
        h = 1e-6 * rho
        num = (e["psi"](rho + h, a, b, R, T, 0.1) - e["psi"](rho - h, a, b, R, T, 0.1)) / (2 * h)
        assert np.isclose(num, dpsi, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("kind,pfun", [(oracle.EOS_VDW, _vdw_p), (oracle.EOS_PR, _pr_p)])
def test_alternative_eos_coexistence(kind, pfun):
    """Coexistence of the alternative EOS: equal textbook pressure, equal
    chemical potential and Maxwell's equal-area rule (integral of p - p_coex
    over 1/rho between the phases vanishes)."""
    e = oracle.eos_k(kind)
    a, b = 0.05, 0.1
    T = 0.75 * e["critical_T"](a, b, R)
    c = e["coexistence"](a, b, R, T)
    rg, rl = c["rho_g"], c["rho_l"]
    pg, pl = pfun(rg, a, b, R, T), pfun(rl, a, b, R, T)
    assert np.isclose(pg, pl, rtol=1e-9)
    assert np.isclose(e["dpsi"](rg, a, b, R, T, 0.0), e["dpsi"](rl, a, b, R, T, 0.0), rtol=1e-9, atol=1e-12)
    area = quad(lambda v: pfun(1.0 / v, a, b, R, T) - pg, 1.0 / rl, 1.0 / rg, limit=400)[0]
    assert abs(area) < 1e-8 * pg * (1.0 / rg - 1.0 / rl)
