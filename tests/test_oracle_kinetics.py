"""Pins of the oracle's lattice kinetics (Sec. II.C) against textbook facts.

- lattice tables: the D1Q3 product lattices' weight moments;
- product-form equilibrium (Eqs. eqrho, A, B): exact mass and momentum, the
  closed-form second moment of the D1Q3 factor, and that ln(f^eq/w) is linear
  in c (f^eq minimises H at fixed mass and momentum);
- entropic alpha (Eq. EntropyEquation): residual, bracket, a 50-digit
  brute-force root, and the small-deviation series of the root;
- g^eq (Sec. II.C): BGK moments phi, phi v, Gamma mu I + phi v v.
"""
import mpmath
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_lattice_weight_moments(lat):
    c, w = oracle.lattice(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    c = c[:, :D].astype(float)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    assert np.allclose((w[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0), np.eye(D) / 3, atol=1e-15)
    # fourth-order isotropy of the product lattices
    assert np.isclose((w * c[:, 0] ** 4).sum(), 1 / 3, atol=1e-15)
    assert np.isclose((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum(), 1 / 9, atol=1e-15)
    assert (c[0] == 0).all() and np.isclose(w[0], (2 / 3) ** D)


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_feq_moments_closed_form(lat):
    rng = np.random.default_rng(1)
    c, w = oracle.lattice(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    c = c[:, :D].astype(float)
    for _ in range(20):
        rho = rng.uniform(0.01, 10.0)
        u = rng.uniform(-0.4, 0.4, D)
        f = oracle.feq(lat, rho, u)
        assert np.isclose(f.sum(), rho, rtol=1e-14)
        assert np.allclose(f @ c, rho * u, rtol=1e-13, atol=1e-15)
        # D1Q3 factor: sum_c c^2 w(c) A B^c = (1/6) A (B + 1/B) = (2 sqrt(1+3u^2) - 1)/3
        for a in range(D):
            assert np.isclose((f * c[:, a] ** 2).sum(), rho * (2 * np.sqrt(1 + 3 * u[a] ** 2) - 1) / 3,
                              rtol=1e-13)
        assert (f > 0).all()
    assert np.allclose(oracle.feq(lat, 2.5, np.zeros(D)), 2.5 * w, rtol=1e-15)


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_feq_is_entropy_minimiser(lat):
    """ln(f_i^eq / w_i) is affine in c_i, i.e. f^eq is the stationary point of
    H = sum f ln(f/w) under the mass and momentum constraints; moving along any
    direction that keeps those moments raises H."""
    rng = np.random.default_rng(2)
    c, w = oracle.lattice(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    c = c[:, :D].astype(float)
    M = np.hstack([np.ones((len(w), 1)), c])            # moment matrix (Q x (1+D))
    for _ in range(10):
        rho, u = rng.uniform(0.1, 5.0), rng.uniform(-0.3, 0.3, D)
        f = oracle.feq(lat, rho, u)
        y = np.log(f / w)
        coef, *_ = np.linalg.lstsq(M, y, rcond=None)
        assert np.abs(M @ coef - y).max() < 1e-12
        null = np.linalg.svd(M.T)[2][1 + D:]            # directions with zero mass/momentum change
        H0 = oracle.entropy(lat, f)
        for d in null[:4]:
            eps = 1e-3 * f.min()
            assert oracle.entropy(lat, f + eps * d / np.abs(d).max()) > H0


def _mirror_and_delta(lat, rng, scale):
    c, w = oracle.lattice(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    c = c[:, :D].astype(float)
    rho, u = rng.uniform(0.1, 5.0), rng.uniform(-0.2, 0.2, D)
    feq = oracle.feq(lat, rho, u)
    fp = feq * (1.0 + scale * rng.uniform(-1, 1, len(w)))
    # project the perturbation so that fp keeps the moments of feq
    M = np.hstack([np.ones((len(w), 1)), c])
    dev = fp - feq
    dev -= M @ np.linalg.lstsq(M, dev, rcond=None)[0]
    fp = feq + dev
    return fp, feq - fp, w


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_alpha_root_residual_and_bracket(lat):
    rng = np.random.default_rng(3)
    for scale in (1e-4, 1e-2, 0.1, 0.4):
        for _ in range(5):
            fp, dl, w = _mirror_and_delta(lat, rng, scale)
            if (fp <= 0).any():
                continue
            al, st = oracle.alpha(lat, fp, dl)
            amax = min([-fp[i] / dl[i] for i in range(len(fp)) if dl[i] < 0] + [np.inf])
            H0 = oracle.entropy(lat, fp)
            if st == 2:
                # no root below the positivity bound: alpha is clipped just below it
                assert oracle.entropy(lat, fp + amax * (1 - 1e-12) * dl) < H0
                assert np.isclose(al, amax * (1 - 1e-6), rtol=1e-12)
                continue
            assert st == 0
            assert 1.0 < al <= amax
            Hs = np.abs(fp * np.log(fp / w)).sum() + fp.sum()
            assert abs(oracle.entropy(lat, fp + al * dl) - H0) <= 1e-13 * Hs


def test_alpha_matches_brute_force_high_precision():
    """The root of h(alpha) = H(f'+alpha delta) - H(f') found in 50-digit
    arithmetic by mpmath agrees with the FP64 oracle."""
    rng = np.random.default_rng(4)
    mpmath.mp.dps = 50
    for scale in (1e-3, 0.05, 0.3):
        fp, dl, w = _mirror_and_delta(oracle.D2Q9, rng, scale)
        F = [mpmath.mpf(float(x)) for x in fp]
        Dl = [mpmath.mpf(float(x)) for x in dl]
        W = [mpmath.mpf(float(x)) for x in w]

        def h(a):
            return (sum((F[i] + a * Dl[i]) * mpmath.log((F[i] + a * Dl[i]) / W[i]) for i in range(9))
                    - sum(F[i] * mpmath.log(F[i] / W[i]) for i in range(9)))

        amax = min([-fp[i] / dl[i] for i in range(9) if dl[i] < 0] + [1e3])
        ref = mpmath.findroot(h, (mpmath.mpf(1.0), mpmath.mpf(amax) * (1 - mpmath.mpf(10) ** -12)),
                              solver="anderson")
        al, st = oracle.alpha(oracle.D2Q9, fp, dl)
        assert abs(al - float(ref)) < 1e-8 * float(ref)


def test_alpha_tends_to_two_near_equilibrium():
    rng = np.random.default_rng(5)
    devs = []
    for scale in (1e-2, 1e-3, 1e-4):
        fp, dl, w = _mirror_and_delta(oracle.D2Q9, rng, scale)
        al, st = oracle.alpha(oracle.D2Q9, fp, dl)
        devs.append(abs(al - 2.0))
    assert devs[2] < devs[0] and devs[2] < 1e-2
    fp, dl, w = _mirror_and_delta(oracle.D2Q9, rng, 1e-9)
    assert oracle.alpha(oracle.D2Q9, fp, dl) == (2.0, 1)


def _series_root(fp, x):
    """alpha = 2 + e1 + ... + e5: the root of h(alpha) = sum_i f'_i [phi(alpha
    x_i) - alpha x_i ln(1 + x_i)] expanded in the moments b_k = a_k / a_2,
    a_k = sum_i f'_i x_i^k, order by order (h(alpha) = sum_k a_k c_k(alpha),
    c_k = (-1)^k alpha (alpha^(k-1) - k) / (k (k - 1)), a_1 = 0)."""
    a = {k: float((fp * x ** k).sum()) for k in range(2, 8)}
    b3, b4, b5, b6, b7 = (a[k] / a[2] for k in range(3, 8))
    e1 = b3 / 3
    e2 = 4 * b3 ** 2 / 9 - 2 * b4 / 3
    e3 = 17 * b3 ** 3 / 27 - 14 * b3 * b4 / 9 + 11 * b5 / 10
    e4 = 76 * b3 ** 4 / 81 - 29 * b3 ** 2 * b4 / 9 + 38 * b3 * b5 / 15 + 4 * b4 ** 2 / 3 - 26 * b6 / 15
    e5 = (118 * b3 ** 5 / 81 - 1037 * b3 ** 3 * b4 / 162 + 239 * b3 ** 2 * b5 / 45 + 148 * b3 * b4 ** 2 / 27
          - 184 * b3 * b6 / 45 - 13 * b4 * b5 / 3 + 19 * b7 / 7)
    return 2.0 + e1 + e2 + e3 + e4 + e5


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_alpha_matches_the_small_deviation_series(lat):
    """Near equilibrium the exact root approaches its asymptotic series: on
    states f' + D = f^eq(rho, U) with D carrying no mass or momentum and
    max_i |D_i / f'_i| = m, the oracle's root and the fifth-order series
    differ by less than 1e-6 at m = 0.1 and 1e-7 at m = 0.07, and the
    difference falls by at least 4 from m = 0.1 to 0.07 (the sixth-order
    term scales as m^6: a factor of 8.5)."""
    c, w = oracle.lattice(lat)
    Q = len(w)
    M = np.vstack([np.ones(Q), c[:, 0], c[:, 1], c[:, 2]])
    P = np.eye(Q) - M.T @ np.linalg.pinv(M.T)
    rng = np.random.default_rng(11)
    worst = {}
    for m in (0.1, 0.07):
        worst[m] = 0.0
        for _ in range(200):
            rho = rng.uniform(0.3, 6.0)
            U = rng.uniform(-0.1, 0.1, 3)
            if lat == oracle.D2Q9:
                U[2] = 0.0
            fe = oracle.feq(lat, rho, U)
            d = P @ rng.normal(size=Q)
            s = m / np.abs(d / fe).max()
            for _ in range(60):        # scale so that max |d / (fe - d)| = m
                s *= m / np.abs(s * d / (fe - s * d)).max()
            d = s * d
            fp = fe - d
            al, st = oracle.alpha(lat, fp, d)
            worst[m] = max(worst[m], abs(al - _series_root(fp, d / fp)))
    assert worst[0.1] < 1e-6 and worst[0.07] < 1e-7, worst
    assert worst[0.1] > 4.0 * worst[0.07], worst


@pytest.mark.parametrize("lat", [oracle.D2Q9, oracle.D3Q27])
def test_geq_moments(lat):
    rng = np.random.default_rng(6)
    c, w = oracle.lattice(lat)
    D = 2 if lat == oracle.D2Q9 else 3
    c = c[:, :D].astype(float)
    for _ in range(10):
        phi, mu, G = rng.uniform(-5, 5), rng.uniform(-0.1, 0.1), rng.uniform(0.5, 2.0)
        v = rng.uniform(-0.2, 0.2, D)
        g = oracle.geq(lat, phi, v, mu, G)
        assert np.isclose(g.sum(), phi, atol=1e-13)
        assert np.allclose(g @ c, phi * v, atol=1e-13)
        second = (g[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
        assert np.allclose(second, G * mu * np.eye(D) + phi * np.outer(v, v), atol=1e-13)


@pytest.mark.parametrize("phase,expect", [("C1", 0.05), ("C2", 0.1), ("C3", 0.03), ("one beta", 1.0 / 6.0)])
def test_shear_wave_decays_at_the_component_viscosity(phase, expect):
    """Per-component viscosity (an extension: the paper has one beta): a
    shear wave u_x = U sin(2 pi y / L) in a uniform phase decays as
    exp(-nu k^2 t), with nu the viscosity given for that component (1/6 for
    beta = 1/2 when none is given), to 1 % (the lattice's own O(k^2)
    correction is below that at L = 64)."""
    import oracle as O
    from paper_1904_06881_gb300 import workloads as W

    rl, rg, chi = W.RHO_L, W.RHO_G, 5.0
    rho0, phi0 = {"C1": (rg, 0.0), "C2": (rl, chi), "C3": (rl, -chi), "one beta": (rl, chi)}[phase]
    nu = (0.0, 0.0, 0.0) if phase == "one beta" else (0.05, 0.1, 0.03)
    nx, ny, U, steps = 4, 64, 1e-4, 400
    o = O.Oracle(nx=nx, ny=ny, rho_l=rl, rho_g=rg, nu=nu)
    o.set_solid(np.zeros((1, ny, nx), np.uint8))
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    s = np.sin(2 * np.pi * y / ny)
    u = np.zeros((2, 1, ny, nx))
    u[0, 0] = U * s
    o.init_fields(np.full((1, ny, nx), rho0), np.full((1, ny, nx), phi0), u)
    o.step(steps)
    ux = o.fields()["u"][0, 0]
    amp = 2.0 * (ux * s).mean()
    k = 2 * np.pi / ny
    nu_meas = -np.log(amp / U) / (k * k * steps)
    assert abs(nu_meas / expect - 1.0) < 0.01, (nu_meas, expect)
