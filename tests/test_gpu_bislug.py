"""The self-propelled bi-slug (Sec. VI) on the GPU against the FP64 oracle:
the same 240 x 21 train (theta = 60 deg) stepped 2000 steps by both, the
centroid trajectory measured by the package's and the oracle's own code, to
2e-3 lattice units (the FP32 fields agree to ~1e-5 normwise); the library's
train at theta = 90 deg stays put to 1e-3.  Then the paper's geometry
(H = 39, L = 1500, 400 gas nodes, 20 000 steps), whose steady velocity is
printed beside the long-train law with the library's own tensions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trajectory_matches_oracle():
    import oracle.bislug as OB
    from paper_1904_06881_gb300 import bislug as B
    from paper_1904_06881_gb300 import workloads as W

    wl = W.bislug_2d(theta=60.0)
    ts, xg = B.run(wl, 2000, 500)
    to, xo = OB.trajectory(wl, 2000, 500)
    assert list(ts) == list(to)
    assert np.max(np.abs(np.array(xg) - np.array(xo))) < 2e-3, (xg, xo)
    _, x90 = B.run(W.bislug_2d(theta=90.0), 2000, 500)
    assert np.max(np.abs(x90 - x90[0])) < 1e-3, x90


def test_paper_geometry_steady_velocity():
    from paper_1904_06881_gb300 import bislug as B
    from paper_1904_06881_gb300 import tension as T
    from paper_1904_06881_gb300 import workloads as W

    H, L, gas, theta = 39, 1500, 400, 60.0
    wl = W.bislug_2d(H=H, L1=L // 2, L2=L - L // 2, gas=gas, theta=theta)
    ts, xs = B.run(wl, 20000, 1000)
    v = np.diff(xs) / np.diff(ts)
    res, _ = T.sweep([dict(lam=wl["params"]["lam"], kappa=wl["params"]["kappa"])], L=96, R=24.0, steps=4000)
    g = res[0]["gamma"]
    law = B.theory(H, L, (g["12"], g["13"], g["23"]), (theta,) * 3, W.RHO_L, W.RHO_G, gas)
    print("bi-slug H %d L %d: steady velocity %.3e (last 5000 steps), long-train law %.3e (ratio %.2f), tau_rel %.0f"
          % (H, L, v[-5:].mean(), law["v_inf"], v[-5:].mean() / law["v_inf"], law["tau_rel"]))
    assert v[-5:].mean() > 0 and np.all(np.isfinite(xs))


def _relaxation_time(ts, vs):
    """tau of v(t) = v_inf - A exp(-t / tau) (Eq. centroidvelocity with a free
    initial offset: the slugs start rectangular and reshape in the first
    steps), least squares over (v_inf, A, tau)."""
    from scipy.optimize import curve_fit

    popt, _ = curve_fit(lambda t, v, A, tau: v - A * np.exp(-t / tau), ts, vs,
                        p0=(vs[-1], vs[-1], 700.0), bounds=([-1.0, -1.0, 50.0], [1.0, 1.0, 5000.0]))
    return float(popt[2])


def test_dynamic_angles_account_for_the_steady_velocity():
    """Sec. VI, paper geometry (H = 39, 400 gas nodes), all angles 60 deg, three
    train lengths: the steady velocity against the long-train law
    (Eqs. capillaryforce-bislugvelocity) with the static angles and with the
    measured dynamic ones (averaged over the last 2000 of 8000 steps) in
    Delta gamma, the paper's correction.  The dynamic angles bring the law
    closer to the measurement for every length (measured ratios 0.63, 0.75,
    0.80 against 0.44, 0.51, 0.52 with the static angles), within 25 % at
    L = 1200 (L/H = 31).  The relaxation time fitted to the velocity (Eq.
    centroidvelocity) and Cox's slip length of each interface are reported:
    the liquid-liquid interface's angle oscillates by 3-4 deg over the run,
    which makes the fitted time scatter (190-990 against H^2/(12 nu) = 760).
    """
    from paper_1904_06881_gb300 import bislug as B
    from paper_1904_06881_gb300 import tension as T
    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    from helpers import record

    H, gas, theta, Ls = 39, 400, 60.0, (300, 600, 1200)
    wls = [W.bislug_2d(H=H, L1=L // 2, L2=L - L // 2, gas=gas, theta=theta) for L in Ls]
    lats = [tlb.lattice_from_workload(w) for w in wls]
    d = lats[0].derived
    b = tlb.Batch(lats)
    every, steps, avg_from = 250, 8000, 6000
    xs = [[B.centroid(l.fields()["C"][:, 0])] for l in lats]
    angs = [[] for _ in lats]
    for k in range(steps // every):
        b.step(every)
        for i, l in enumerate(lats):
            f = l.fields()
            xs[i].append(B.centroid(f["C"][:, 0], xs[i][-1]))
            if (k + 1) * every > avg_from:
                angs[i].append(B.dynamic_angles(f, d["rho_l"], d["rho_g"]))
    res, _ = T.sweep([dict(lam=wls[0]["params"]["lam"], kappa=wls[0]["params"]["kappa"])], L=96, R=24.0, steps=4000)
    g = res[0]["gamma"]
    gam = (g["12"], g["13"], g["23"])
    tau_law = H * H / (12.0 / 6.0)
    runs = []
    for L, x, al in zip(Ls, xs, angs):
        x = np.array(x)
        v = np.diff(x) / every
        tv = every * (np.arange(len(v)) + 0.5)
        v_inf = float(v[-8:].mean())
        ang = {k: float(np.mean([a[k] for a in al])) for k in al[0]}
        law = B.theory(H, L, gam, (theta,) * 3, d["rho_l"], d["rho_g"], gas)["v_inf"]
        law_dyn = B.theory(H, L, gam, (ang["theta_21"], ang["theta_31"], ang["theta_23"]), d["rho_l"], d["rho_g"],
                           gas)["v_inf"]
        tau = _relaxation_time(tv[tv >= 500], v[tv >= 500])
        record("bi-slug H 39 L %d theta 60" % L, v_inf=v_inf, law_static=law, law_dynamic=law_dyn,
               ratio_static=v_inf / law, ratio_dynamic=v_inf / law_dyn, tau_rel=tau, tau_law=tau_law, angles=ang,
               angle_spread={k: float(np.ptp([a[k] for a in al])) for k in al[0]})
        runs.append((v_inf, ang))
        assert abs(v_inf / law_dyn - 1.0) < abs(v_inf / law - 1.0), (v_inf, law, law_dyn)
        if L == 1200:
            assert abs(v_inf / law_dyn - 1.0) < 0.25, (v_inf, law_dyn)
    slip = B.cox_slip(runs, gam, (d["rho_g"], d["rho_l"], d["rho_l"]), Lc=float(H))
    record("bi-slug Cox slip lengths, theta 60, L 300-1200", **{k: v["L_s"] for k, v in slip.items()},
           **{k + "_w": v["theta_w"] for k, v in slip.items()})
    assert all(np.isfinite(v["L_s"]) and v["L_s"] > 0 for v in slip.values())
