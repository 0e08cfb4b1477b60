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
