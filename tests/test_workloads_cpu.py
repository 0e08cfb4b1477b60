"""The seeded synthetic inputs (workloads.py) follow their stated recipes.

- c0 (the D2Q9 sessile drop with its seeded noise), c1 (the capillary
  channel) and c2 (the bench's headline D3Q27 lubricated substrate): sizes,
  walls, phases and wetting parameters.
- c3, the batched contact-angle sweep: 256 draws of L in {64, 128, 256, 512}
  and theta_21 ~ U[30, THETA_MAX], each run with force and with geometric-
  interpolation wetting (512 lattices); a sessile drop of radius L/4 on the
  bottom wall; the force lattices carry a strength of the angle's sign.
- c4, the served mix: 256 requests with Poisson arrivals at 20 per second;
  drops, channels, lubricated substrates (D3Q27), lenses and drop trains;
  2D requests take 1000-5000 steps and 3D requests 500-2000; liquid-gas
  density ratios between 4 and 14.1, and liquid-liquid requests.
Both are deterministic for their seeds.  The c4 mix is built here with small
3D sizes (the arrays of its 96^3-192^3 lattices need about 1.5 GB); what is
checked does not depend on them, and the default sizes are checked apart.
"""
import inspect

import numpy as np

from paper_1904_06881_gb300 import workloads as W


def test_c3_sweep_recipe():
    items = W.c3_sweep()
    assert len(items) == 512
    assert items == W.c3_sweep()
    for a, b in zip(items[0::2], items[1::2]):
        assert (a["L"], a["theta"]) == (b["L"], b["theta"])
        assert (a["wetting"], b["wetting"]) == (W.WET_FORCE, W.WET_GEOM_INTERP)
    Ls = [it["L"] for it in items]
    assert set(Ls) == {64, 128, 256, 512}
    th = np.array([it["theta"] for it in items[0::2]])
    assert th.min() >= 30.0 and th.max() <= W.THETA_MAX
    assert th.min() < 35.0 and th.max() > W.THETA_MAX - 5.0          # the range is spanned


def test_provisional_strength_has_the_angle_sign():
    assert W.provisional_kw(90.0) == 0.0
    for t in (30.0, 60.0, 85.0):
        assert 0.0 < W.provisional_kw(t) <= 0.25
    for t in (95.0, 120.0, 150.0):
        assert -0.25 <= W.provisional_kw(t) < 0.0
    assert W.provisional_kw(10.0) == 0.25 and W.provisional_kw(170.0) == -0.25


def test_c3_lattice_is_a_sessile_drop_of_radius_quarter_L():
    L = 64
    for wet in (W.WET_FORCE, W.WET_GEOM_INTERP):
        wl = W.c3_lattice(dict(L=L, theta=60.0, wetting=wet))
        assert (wl["nx"], wl["ny"], wl["nz"]) == (L, L, 1)
        m = wl["mask"].reshape(L, L)
        assert m[0].all() and m[-1].all() and not m[1:-1].any()
        p = wl["params"]
        C_liquid = (wl["rho"].reshape(L, L) - p["rho_g"]) / (p["rho_l"] - p["rho_g"])
        # a half disc of radius L/4 centred on the wall plane (y = 0.5) above row 0
        area = C_liquid[1:-1].sum()
        assert abs(area / (0.5 * np.pi * (L / 4.0) ** 2) - 1.0) < 0.05, area
        if wet == W.WET_FORCE:
            assert p["kw_rho"] == W.provisional_kw(60.0) > 0.0
        else:
            assert tuple(p["theta_deg"])[:2] == (60.0, 60.0)


def test_c4_default_sizes():
    sig = inspect.signature(W.c4_requests).parameters
    assert sig["n"].default == 256 and sig["rate"].default == 20.0
    assert sig["sizes_2d"].default == (64, 128, 256, 512, 1024)
    assert sig["sizes_3d"].default == (96, 128, 160, 192)


def test_c4_request_mix_recipe():
    reqs = W.c4_requests(sizes_3d=(24, 32))
    assert len(reqs) == 256
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals at 20 per second: mean gap 0.05 s (its standard error over 256 gaps is 6 %)
    assert abs(np.diff(np.concatenate([[0.0], t])).mean() / 0.05 - 1.0) < 0.2
    kinds = {"drop_": 0, "c1_capillary": 0, "c2_lubricated": 0, "lens_": 0, "drop_train_": 0}
    n_ll = n_2d = 0
    for _, wl, steps in reqs:
        name = wl["name"]
        k = max((p for p in kinds if name.startswith(p)), key=len, default=None)    # drop_train_ before drop_
        assert k is not None, name
        kinds[k] += 1
        if wl["lattice"] == W.D3Q27:
            assert 500 <= steps <= 2000
            assert not name.endswith("_ll")
        else:
            assert 1000 <= steps <= 5000
            n_2d += 1
            n_ll += name.endswith("_ll")
        p = wl["params"]
        ratio = p["rho_l"] / p["rho_g"]
        assert 4.0 - 1e-9 <= ratio <= W.RHO_L / W.RHO_G + 1e-9, (name, ratio)
        assert wl["rho"].shape == wl["mask"].shape or wl["rho"].size == wl["mask"].size
    share = {k: v / 256.0 for k, v in kinds.items()}
    want = {"drop_": 0.35, "c1_capillary": 0.2, "c2_lubricated": 0.1, "lens_": 0.15, "drop_train_": 0.2}
    for k in want:
        assert abs(share[k] - want[k]) < 0.08, (k, share)
    assert 0.04 < n_ll / n_2d < 0.25, (n_ll, n_2d)
    again = W.c4_requests(sizes_3d=(24, 32))
    assert [(r[0], r[1]["name"], r[2]) for r in again] == [(r[0], r[1]["name"], r[2]) for r in reqs]


def _concentrations(wl):
    """C1, C2, C3 from (rho, phi) by the inverse of workloads.phase_fields."""
    p = wl["params"]
    C1 = (wl["rho"] - p["rho_l"]) / (p["rho_g"] - p["rho_l"])
    d = wl["phi"] / p["chi"]                      # C2 - C3
    return C1, 0.5 * (1.0 - C1 + d), 0.5 * (1.0 - C1 - d)


def test_c0_recipe():
    """D2Q9 64x64, walls at rows 0 and 63, a liquid-1 cap of radius 16 on the
    bottom wall, U[-1e-3, 1e-3] noise on C2 and C3, force wetting with
    kappa^w = 0; the noise is the seed's."""
    wl = W.c0_sessile_drop()
    assert (wl["nx"], wl["ny"], wl["nz"], wl["lattice"]) == (64, 64, 1, W.D2Q9)
    m = wl["mask"].reshape(64, 64)
    assert m[0].all() and m[63].all() and not m[1:63].any()
    C1, C2, C3 = (c.reshape(64, 64) for c in _concentrations(wl))
    area = C2[1:63].sum()
    assert abs(area / (0.5 * np.pi * 16.0 ** 2) - 1.0) < 0.05, area
    gas = C1[40:63] > 0.99                        # far above the cap
    assert gas.sum() > 1000
    assert np.abs(C3[40:63][gas]).max() <= 1e-3 + 1e-12 and np.abs(C3[40:63][gas]).max() > 5e-4
    assert np.abs(C2[40:63][gas]).max() <= 1e-3 + 1e-12
    p = wl["params"]
    assert p["wetting"] == W.WET_FORCE and p["kw_rho"] == 0.0 and p["kw_phi"] == 0.0
    assert np.array_equal(W.c0_sessile_drop()["rho"], wl["rho"])
    assert not np.array_equal(W.c0_sessile_drop(seed=1)["rho"], wl["rho"])


def test_c1_recipe():
    """D2Q9 1024x64: solid slabs y < 12 and y >= 52 for x in [256, 960) leave a
    channel of height 40; liquid 1 fills x < 256 at full height, gas the rest;
    geometric interpolation with 30/60/120 deg."""
    wl = W.c1_capillary()
    assert (wl["nx"], wl["ny"], wl["lattice"]) == (1024, 64, W.D2Q9)
    m = wl["mask"].reshape(64, 1024)
    y, x = np.mgrid[0:64, 0:1024]
    want = (x >= 256) & (x < 960) & ((y < 12) | (y >= 52))
    assert np.array_equal(m.astype(bool), want)
    assert wl["channel"]["H"] == 40
    C1, C2, C3 = (c.reshape(64, 1024) for c in _concentrations(wl))
    assert C2[:, 20:236].min() > 0.99 and C1[:, 300:940].min() > 0.99
    assert np.abs(C3).max() < 1e-12
    p = wl["params"]
    assert p["wetting"] == W.WET_GEOM_INTERP and tuple(p["theta_deg"]) == (30.0, 60.0, 120.0)


def test_c2_headline_recipe():
    """The bench's headline lattice: D3Q27 192x192x128, walls at z = 0 and 127,
    a liquid-2 film z in [1, 6], a liquid-1 sphere of radius 32 whose bottom
    lies 4 nodes above the film, force wetting with kappa_rho^w = 0.02."""
    import bench

    wl = bench.workload()
    assert (wl["nx"], wl["ny"], wl["nz"], wl["lattice"]) == (192, 192, 128, W.D3Q27)
    m = wl["mask"]
    assert m[0].all() and m[127].all() and not m[1:127].any()
    C1, C2, C3 = _concentrations(wl)
    # the film, away from the drop: its tanh edge (width 2) puts C3 = 1/2 at z = 6.5
    assert C3[1, 10, 10] > 0.99 and C3[6, 10, 10] > 0.5 > C3[7, 10, 10] and C2[3, 10, 10] < 1e-6
    assert C1[60, 10, 10] > 0.99                                 # gas above the film
    assert C2[42, 96, 96] > 0.99                                 # the sphere's centre, z = 6 + 4 + 32
    assert abs(C2[10, 96, 96] - 0.5) < 0.05                     # its bottom, 4 nodes above the film
    p = wl["params"]
    assert p["wetting"] == W.WET_FORCE and p["kw_rho"] == 0.02
