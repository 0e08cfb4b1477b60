"""The allocation-free entry point tlb_step_noalloc gives the same populations
as the regular context API (tlb_step), bit for bit (it runs the same kernels
on a tile table of its own), on two calls in a row.

tlb_step_noalloc serves callers that cannot allocate device memory while they
run (a fixed device-memory budget carved up in advance, a framework's memory
pool that a raw cudaMalloc would bypass, a loop that cannot take the
synchronisation an allocation may imply); its scratch is a static device
array inside the library.  The cases cover geometric wetting (D2Q9 channel),
force wetting given by contact angles only, whose strengths come from the
registered calibration tables exactly as for a context, a small D3Q27
lattice, and two masks in turn (the node flags and tile table kept from the
previous call are reused only for the same geometry).

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
"""
import json

import numpy as np
import pytest

from paper_1904_06881_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fp32_weights(c, D):
    """The lattice weights as the library forms them in FP32: the product over
    the D axes of 2/3 (c = 0) and 1/6 (c = +-1), each factor and product
    rounded to single precision.  The library stores f - w_i in FP32 and
    reports f as that value plus these weights, so this converts both ways
    without rounding."""
    two3, one6 = np.float32(2.0) / np.float32(3.0), np.float32(1.0) / np.float32(6.0)
    out = []
    for ci in c:
        wv = np.float32(1.0)
        for a in range(D):
            wv = np.float32(wv * (two3 if ci[a] == 0 else one6))
        out.append(float(wv))
    return np.array(out)


def _compare(wl, nsteps):
    import torch

    from paper_1904_06881_gb300 import tlb

    ref = tlb.lattice_from_workload(wl)
    c, _ = tlb.tlb_lattice_directions(wl["lattice"])
    w = _fp32_weights(c, 2 if wl["lattice"] == W.D2Q9 else 3)
    f0, g0 = ref.populations()                      # FP64, library direction order
    dev = torch.device("cuda")
    f = torch.tensor((f0 - w[:, None]).astype(np.float32), device=dev)
    g = torch.tensor(g0.astype(np.float32), device=dev)
    f_tmp, g_tmp = torch.empty_like(f), torch.empty_like(g)
    p = tlb.make_params(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], **wl["params"])
    stream = torch.cuda.current_stream().cuda_stream
    fl = wl["mask"].reshape(-1) == 0
    for call in range(2):                           # two calls in a row: the scratch is reused
        tlb.tlb_step_noalloc(p, wl["mask"], f.data_ptr(), f_tmp.data_ptr(), g.data_ptr(), g_tmp.data_ptr(),
                             nsteps, stream)
        ref.step(nsteps)
        torch.cuda.synchronize()
        fr, gr = ref.populations()
        fn = f.double().cpu().numpy() + w[:, None]
        gn = g.double().cpu().numpy()
        # the kernels of tlb_step on the same inputs: bit-identical populations
        assert np.array_equal(fn[:, fl], fr[:, fl]), (call, np.abs(fn[:, fl] - fr[:, fl]).max())
        assert np.array_equal(gn[:, fl], gr[:, fl]), (call, np.abs(gn[:, fl] - gr[:, fl]).max())


def test_step_noalloc_matches_context_steps():
    _compare(W.c1_capillary(wetting=W.WET_GEOM_INTERP), 7)


def _table_angle(lattice):
    from paper_1904_06881_gb300 import tlb

    with open(tlb.CALIBRATION_PATH) as fh:
        tabs = [t for t in json.load(fh)["tables"] if t["lattice"] == lattice]
    th = tabs[0]["theta_deg"]
    return 0.5 * (th[0] + th[-1])                   # inside the calibrated range


def test_step_noalloc_force_wetting_by_angles():
    """Force wetting given by angles only (kappa^w = 0): both entry points map
    the angles through the same calibration table."""
    th = _table_angle(W.D2Q9)
    mask, rho, phi = W.sessile_drop_2d(64, 48, 14.0, xc=30.3, yc=0.5)
    wl = dict(lattice=W.D2Q9, nx=64, ny=48, nz=1, mask=mask, rho=rho, phi=phi,
              params=W.base_params(wetting=W.WET_FORCE, theta_deg=(th, th, 90.0)))
    _compare(wl, 5)


def test_step_noalloc_d3q27():
    th = _table_angle(W.D3Q27)
    wl = W.c2_lubricated(nx=24, ny=20, nz=20, R=5.0, lub=3, gap=2)
    wl["params"] = W.base_params(wetting=W.WET_FORCE, theta_deg=(90.0, th, 90.0))
    _compare(wl, 3)


def test_step_noalloc_reuses_and_rebuilds_the_geometry():
    """Two lattices of the same type and size whose masks differ (a wall
    below; walls below and above), stepped in the order A, B, A, A on one
    stream: the node flags and tile table are reused for the repeated A and
    rebuilt at each change of mask, and every call matches its context."""
    import torch

    from paper_1904_06881_gb300 import tlb

    nx, ny = 64, 48
    mask_a, rho, phi = W.sessile_drop_2d(nx, ny, 14.0, xc=30.3, yc=0.5, walls=("bottom",))
    mask_b = mask_a.copy()
    mask_b[..., ny - 1, :] = 1
    params = W.base_params(wetting=W.WET_GEOM_INTERP, theta_deg=(60.0, 60.0, 120.0))
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    state = {}
    for name, mask in (("A", mask_a), ("B", mask_b)):
        wl = dict(lattice=W.D2Q9, nx=nx, ny=ny, nz=1, mask=mask, rho=rho, phi=phi, params=params)
        ref = tlb.lattice_from_workload(wl)
        c, _ = tlb.tlb_lattice_directions(W.D2Q9)
        w = _fp32_weights(c, 2)
        f0, g0 = ref.populations()
        f = torch.tensor((f0 - w[:, None]).astype(np.float32), device=dev)
        g = torch.tensor(g0.astype(np.float32), device=dev)
        state[name] = (wl, ref, w, f, g, torch.empty_like(f), torch.empty_like(g))
    p = tlb.make_params(W.D2Q9, nx, ny, 1, **params)
    for name in ("A", "B", "A", "A"):
        wl, ref, w, f, g, f_tmp, g_tmp = state[name]
        tlb.tlb_step_noalloc(p, wl["mask"], f.data_ptr(), f_tmp.data_ptr(), g.data_ptr(), g_tmp.data_ptr(), 4,
                             stream)
        ref.step(4)
        torch.cuda.synchronize()
        fr, gr = ref.populations()
        fl = wl["mask"].reshape(-1) == 0
        fn = f.double().cpu().numpy() + w[:, None]
        gn = g.double().cpu().numpy()
        assert np.array_equal(fn[:, fl], fr[:, fl]), (name, np.abs(fn[:, fl] - fr[:, fl]).max())
        assert np.array_equal(gn[:, fl], gr[:, fl]), (name, np.abs(gn[:, fl] - gr[:, fl]).max())


def test_step_noalloc_rejects_oversize_lattice():
    from paper_1904_06881_gb300 import tlb

    p = tlb.make_params(tlb.D2Q9, 2048, 1024, 1)
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_step_noalloc(p, None, 1, 1, 1, 1, 1)
    assert e.value.code == -1
