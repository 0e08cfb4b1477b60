"""The bounds-checked build (built with -DTLB_BOUNDS_CHECK): every global node
index that the step, moment and ghost kernels compute for a neighbour, a halo
or an extrapolation/interpolation stencil is tested against the lattice
size; one outside it is recorded (and the access skipped), and tlb_sync then
returns TLB_E_BOUNDS.  This stands in for a memory checker, which this GPU
pool does not offer.

The cases cover the index arithmetic's corners: lattices smaller than a tile
and ragged ones, every wetting mode, both lattices, FP16 g storage, a batch
of uneven lattices with a launch large enough for the 64-register build of
the D2Q9 step kernel, and the full-size capillary channel and lubricated
drop.  They run in a child process that loads the checked library
(TLB_LIBRARY); each must report no violation and give fields bit-identical
to the normal build's (the check changes no arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1904_06881_gb300 import workloads as W  # noqa: E402

STEPS = 60


def _cap(lattice, nx, ny, nz, wet, R, g_fp16=0):
    """Liquid-1 cap of radius R on a solid bottom (and top) plane, gas around,
    its centre off the lattice nodes."""
    if lattice == W.D2Q9:
        mask, rho, phi = W.sessile_drop_2d(nx, ny, R, xc=nx / 2 + 0.3, noise=1e-3, seed=5)
    else:
        z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
        C2 = 0.5 * (1.0 - np.tanh((np.sqrt((x - nx / 2 - 0.31) ** 2 + (y - ny / 2 - 0.17) ** 2 + (z - 0.5) ** 2)
                                   - R) / 2.0))
        rho, phi = W.phase_fields(C2, np.zeros_like(C2))
        mask = np.zeros((nz, ny, nx), np.uint8)
        mask[0] = 1
        mask[nz - 1] = 1
    params = (W.base_params(wetting=wet, kw_rho=0.05) if wet == W.WET_FORCE
              else W.base_params(wetting=wet, theta_deg=(60.0, 60.0, 120.0)))
    params["g_fp16"] = g_fp16
    return dict(lattice=lattice, nx=nx, ny=ny, nz=nz, params=params, mask=mask, rho=rho, phi=phi)


def _cases():
    """(name, list of workloads stepped together) pairs."""
    c = []
    for wet in (W.WET_FORCE, W.WET_GEOM_EXTRAP, W.WET_GEOM_INTERP):
        c.append(("d2_tiny_%d" % wet, [_cap(W.D2Q9, 3, 5, 1, wet, 1.0)]))
        c.append(("d2_ragged_%d" % wet, [_cap(W.D2Q9, 37, 23, 1, wet, 6.0)]))
        c.append(("d3_tiny_%d" % wet, [_cap(W.D3Q27, 6, 5, 5, wet, 2.5)]))
        c.append(("d3_ragged_%d" % wet, [_cap(W.D3Q27, 19, 13, 11, wet, 4.0)]))
    c.append(("d2_ragged_fp16", [_cap(W.D2Q9, 37, 23, 1, W.WET_GEOM_INTERP, 6.0, g_fp16=1)]))
    c.append(("d3_ragged_fp16", [_cap(W.D3Q27, 19, 13, 11, W.WET_GEOM_INTERP, 4.0, g_fp16=1)]))
    periodic = W.big_periodic_drop_3d(n=20)
    c.append(("d3_periodic", [periodic]))
    c.append(("d2_batch_large_launch", [W.c3_lattice(dict(L=64, theta=45.0, wetting=W.WET_GEOM_INTERP)),
                                        _cap(W.D2Q9, 37, 23, 1, W.WET_FORCE, 6.0),
                                        W.c3_lattice(dict(L=512, theta=60.0, wetting=W.WET_GEOM_EXTRAP))]))
    c.append(("d3_batch", [_cap(W.D3Q27, 19, 13, 11, W.WET_GEOM_EXTRAP, 4.0),
                           _cap(W.D3Q27, 6, 5, 5, W.WET_FORCE, 2.5)]))
    c.append(("c1_capillary", [W.c1_capillary()]))
    c.append(("c2_lubricated", [W.c2_lubricated(kw_rho=0.02)]))
    return c


def run_cases(out_path):
    """Step every case with whatever library the binding loads; write the
    fields and each case's tlb_sync status to out_path (npz)."""
    from paper_1904_06881_gb300 import tlb

    res = {}
    for name, wls in _cases():
        lats = [tlb.lattice_from_workload(wl) for wl in wls]
        if len(lats) == 1:
            lats[0].step(STEPS)
        else:
            tlb.tlb_step_batch([x.h for x in lats], STEPS)
        for k, x in enumerate(lats):
            st = tlb.lib().tlb_sync(x.h)
            res["%s/%d/status" % (name, k)] = np.array(st)
            if st == 0:
                fl = x.fields()
                res["%s/%d/rho" % (name, k)] = fl["rho"]
                res["%s/%d/phi" % (name, k)] = fl["phi"]
            x.close()
    np.savez(out_path, **res)


@pytest.mark.gpu
def test_checked_build_flags_nothing_and_changes_nothing(tmp_path):
    from paper_1904_06881_gb300 import build as B

    checked = B.build(check=True)
    out_c, out_n = str(tmp_path / "checked.npz"), str(tmp_path / "normal.npz")
    env = dict(os.environ, TLB_LIBRARY=checked)
    subprocess.run([sys.executable, os.path.abspath(__file__), out_c], env=env, cwd=ROOT, check=True, timeout=900)
    env = {k: v for k, v in os.environ.items() if k != "TLB_LIBRARY"}
    subprocess.run([sys.executable, os.path.abspath(__file__), out_n], env=env, cwd=ROOT, check=True, timeout=900)
    c, n = np.load(out_c), np.load(out_n)
    status = [k for k in c.files if k.endswith("/status")]
    assert len(status) == sum(len(w) for _, w in _cases())
    bad = {k: int(c[k]) for k in status if int(c[k]) != 0}
    assert not bad, bad                        # -10: TLB_E_BOUNDS
    assert sorted(c.files) == sorted(n.files)
    diff = [k for k in c.files if not np.array_equal(c[k], n[k])]
    assert not diff, diff


if __name__ == "__main__":
    run_cases(sys.argv[1])
