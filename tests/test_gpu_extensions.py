"""GPU (CUDA, sm_103a) vs FP64 oracle on the widened physics: the van der
Waals and Peng-Robinson equations of state in Psi_eos (Sec. II.A names them
as EOS the model hosts) and per-component kinematic viscosities (an
extension; the paper has one beta).  Same normwise bar as the parity tests:
1e-5 after 1000 steps."""
import numpy as np
import pytest

from paper_1904_06881_gb300 import workloads as W

from helpers import gpu_from_workload, normwise, oracle_from_workload, pointwise_rho, record

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _drop(ratio=10.0, **params):
    rho_g = W.RHO_L / ratio
    mask, rho, phi = W.sessile_drop_2d(64, 64, 16.0, xc=32.3, yc=0.5, noise=1e-3, rho_g=rho_g)
    p = W.base_params(rho_g=rho_g, **params)
    return dict(name="drop", lattice=W.D2Q9, nx=64, ny=64, nz=1, mask=mask, rho=rho, phi=phi, params=p)


@pytest.mark.parametrize("eos", [1, 2])
def test_alternative_eos_1000_steps(eos):
    wl = _drop(eos=eos, wetting=W.WET_GEOM_INTERP, theta_deg=(70.0, 70.0, 90.0))
    g, o = gpu_from_workload(wl), oracle_from_workload(wl)
    g.step(1000)
    o.step(1000)
    fg, fo = g.fields(), o.fields()
    e = normwise(fg, fo, o.derived, mask=wl["mask"])
    record("EOS %s drop, ratio 10, 1000 steps" % {1: "van der Waals", 2: "Peng-Robinson"}[eos], normwise=e,
           pointwise_rho=pointwise_rho(fg, fo, wl["mask"]), bound=TOL)
    assert e["rho"] <= TOL and e["phi"] <= TOL and e["C"] <= TOL, e


def _nu_case(lattice, nu):
    if lattice == W.D2Q9:
        return _drop(ratio=W.RHO_L / W.RHO_G, nu=nu, wetting=W.WET_FORCE, kw_rho=0.05)
    wl = W.c2_lubricated(nx=32, ny=32, nz=20, R=7.0, lub=3, gap=2, kw_rho=0.02)
    wl["params"] = dict(wl["params"], nu=nu)
    return wl


@pytest.mark.parametrize("lattice", [W.D2Q9, W.D3Q27])
def test_component_viscosities_one_step(lattice):
    """Viscosities well below the default (0.05, 0.1, 0.03 against 1/6): one
    step from the same populations matches to FP32 rounding."""
    from helpers import match_directions

    wl = _nu_case(lattice, (0.05, 0.1, 0.03))
    g, o = gpu_from_workload(wl), oracle_from_workload(wl)
    g.step(50)
    perm = match_directions(wl["lattice"])
    fg, gg = g.populations()
    o.set_populations(fg[perm], gg[perm])
    g.step(1)
    o.step(1)
    fg, gg = g.populations()
    fo, go = o.populations()
    fl = wl["mask"].reshape(-1) == 0
    err = np.abs(fg[perm][:, fl] - fo[:, fl]).max() / np.abs(fo[:, fl]).max()
    record("per-component viscosity %s, one step" % ("D2Q9" if lattice == W.D2Q9 else "D3Q27"),
           max_rel_population_err=err, bound=3e-6)
    assert err <= 3e-6, err


@pytest.mark.parametrize("lattice", [W.D2Q9, W.D3Q27])
def test_component_viscosities_1000_steps(lattice):
    """1000 steps with viscosities around the default (0.12, 1/6, 0.25);
    lower ones make the drop's currents grow and amplify rounding."""
    wl = _nu_case(lattice, (0.12, 1.0 / 6.0, 0.25))
    g, o = gpu_from_workload(wl), oracle_from_workload(wl)
    g.step(1000)
    o.step(1000)
    fg, fo = g.fields(), o.fields()
    e = normwise(fg, fo, o.derived, mask=wl["mask"])
    record("per-component viscosity %s, 1000 steps" % ("D2Q9" if lattice == W.D2Q9 else "D3Q27"), normwise=e,
           pointwise_rho=pointwise_rho(fg, fo, wl["mask"]), bound=TOL)
    assert e["rho"] <= TOL and e["phi"] <= TOL and e["C"] <= TOL, e
