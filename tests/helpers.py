"""Shared helpers of the GPU parity tests: the same seeded workload fed to the
CUDA library (through the C ABI) and to the FP64 oracle."""
import numpy as np

import oracle


def oracle_from_workload(wl, **over):
    return oracle.from_workload(wl, **over)


def gpu_from_workload(wl, **over):
    from paper_1904_06881_gb300 import tlb

    return tlb.lattice_from_workload(wl, **over)


def normwise(fg, fo, derived, chi=5.0, mask=None):
    """Normwise field errors (densities over rho_l - rho_g, phi over chi,
    concentrations absolute) on fluid nodes."""
    fl = np.ones(fg["rho"].shape, bool) if mask is None else (mask == 0)
    drho = derived["rho_l"] - derived["rho_g"]
    return dict(rho=np.abs(fg["rho"] - fo["rho"])[fl].max() / drho,
                phi=np.abs(fg["phi"] - fo["phi"])[fl].max() / chi,
                C=max(np.abs(fg["C"][k] - fo["C"][k])[fl].max() for k in range(3)))


def match_directions(lattice):
    """Permutation p with gpu_direction[p[i]] == oracle_direction[i]."""
    from paper_1904_06881_gb300 import tlb

    cg, _ = tlb.tlb_lattice_directions(lattice)
    co, _ = oracle.lattice(lattice)
    return np.array([int(np.where((cg == co[i]).all(1))[0][0]) for i in range(len(co))])
