"""CPU-side checks of the C ABI library: it loads without a GPU and exports
every entry point that include/tlb.h declares; host-only calls behave."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1904_06881_gb300 import build, tlb

    build.build()
    return tlb.lib()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "tlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tlb_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_1904_06881_gb300 import tlb

    assert declared_entry_points() == sorted(tlb.ENTRY_POINTS)


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_entry_points() if not hasattr(L, n)]
    assert not missing


def test_host_only_calls(L):
    from paper_1904_06881_gb300 import tlb

    assert L.tlb_strerror(-6) == b"non-positive density or population"
    maj, mnr, sm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.tlb_version(ctypes.byref(maj), ctypes.byref(mnr), ctypes.byref(sm)) == 0 and sm.value == 103
    p = tlb.tlb_params_default()
    assert p.lam[0] == 0.6 and p.kappa[1] == 1.0 and p.beta == 0.5 and p.chi == 5.0
    c, w = tlb.tlb_lattice_directions(tlb.D3Q27)
    assert np.isclose(w.sum(), 1.0) and (c.sum(0) == 0).all()
    # opposite directions come in (+c, -c) pairs after the rest direction
    assert (c[1::2] == -c[2::2]).all()


def test_invalid_arguments_rejected_on_host(L):
    from paper_1904_06881_gb300 import tlb

    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_create(tlb.D2Q9, 64, 64, 1, (1.0, 1e-3), (0.01, 1, 1), (0.1, -0.2, 0.1), tlb.WET_FORCE, (90, 90, 90))
    assert e.value.code == -1          # a non-positive viscosity
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_derive(tlb.make_params(tlb.D2Q9, 64, 64, 1, eos=7))
    assert e.value.code == -1          # unknown equation of state
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_create(tlb.D2Q9, 64, 64, 1, (1.0, 1e-3), (0.01, 1, 1), (1 / 6,) * 3, tlb.WET_FORCE, (60, 90, 90))
    assert e.value.code == -5          # force wetting: no calibration table for this parameter set
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_create(tlb.D2Q9, 2, 64, 1, (1.0, 1e-3), (0.01, 1, 1), (1 / 6,) * 3, tlb.WET_FORCE, (90, 90, 90))
    assert e.value.code == -1
    p = tlb.make_params(tlb.D2Q9, 64, 64, 1, wetting=tlb.WET_GEOM_INTERP, theta_deg=(10, 90, 90))
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_create_ex(p)
    assert e.value.code == -4          # geometric angles limited to [20, 160] deg
    import ctypes
    assert L.tlb_server_set_policy(None, tlb.SCHED_SHORTEST, ctypes.c_double(0.0)) == -1   # null server


@pytest.mark.parametrize("variant", ["check", "timeout_test"])
def test_test_builds_compile_and_export_the_same_symbols(variant):
    """The bounds-checked and the timeout test builds (loaded by the GPU
    tests through TLB_LIBRARY) compile here and export every declared entry
    point; they report their own error codes by name."""
    import subprocess
    import sys

    from paper_1904_06881_gb300 import build

    path = build.build(**{variant: True})
    code = ("import ctypes, sys; L = ctypes.CDLL(sys.argv[1]); names = sys.argv[2:]; "
            "missing = [n for n in names if not hasattr(L, n)]; "
            "L.tlb_strerror.restype = ctypes.c_char_p; "
            "print(missing, L.tlb_strerror(-10).decode(), L.tlb_strerror(-7).decode())")
    out = subprocess.run([sys.executable, "-c", code, path] + declared_entry_points(), capture_output=True,
                         text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "[] index outside its array (bounds-checked build) device wait timed out", out.stdout


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the compiled library the binding raises on
    first use (here: TLB_LIBRARY pointing at a file that does not exist)."""
    import subprocess
    import sys

    code = ("from paper_1904_06881_gb300 import tlb\n"
            "try:\n    tlb.Lattice(tlb.D2Q9, 16, 16, 1)\nexcept RuntimeError as e:\n    print('RAISED', e)\n")
    env = dict(os.environ, TLB_LIBRARY=str(tmp_path / "absent" / "libtlb.so"))
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("RAISED libtlb.so not built"), out.stdout


@pytest.mark.parametrize("eos", [0, 1, 2])
@pytest.mark.parametrize("ratio", [10.0, 14.141345641130298, 40.0])
def test_derived_constants_match_oracle(L, eos, ratio):
    """The library's host EOS code (closed-form textbook pressures and
    chemical potentials, a search over ln rho_g) and the oracle's (pressure
    p = rho Psi' - Psi, bisection on the common pressure) give the same
    temperature, coexistence densities and Psi_eos constants for the
    Carnahan-Starling, van der Waals and Peng-Robinson equations of state."""
    import oracle
    from paper_1904_06881_gb300 import tlb

    rho_l = 6.143914427184784
    p = tlb.make_params(tlb.D2Q9, 16, 16, 1, rho_l=rho_l, rho_g=rho_l / ratio, eos=eos)
    d = tlb.tlb_derive(p)
    o = oracle.Oracle(nx=16, ny=16, rho_l=rho_l, rho_g=rho_l / ratio, eos=eos).derived
    # the oracle's critical point comes from a scan of a finite-difference
    # dp/drho (5e-8 relative for vdW against the exact 8a/(27bR))
    for k in ("T", "Tc", "a", "b", "rho_l", "rho_g"):
        assert np.isclose(d[k], o[k], rtol=1e-6, atol=0), (k, d[k], o[k])
    for k in ("C", "Psi0"):
        assert np.isclose(d[k], o[k], rtol=1e-5, atol=1e-9), (k, d[k], o[k])


def test_committed_counters_match_the_kernel_sources():
    """The ncu counters in profiles/traffic.json (the bench line's `traffic`
    and `issue` figures) were taken on the device code as committed: their
    recorded source hash equals the hash of the current kernel sources, and
    every workload they cover has a committed summary."""
    import json
    import os

    import bench

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    assert d["source_sha256"] == bench.kernel_source_hash()
    for name, path in d["captures"].items():
        assert name in d["traffic_bytes_per_launch"] and name in d["warp_instructions_per_launch"]
        assert os.path.exists(os.path.join(root, path)), path
