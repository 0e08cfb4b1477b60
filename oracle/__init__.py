"""FP64 CPU oracle of the ternary free-energy ELBM update (arXiv:1904.06881).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow restatement of the
paper's equations in C (``tlbo.c``), loaded here through ctypes.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never does, and the
two share no code.

Parity pins that constrain each part are in ``tests/test_oracle_*.py`` and
``tests/test_golden_cpu.py`` (values the paper prints, ``tests/golden/``).
Parts with no pin beyond the oracle's own consistency ("parity unpinned"):
the tie-break of the 3D interpolation support (Sec. IV.B, Eq. interp3D) when
two corners lie equally near (i, j), and the weights of the corner/wedge
ghost average (its mirror symmetry is pinned, which any symmetric
combination of the single-axis values keeps).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtlbo.so")
_lib = None

D2Q9, D3Q27 = 0, 1
WET_FORCE, WET_GEOM_EXTRAP, WET_GEOM_INTERP = 0, 1, 2


def build(force=False):
    """Compile tlbo.c into oracle/_build/libtlbo.so with gcc (OpenMP)."""
    src = os.path.join(_HERE, "tlbo.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                   os.path.getmtime(os.path.join(_HERE, "tlbo.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("lam", ctypes.c_double * 3), ("kappa", ctypes.c_double * 3),
                ("chi", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("R", ctypes.c_double), ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
                ("beta", ctypes.c_double), ("tau_g", ctypes.c_double), ("Gamma", ctypes.c_double),
                ("wetting", ctypes.c_int), ("theta_deg", ctypes.c_double * 3),
                ("kw_rho", ctypes.c_double), ("kw_phi", ctypes.c_double), ("eos", ctypes.c_int),
                ("omega", ctypes.c_double), ("nu", ctypes.c_double * 3)]


class Derived(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("T", "a", "b", "R", "rho_l", "rho_g", "C", "Psi0", "Tc",
                 "kappa_rr", "kappa_pp", "kappa_rp")]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.tlbo_eos_critical_T.restype = d
        L.tlbo_eos_critical_T.argtypes = [d, d, d]
        L.tlbo_eos_coexistence.argtypes = [d, d, d, d, dp]
        L.tlbo_eos_psi.restype = d
        L.tlbo_eos_psi.argtypes = [d, d, d, d, d, d]
        L.tlbo_eos_dpsi.restype = d
        L.tlbo_eos_dpsi.argtypes = [d, d, d, d, d, d]
        for name in ("tlbo_eos_psi_k", "tlbo_eos_dpsi_k"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [i, d, d, d, d, d, d, d]
        L.tlbo_eos_p_k.restype = d
        L.tlbo_eos_p_k.argtypes = [i, d, d, d, d, d, d]
        L.tlbo_eos_critical_T_k.restype = d
        L.tlbo_eos_critical_T_k.argtypes = [i, d, d, d, d]
        L.tlbo_eos_coexistence_k.argtypes = [i, d, d, d, d, d, dp]
        L.tlbo_lattice.argtypes = [i, ctypes.POINTER(ctypes.c_int), dp]
        L.tlbo_feq.argtypes = [i, d, dp, dp]
        L.tlbo_entropy.restype = d
        L.tlbo_entropy.argtypes = [i, dp]
        L.tlbo_alpha.restype = d
        L.tlbo_alpha.argtypes = [i, dp, dp, ctypes.POINTER(ctypes.c_int)]
        L.tlbo_geq.argtypes = [i, d, dp, d, d, dp]
        L.tlbo_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(p)]
        L.tlbo_destroy.argtypes = [p]
        L.tlbo_get_derived.argtypes = [p, ctypes.POINTER(Derived)]
        L.tlbo_set_solid.argtypes = [p, ctypes.POINTER(ctypes.c_uint8)]
        L.tlbo_init_fields.argtypes = [p, dp, dp, dp]
        L.tlbo_step.argtypes = [p, i]
        L.tlbo_get_fields.argtypes = [p, dp, dp, dp, dp]
        L.tlbo_get_populations.argtypes = [p, dp, dp]
        L.tlbo_set_populations.argtypes = [p, dp, dp]
        L.tlbo_get_aux.argtypes = [p, i, dp]
        L.tlbo_diagnostics.argtypes = [p, dp]
        L.tlbo_alpha_clipped.restype = ctypes.c_long
        L.tlbo_alpha_clipped.argtypes = [p]
        L.tlbo_threads.restype = i
        L.tlbo_threads.argtypes = [i]
        _lib = L
    return _lib


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads(n=0):
    """Set the oracle's host thread count (n > 0); returns the count in use."""
    return lib().tlbo_threads(int(n))


# ---- thermodynamics and single-node kinetics -------------------------------
def eos_critical_T(a, b, R=1.0):
    return lib().tlbo_eos_critical_T(a, b, R)


def eos_coexistence(a, b, R, T):
    out = np.zeros(4)
    rc = lib().tlbo_eos_coexistence(a, b, R, T, _dptr(out))
    if rc != 0:
        raise ValueError("no coexistence at T=%g" % T)
    return dict(rho_g=out[0], rho_l=out[1], C=out[2], Psi0=out[3])


EOS_CS, EOS_VDW, EOS_PR = 0, 1, 2


def eos_k(kind, omega=0.344):
    """Functions of the equation of state `kind` (EOS_*): psi, dpsi, p,
    critical_T, coexistence (same arguments as the Carnahan-Starling ones)."""
    L = lib()

    def coexistence(a, b, R, T):
        out = np.zeros(4)
        if L.tlbo_eos_coexistence_k(kind, omega, a, b, R, T, _dptr(out)) != 0:
            raise ValueError("no coexistence at T=%g" % T)
        return dict(rho_g=out[0], rho_l=out[1], C=out[2], Psi0=out[3])

    return dict(psi=lambda r, a, b, R, T, C: L.tlbo_eos_psi_k(kind, omega, r, a, b, R, T, C),
                dpsi=lambda r, a, b, R, T, C: L.tlbo_eos_dpsi_k(kind, omega, r, a, b, R, T, C),
                p=lambda r, a, b, R, T: L.tlbo_eos_p_k(kind, omega, r, a, b, R, T),
                critical_T=lambda a, b, R=1.0: L.tlbo_eos_critical_T_k(kind, omega, a, b, R),
                coexistence=coexistence)


def eos_psi(rho, a, b, R, T, C):
    return lib().tlbo_eos_psi(rho, a, b, R, T, C)


def eos_dpsi(rho, a, b, R, T, C):
    return lib().tlbo_eos_dpsi(rho, a, b, R, T, C)


def lattice(lat):
    Q = 27 if lat == D3Q27 else 9
    c = np.zeros(Q * 3, dtype=np.int32)
    w = np.zeros(Q)
    lib().tlbo_lattice(lat, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(w))
    return c.reshape(Q, 3), w


def feq(lat, rho, u):
    Q = 27 if lat == D3Q27 else 9
    out = np.zeros(Q)
    lib().tlbo_feq(lat, rho, _dptr(np.ascontiguousarray(u, dtype=np.float64)), _dptr(out))
    return out


def entropy(lat, f):
    return lib().tlbo_entropy(lat, _dptr(np.ascontiguousarray(f, dtype=np.float64)))


def alpha(lat, fp, delta):
    st = ctypes.c_int(0)
    a = lib().tlbo_alpha(lat, _dptr(np.ascontiguousarray(fp, dtype=np.float64)),
                         _dptr(np.ascontiguousarray(delta, dtype=np.float64)), ctypes.byref(st))
    return a, st.value


def geq(lat, phi, v, mu_phi, Gamma=1.0):
    Q = 27 if lat == D3Q27 else 9
    out = np.zeros(Q)
    lib().tlbo_geq(lat, phi, _dptr(np.ascontiguousarray(v, dtype=np.float64)), mu_phi, Gamma,
                   _dptr(out))
    return out


# ---- simulation context -----------------------------------------------------
AUX = dict(p0=0, mu_rho=1, mu_phi=2, Fx=3, Fy=4, Fz=5, Pxx=6, Pyy=7, Pzz=8, Pxy=9, Pxz=10,
           Pyz=11, rho_ghost=12, phi_ghost=13)


class Oracle:
    """One lattice advanced by the FP64 oracle.  Arrays are numpy, x fastest."""

    def __init__(self, lattice=D2Q9, nx=64, ny=64, nz=1, lam=(0.6, 1.0, 1.0),
                 kappa=(0.01, 1.0, 1.0), chi=5.0, a=0.037, b=0.2, R=1.0, rho_l=1.0,
                 rho_g=1e-3, beta=0.5, tau_g=1.0, Gamma=1.0, wetting=WET_FORCE,
                 theta_deg=(90.0, 90.0, 90.0), kw_rho=0.0, kw_phi=0.0, eos=0, omega=0.344,
                 nu=(0.0, 0.0, 0.0)):
        p = Params()
        p.lattice, p.nx, p.ny, p.nz = lattice, nx, ny, nz
        p.lam[:] = list(lam)
        p.kappa[:] = list(kappa)
        p.chi, p.a, p.b, p.R = chi, a, b, R
        p.rho_l, p.rho_g = rho_l, rho_g
        p.beta, p.tau_g, p.Gamma = beta, tau_g, Gamma
        p.wetting = wetting
        p.theta_deg[:] = list(theta_deg)
        p.kw_rho, p.kw_phi = kw_rho, kw_phi
        p.eos, p.omega = eos, omega
        p.nu[:] = list(nu)
        self.params = p
        self.lattice = lattice
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.D = 3 if lattice == D3Q27 else 2
        self.Q = 27 if lattice == D3Q27 else 9
        h = ctypes.c_void_p()
        rc = lib().tlbo_create(ctypes.byref(p), ctypes.byref(h))
        if rc != 0:
            raise ValueError("tlbo_create failed (%d)" % rc)
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.tlbo_destroy(h)
            self._h = None

    @property
    def derived(self):
        d = Derived()
        lib().tlbo_get_derived(self._h, ctypes.byref(d))
        return {k: getattr(d, k) for k, _ in Derived._fields_}

    def set_solid(self, mask):
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        assert m.size == self.N
        lib().tlbo_set_solid(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))

    def init_fields(self, rho, phi, u=None):
        r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        ph = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        lib().tlbo_init_fields(self._h, _dptr(r), _dptr(ph), _dptr(uu))

    def step(self, n=1):
        rc = lib().tlbo_step(self._h, int(n))
        if rc != 0:
            raise FloatingPointError("oracle step failed (%d): non-positive population" % rc)

    def fields(self):
        N = self.N
        rho, phi = np.zeros(N), np.zeros(N)
        u, C = np.zeros(self.D * N), np.zeros(3 * N)
        lib().tlbo_get_fields(self._h, _dptr(rho), _dptr(phi), _dptr(u), _dptr(C))
        s = self.shape
        return dict(rho=rho.reshape(s), phi=phi.reshape(s), u=u.reshape((self.D,) + s),
                    C=C.reshape((3,) + s))

    def populations(self):
        f, g = np.zeros(self.Q * self.N), np.zeros(self.Q * self.N)
        lib().tlbo_get_populations(self._h, _dptr(f), _dptr(g))
        return f.reshape(self.Q, self.N), g.reshape(self.Q, self.N)

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        lib().tlbo_set_populations(self._h, _dptr(f), _dptr(g))

    def aux(self, name):
        out = np.zeros(self.N)
        lib().tlbo_get_aux(self._h, AUX[name], _dptr(out))
        return out.reshape(self.shape)

    def diagnostics(self):
        out = np.zeros(6)
        lib().tlbo_diagnostics(self._h, _dptr(out))
        return dict(mass_rho=out[0], mass_phi=out[1], C1=out[2], C2=out[3], C3=out[4],
                    kinetic=out[5])

    @property
    def alpha_clipped(self):
        return lib().tlbo_alpha_clipped(self._h)


def from_workload(wl, **over):
    """Oracle lattice with the mask and initial fields of a workloads.* dict."""
    p = dict(wl["params"])
    p.update(over)
    o = Oracle(lattice=wl["lattice"], nx=wl["nx"], ny=wl["ny"], nz=wl["nz"], lam=p["lam"], kappa=p["kappa"],
               chi=p["chi"], a=p["a"], b=p["b"], R=p["R"], rho_l=p["rho_l"], rho_g=p["rho_g"], beta=p["beta"],
               tau_g=p["tau_g"], Gamma=p["Gamma"], wetting=p["wetting"], theta_deg=p["theta_deg"],
               kw_rho=p["kw_rho"], kw_phi=p["kw_phi"], eos=p.get("eos", 0), omega=p.get("omega", 0.344),
               nu=p.get("nu", (0.0, 0.0, 0.0)))
    o.set_solid(wl["mask"])
    o.init_fields(wl["rho"], wl["phi"])
    return o
