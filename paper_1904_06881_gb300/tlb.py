"""Python binding of the C ABI in include/tlb.h (argument marshalling only).

Every function here has the name of the C entry point it calls; all work is
done by libtlb.so (CUDA kernels for sm_103a).  There is no CPU fallback: if
the library has not been built, ``lib()`` raises.

``Lattice`` wraps a context for numpy users.  ``use_torch_allocator()`` routes
the library's device allocations through PyTorch's caching allocator.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TLB_LIBRARY selects another build of the same library (the bounds-checked
# one, build(check=True)); it must export the same entry points
LIB_PATH = os.environ.get("TLB_LIBRARY") or os.path.join(_HERE, "_build", "libtlb.so")

TLB_OK = 0
ERRORS = {-1: "TLB_E_INVAL", -2: "TLB_E_NOMEM", -3: "TLB_E_CUDA", -4: "TLB_E_UNSUPPORTED",
          -5: "TLB_E_UNCALIBRATED", -6: "TLB_E_DIVERGED", -7: "TLB_E_TIMEOUT", -8: "TLB_E_BUSY",
          -9: "TLB_E_NOTFOUND", -10: "TLB_E_BOUNDS"}
D2Q9, D3Q27 = 0, 1
EOS_CS, EOS_VDW, EOS_PR = 0, 1, 2
WET_FORCE, WET_GEOM_EXTRAP, WET_GEOM_INTERP = 0, 1, 2
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3

# names of every entry point declared in include/tlb.h
ENTRY_POINTS = (
    "tlb_strerror", "tlb_last_error_message", "tlb_version", "tlb_set_allocator", "tlb_params_default",
    "tlb_create", "tlb_create_ex", "tlb_destroy", "tlb_get_params", "tlb_get_derived", "tlb_set_stream",
    "tlb_set_solid", "tlb_init_fields", "tlb_init_fields_device", "tlb_step", "tlb_step_phase", "tlb_sync", "tlb_get_fields",
    "tlb_get_fields_device", "tlb_diagnostics", "tlb_get_aux", "tlb_get_populations", "tlb_set_populations",
    "tlb_lattice_directions", "tlb_snapshot_bytes", "tlb_snapshot", "tlb_restore", "tlb_steps_done",
    "tlb_device_bytes", "tlb_launch_count", "tlb_step_batch", "tlb_server_create", "tlb_submit",
    "tlb_server_pump", "tlb_poll", "tlb_server_stats", "tlb_server_destroy", "tlb_step_noalloc",
    "tlb_set_force_calibration", "tlb_batch_create", "tlb_batch_step", "tlb_batch_tune", "tlb_batch_get_config",
    "tlb_batch_destroy", "tlb_derive", "tlb_server_set_policy",
)
SCHED_FIFO, SCHED_SHORTEST = 0, 1
ORDER_LATTICE, ORDER_INTERLEAVED, ORDER_LARGEST_FIRST = 0, 1, 2


class TlbError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = ""
        if _lib is not None:
            msg = _lib.tlb_last_error_message().decode()
        super().__init__("%s failed: %s (%s)" % (where, ERRORS.get(code, code), msg))


class Params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lam", ctypes.c_double * 3), ("kappa", ctypes.c_double * 3), ("chi", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
                ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double), ("beta", ctypes.c_double),
                ("tau_g", ctypes.c_double), ("Gamma", ctypes.c_double), ("wetting", ctypes.c_int),
                ("theta_deg", ctypes.c_double * 3), ("kw_rho", ctypes.c_double), ("kw_phi", ctypes.c_double),
                ("g_fp16", ctypes.c_int), ("eos", ctypes.c_int), ("omega", ctypes.c_double),
                ("nu", ctypes.c_double * 3)]


class Derived(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("T", "a", "b", "R", "rho_l", "rho_g", "C", "Psi0", "Tc", "kappa_rr", "kappa_pp", "kappa_rp",
                 "aA")]


class BatchConfig(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("tile_order", ctypes.c_int), ("graph_depth", ctypes.c_int),
                ("us_per_step", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("params", Params), ("mask", ctypes.POINTER(ctypes.c_uint8)),
                ("rho", ctypes.POINTER(ctypes.c_double)), ("phi", ctypes.POINTER(ctypes.c_double)),
                ("nsteps", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("done_s", ctypes.c_double), ("mass", ctypes.c_double * 6)]


_lib = None


def lib():
    """Load libtlb.so; raises if it was not built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtlb.so not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    i, d, vp, sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    sig = {
        "tlb_strerror": (ctypes.c_char_p, [i]),
        "tlb_last_error_message": (ctypes.c_char_p, []),
        "tlb_version": (i, [ctypes.POINTER(i)] * 3),
        "tlb_set_allocator": (i, [vp, vp, vp]),
        "tlb_params_default": (i, [ctypes.POINTER(Params)]),
        "tlb_create": (i, [i, i, i, i, dp, dp, dp, i, dp, ctypes.POINTER(vp)]),
        "tlb_create_ex": (i, [ctypes.POINTER(Params), ctypes.POINTER(vp)]),
        "tlb_destroy": (None, [vp]),
        "tlb_get_params": (i, [vp, ctypes.POINTER(Params)]),
        "tlb_get_derived": (i, [vp, ctypes.POINTER(Derived)]),
        "tlb_set_stream": (i, [vp, vp]),
        "tlb_set_solid": (i, [vp, u8p]),
        "tlb_init_fields": (i, [vp, dp, dp, dp]),
        "tlb_init_fields_device": (i, [vp, vp, vp, vp]),
        "tlb_step": (i, [vp, i]),
        "tlb_step_phase": (i, [vp, i]),
        "tlb_sync": (i, [vp]),
        "tlb_get_fields": (i, [vp, dp, dp, dp, dp]),
        "tlb_get_fields_device": (i, [vp, vp, vp, vp]),
        "tlb_diagnostics": (i, [vp, dp]),
        "tlb_get_aux": (i, [vp, i, dp]),
        "tlb_get_populations": (i, [vp, dp, dp]),
        "tlb_set_populations": (i, [vp, dp, dp]),
        "tlb_lattice_directions": (i, [i, ctypes.POINTER(i), dp]),
        "tlb_snapshot_bytes": (sz, [vp]),
        "tlb_snapshot": (i, [vp, vp, sz]),
        "tlb_restore": (i, [vp, vp, sz]),
        "tlb_steps_done": (ctypes.c_longlong, [vp]),
        "tlb_device_bytes": (sz, [vp]),
        "tlb_launch_count": (ctypes.c_longlong, [vp]),
        "tlb_step_batch": (i, [ctypes.POINTER(vp), i, i]),
        "tlb_server_create": (i, [sz, i, i, vp, ctypes.POINTER(vp)]),
        "tlb_submit": (i, [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "tlb_server_pump": (i, [vp]),
        "tlb_poll": (i, [vp, ctypes.c_uint64, ctypes.POINTER(Result), dp, dp]),
        "tlb_server_stats": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(sz)]),
        "tlb_server_destroy": (None, [vp]),
        "tlb_step_noalloc": (i, [ctypes.POINTER(Params), u8p, vp, vp, vp, vp, i, vp]),
        "tlb_set_force_calibration": (i, [ctypes.POINTER(Params), dp, dp, i]),
        "tlb_batch_create": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(BatchConfig), ctypes.POINTER(vp)]),
        "tlb_batch_step": (i, [vp, i]),
        "tlb_batch_tune": (i, [vp, i, ctypes.POINTER(BatchConfig)]),
        "tlb_batch_get_config": (i, [vp, ctypes.POINTER(BatchConfig)]),
        "tlb_batch_destroy": (None, [vp]),
        "tlb_derive": (i, [ctypes.POINTER(Params), ctypes.POINTER(Derived)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    register_force_calibration()
    return L


CALIBRATION_PATH = os.path.join(_HERE, "force_wetting_calibration.json")


def tlb_set_force_calibration(params, kappa_w, theta_deg):
    kw = np.ascontiguousarray(kappa_w, dtype=np.float64)
    th = np.ascontiguousarray(theta_deg, dtype=np.float64)
    return _check(lib().tlb_set_force_calibration(ctypes.byref(params), _dptr(kw), _dptr(th), len(kw)),
                  "tlb_set_force_calibration")


def register_force_calibration(path=None):
    """Register the force-wetting calibration tables of a JSON file (default:
    the tables shipped with the package, written by calibrate.py) with the
    library; returns the number of tables.  A missing default file registers
    nothing."""
    path = CALIBRATION_PATH if path is None else path
    if not os.path.exists(path):
        return 0
    import json

    with open(path) as fh:
        tables = json.load(fh)["tables"]
    for t in tables:
        p = make_params(t["lattice"], 8, 8, 1 if t["lattice"] == D2Q9 else 8, **t["params"])
        tlb_set_force_calibration(p, t["kappa_w"], t["theta_deg"])
    return len(tables)


def _check(rc, where):
    if rc < 0:
        raise TlbError(rc, where)
    return rc


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- thin wrappers with the C names ------------------------------------------
def tlb_params_default():
    p = Params()
    _check(lib().tlb_params_default(ctypes.byref(p)), "tlb_params_default")
    return p


def tlb_create_ex(params):
    h = ctypes.c_void_p()
    _check(lib().tlb_create_ex(ctypes.byref(params), ctypes.byref(h)), "tlb_create_ex")
    return h


def tlb_create(lattice, nx, ny, nz, densities, kappas, viscosities, wetting, angles_deg):
    h = ctypes.c_void_p()
    arr = lambda v: (ctypes.c_double * len(v))(*v)
    _check(lib().tlb_create(lattice, nx, ny, nz, arr(densities), arr(kappas), arr(viscosities), wetting,
                            arr(angles_deg), ctypes.byref(h)), "tlb_create")
    return h


def tlb_destroy(h):
    lib().tlb_destroy(h)


def tlb_set_stream(h, stream_ptr):
    _check(lib().tlb_set_stream(h, ctypes.c_void_p(stream_ptr)), "tlb_set_stream")


def tlb_set_solid(h, mask):
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    _check(lib().tlb_set_solid(h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "tlb_set_solid")


def tlb_init_fields(h, rho, phi, u=None):
    r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    p = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    _check(lib().tlb_init_fields(h, _dptr(r), _dptr(p), _dptr(uu)), "tlb_init_fields")


def tlb_init_fields_device(h, rho_ptr, phi_ptr, u_ptr=None):
    _check(lib().tlb_init_fields_device(h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(phi_ptr),
                                        ctypes.c_void_p(u_ptr) if u_ptr else None), "tlb_init_fields_device")


def tlb_step(h, n):
    return _check(lib().tlb_step(h, int(n)), "tlb_step")


def tlb_step_phase(h, phase):
    return _check(lib().tlb_step_phase(h, int(phase)), "tlb_step_phase")


def tlb_sync(h):
    return _check(lib().tlb_sync(h), "tlb_sync")


def tlb_get_fields_device(h, rho_ptr, phi_ptr, u_ptr=None):
    _check(lib().tlb_get_fields_device(h, ctypes.c_void_p(rho_ptr) if rho_ptr else None,
                                       ctypes.c_void_p(phi_ptr) if phi_ptr else None,
                                       ctypes.c_void_p(u_ptr) if u_ptr else None), "tlb_get_fields_device")


def tlb_lattice_directions(lattice):
    Q = 27 if lattice == D3Q27 else 9
    c = (ctypes.c_int * (3 * Q))()
    w = np.zeros(Q)
    _check(lib().tlb_lattice_directions(lattice, c, _dptr(w)), "tlb_lattice_directions")
    return np.array(c[:], dtype=np.int64).reshape(Q, 3), w


def tlb_step_batch(handles, nsteps):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    return _check(lib().tlb_step_batch(arr, len(handles), int(nsteps)), "tlb_step_batch")


def tlb_step_noalloc(params, mask, f_ptr, f_tmp_ptr, g_ptr, g_tmp_ptr, nsteps, stream_ptr=None):
    """Allocation-free stepping of caller-owned device populations (see tlb.h)."""
    m = None
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    return _check(lib().tlb_step_noalloc(ctypes.byref(params),
                                         None if m is None else m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                         ctypes.c_void_p(f_ptr), ctypes.c_void_p(f_tmp_ptr), ctypes.c_void_p(g_ptr),
                                         ctypes.c_void_p(g_tmp_ptr), int(nsteps),
                                         ctypes.c_void_p(stream_ptr) if stream_ptr else None), "tlb_step_noalloc")


_alloc_keep = []


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    import torch

    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

    def _alloc(nbytes, user):
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC(_alloc), FREE(_free)
    _alloc_keep[:] = [a, f]
    _check(lib().tlb_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None),
           "tlb_set_allocator")


def default_allocator():
    _check(lib().tlb_set_allocator(None, None, None), "tlb_set_allocator")
    _alloc_keep[:] = []


def tlb_derive(params):
    """Host-only derived constants (dict) of a parameter set (see tlb.h)."""
    d = Derived()
    _check(lib().tlb_derive(ctypes.byref(params), ctypes.byref(d)), "tlb_derive")
    return {k: getattr(d, k) for k, _ in Derived._fields_}


def make_params(lattice=D2Q9, nx=64, ny=64, nz=1, **kw):
    """Params from tlb_params_default() with the given overrides (names as in
    the workloads module: lam, kappa, chi, a, b, R, rho_l, rho_g, beta, tau_g,
    Gamma, wetting, theta_deg, kw_rho, kw_phi, g_fp16, eos, omega, nu)."""
    p = tlb_params_default()
    p.lattice, p.nx, p.ny, p.nz = lattice, nx, ny, nz
    for k, v in kw.items():
        if k in ("lam", "kappa", "theta_deg", "nu"):
            getattr(p, k)[:] = list(v)
        else:
            setattr(p, k, v)
    return p


class Lattice:
    """One lattice on the GPU.  Arrays are numpy, shaped (nz, ny, nx)."""

    def __init__(self, lattice=D2Q9, nx=64, ny=64, nz=1, stream=None, **kw):
        self.params = make_params(lattice, nx, ny, nz, **kw)
        self.lattice = lattice
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.D = 3 if lattice == D3Q27 else 2
        self.Q = 27 if lattice == D3Q27 else 9
        self.h = tlb_create_ex(self.params)
        if stream is not None:
            tlb_set_stream(self.h, stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value and _lib is not None:
            _lib.tlb_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def derived(self):
        d = Derived()
        _check(lib().tlb_get_derived(self.h, ctypes.byref(d)), "tlb_get_derived")
        return {k: getattr(d, k) for k, _ in Derived._fields_}

    def set_solid(self, mask):
        tlb_set_solid(self.h, mask)

    def init_fields(self, rho, phi, u=None):
        tlb_init_fields(self.h, rho, phi, u)

    def step(self, n=1):
        tlb_step(self.h, n)

    def sync(self):
        tlb_sync(self.h)

    def fields(self):
        N = self.N
        rho, phi, u, C = np.zeros(N), np.zeros(N), np.zeros(self.D * N), np.zeros(3 * N)
        _check(lib().tlb_get_fields(self.h, _dptr(rho), _dptr(phi), _dptr(u), _dptr(C)), "tlb_get_fields")
        s = self.shape
        return dict(rho=rho.reshape(s), phi=phi.reshape(s), u=u.reshape((self.D,) + s), C=C.reshape((3,) + s))

    def aux(self, name):
        """Auxiliary field by name (see AUX): p0, mu_rho, mu_phi, Fx..Fz, Pxx..Pyz,
        rho_ghost, phi_ghost."""
        out = np.zeros(self.N)
        _check(lib().tlb_get_aux(self.h, AUX[name], _dptr(out)), "tlb_get_aux")
        return out.reshape(self.shape)

    def diagnostics(self):
        out = np.zeros(6)
        _check(lib().tlb_diagnostics(self.h, _dptr(out)), "tlb_diagnostics")
        return dict(mass_rho=out[0], mass_phi=out[1], C1=out[2], C2=out[3], C3=out[4], kinetic=out[5])

    def populations(self):
        f, g = np.zeros(self.Q * self.N), np.zeros(self.Q * self.N)
        _check(lib().tlb_get_populations(self.h, _dptr(f), _dptr(g)), "tlb_get_populations")
        return f.reshape(self.Q, self.N), g.reshape(self.Q, self.N)

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        _check(lib().tlb_set_populations(self.h, _dptr(f), _dptr(g)), "tlb_set_populations")

    def snapshot(self):
        n = lib().tlb_snapshot_bytes(self.h)
        buf = ctypes.create_string_buffer(n)
        _check(lib().tlb_snapshot(self.h, buf, n), "tlb_snapshot")
        return buf

    def restore(self, buf):
        _check(lib().tlb_restore(self.h, buf, len(buf)), "tlb_restore")

    @property
    def steps_done(self):
        return lib().tlb_steps_done(self.h)

    @property
    def launches(self):
        return lib().tlb_launch_count(self.h)

    @property
    def device_bytes(self):
        return lib().tlb_device_bytes(self.h)


AUX = dict(p0=0, mu_rho=1, mu_phi=2, Fx=3, Fy=4, Fz=5, Pxx=6, Pyy=7, Pzz=8, Pxy=9, Pxz=10, Pyz=11,
           rho_ghost=12, phi_ghost=13)


def lattice_from_workload(wl, **over):
    """Lattice + solid mask + initial fields from a workloads.* dict."""
    p = dict(wl["params"])
    p.update(over)
    lat = Lattice(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], **p)
    lat.set_solid(wl["mask"])
    lat.init_fields(wl["rho"], wl["phi"])
    return lat


def _config_dict(c):
    return dict(variant=c.variant, tile_order=c.tile_order, graph_depth=c.graph_depth, us_per_step=c.us_per_step)


class Batch:
    """Resident batch of lattices (tlb_batch_*): one table, graph replays,
    tuned launch configuration.  The lattices must outlive the batch."""

    def __init__(self, lattices, variant=-1, tile_order=ORDER_LATTICE, graph_depth=8):
        handles = [l.h for l in lattices]
        arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
        cfg = BatchConfig(int(variant), int(tile_order), int(graph_depth), 0.0)
        h = ctypes.c_void_p()
        _check(lib().tlb_batch_create(arr, len(handles), ctypes.byref(cfg), ctypes.byref(h)), "tlb_batch_create")
        self.h = h
        self.lattices = list(lattices)

    def step(self, nsteps):
        _check(lib().tlb_batch_step(self.h, int(nsteps)), "tlb_batch_step")

    def tune(self, reps=4):
        c = BatchConfig()
        _check(lib().tlb_batch_tune(self.h, int(reps), ctypes.byref(c)), "tlb_batch_tune")
        return _config_dict(c)

    @property
    def config(self):
        c = BatchConfig()
        _check(lib().tlb_batch_get_config(self.h, ctypes.byref(c)), "tlb_batch_get_config")
        return _config_dict(c)

    def close(self):
        if self.h is not None and self.h.value:
            lib().tlb_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (tlb_server_*)."""

    def __init__(self, budget_bytes, max_active=64, steps_per_round=100, stream=None, policy=SCHED_FIFO,
                 max_wait_s=0.0):
        h = ctypes.c_void_p()
        _check(lib().tlb_server_create(int(budget_bytes), int(max_active), int(steps_per_round),
                                       ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)),
               "tlb_server_create")
        self.h = h
        self._keep = {}
        if policy != SCHED_FIFO or max_wait_s:
            self.set_policy(policy, max_wait_s)

    def set_policy(self, policy, max_wait_s=0.0):
        _check(lib().tlb_server_set_policy(self.h, int(policy), ctypes.c_double(max_wait_s)),
               "tlb_server_set_policy")

    def submit(self, lattice, nx, ny, nz, mask, rho, phi, nsteps, **kw):
        r = Request()
        r.params = make_params(lattice, nx, ny, nz, **kw)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        rr = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        pp = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        r.mask = None if m is None else m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        r.rho, r.phi, r.nsteps = _dptr(rr), _dptr(pp), int(nsteps)
        t = ctypes.c_uint64()
        _check(lib().tlb_submit(self.h, ctypes.byref(r), ctypes.byref(t)), "tlb_submit")
        self._keep[t.value] = (nx * ny * nz, (nz, ny, nx))
        return t.value

    def pump(self):
        return _check(lib().tlb_server_pump(self.h), "tlb_server_pump")

    def poll(self, ticket):
        res = Result()
        N, shape = self._keep[ticket]
        rho, phi = np.zeros(N), np.zeros(N)
        _check(lib().tlb_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(res), _dptr(rho), _dptr(phi)),
               "tlb_poll")
        out = dict(state=res.state, status=res.status, submit_s=res.submit_s, start_s=res.start_s,
                   done_s=res.done_s, mass=list(res.mass))
        if res.state in (REQ_DONE, REQ_FAILED):
            out["rho"], out["phi"] = rho.reshape(shape), phi.reshape(shape)
            del self._keep[ticket]
        return out

    def stats(self):
        q, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(lib().tlb_server_stats(self.h, ctypes.byref(q), ctypes.byref(a), ctypes.byref(b)), "tlb_server_stats")
        return dict(queued=q.value, active=a.value, bytes=b.value)

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tlb_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
