"""Failure handling, with the failures made on the host (no GPU fault): a
device allocator that gives out, requests the server must refuse or cannot
admit, next to requests that must complete undisturbed."""
import ctypes

import numpy as np
import pytest

from paper_1904_06881_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_failed_allocation_frees_what_was_allocated():
    """An allocator that fails after k successful calls: creation returns
    TLB_E_NOMEM and hands every block it got back; afterwards the default
    allocator works again."""
    import torch

    from paper_1904_06881_gb300 import tlb

    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    wl = W.c0_sessile_drop()
    try:
        for k in (0, 1, 3, 6):
            live, calls = set(), [0]

            def _alloc(nbytes, user):
                calls[0] += 1
                if calls[0] > k:
                    return None
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
                live.add(ptr)
                return ptr

            def _free(ptr, user):
                live.discard(ptr)
                torch.cuda.caching_allocator_delete(ptr)

            a, f = ALLOC(_alloc), FREE(_free)
            assert tlb.lib().tlb_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p),
                                               None) == 0
            with pytest.raises(tlb.TlbError) as e:
                tlb.Lattice(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], **wl["params"])
            assert e.value.code == -2, (k, e.value.code)
            assert calls[0] == k + 1 and not live, (k, calls[0], len(live))
    finally:
        tlb.default_allocator()
    lat = tlb.lattice_from_workload(wl)
    lat.step(10)
    assert np.isfinite(lat.fields()["rho"]).all()
    lat.close()


def _run_server(srv, tickets, pumps=2000):
    from paper_1904_06881_gb300 import tlb

    results = {}
    for _ in range(pumps):
        srv.pump()
        for t in tickets:
            if t not in results:
                r = srv.poll(t)
                if r["state"] in (tlb.REQ_DONE, tlb.REQ_FAILED):
                    results[t] = r
        if len(results) == len(tickets):
            break
    return results


def test_server_rejects_bad_requests_and_finishes_the_rest():
    """Requests with an unsupported parameter or larger than the memory
    budget are refused at submission; one whose device allocation fails at
    admission (an allocator that refuses large blocks) fails with
    TLB_E_NOMEM; the others complete with the results they give alone."""
    import torch

    from paper_1904_06881_gb300 import tlb

    good = [W.c3_lattice(dict(L=64, theta=70.0, wetting=W.WET_GEOM_INTERP)),
            W.c3_lattice(dict(L=64, theta=110.0, wetting=W.WET_GEOM_EXTRAP))]
    srv = tlb.Server(budget_bytes=16 << 20, max_active=4, steps_per_round=50)

    def submit(wl, n):
        return srv.submit(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], wl["mask"], wl["rho"], wl["phi"], n,
                          **wl["params"])

    bad = W.c3_lattice(dict(L=64, theta=70.0, wetting=W.WET_GEOM_INTERP))
    bad["params"] = dict(bad["params"], theta_deg=(10.0, 60.0, 120.0))      # outside [20, 160] deg
    with pytest.raises(tlb.TlbError) as e:
        submit(bad, 10)
    assert e.value.code == -4
    with pytest.raises(tlb.TlbError) as e:
        submit(W.c3_lattice(dict(L=512, theta=90.0, wetting=W.WET_GEOM_INTERP)), 10)
    assert e.value.code == -1

    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    live = set()

    def _alloc(nbytes, user):                  # refuses blocks of 400 KB and more
        if nbytes >= 400 << 10:
            return None
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
        live.add(ptr)
        return ptr

    def _free(ptr, user):
        live.discard(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC(_alloc), FREE(_free)
    assert tlb.lib().tlb_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None) == 0
    try:
        large = W.c3_lattice(dict(L=128, theta=90.0, wetting=W.WET_GEOM_INTERP))     # 590 KB population arrays
        tickets = [submit(good[0], 150), submit(large, 150), submit(good[1], 120)]
        res = _run_server(srv, tickets)
    finally:
        tlb.default_allocator()
    assert len(res) == 3
    assert res[tickets[1]]["state"] == tlb.REQ_FAILED and res[tickets[1]]["status"] == -2
    for wl, n, t in ((good[0], 150, tickets[0]), (good[1], 120, tickets[2])):
        r = res[t]
        assert r["state"] == tlb.REQ_DONE and r["status"] == 0
        a = tlb.lattice_from_workload(wl)
        a.step(n)
        fl = a.fields()
        assert np.array_equal(fl["rho"], r["rho"]) and np.array_equal(fl["phi"], r["phi"])
        a.close()


def test_invalid_initial_field_fails_alone():
    """A request whose initial density is negative at one node is refused at
    admission by the field check (TLB_E_INVAL); the request admitted beside
    it completes.  (Divergence during stepping is reported as TLB_E_DIVERGED:
    test_gpu_parity.test_diverged_state_is_reported.)"""
    from paper_1904_06881_gb300 import tlb

    ok = W.c3_lattice(dict(L=64, theta=80.0, wetting=W.WET_GEOM_INTERP))
    broken = W.c3_lattice(dict(L=64, theta=80.0, wetting=W.WET_GEOM_INTERP))
    broken["rho"] = broken["rho"].copy()
    broken["rho"][0, 40, 20] = -1.0
    srv = tlb.Server(budget_bytes=64 << 20, max_active=4, steps_per_round=50)
    tickets = [srv.submit(w["lattice"], w["nx"], w["ny"], w["nz"], w["mask"], w["rho"], w["phi"], 100, **w["params"])
               for w in (broken, ok)]
    res = _run_server(srv, tickets)
    assert res[tickets[0]]["state"] == tlb.REQ_FAILED and res[tickets[0]]["status"] == -1
    assert res[tickets[1]]["state"] == tlb.REQ_DONE and res[tickets[1]]["status"] == 0
