"""Batched stepping (many uneven lattices, one launch per phase) and the
request server: every lattice gives the same result alone and in the mix.
A lattice stepped alone runs as a batch of one through the same kernels, so
the results are bit-identical."""
import numpy as np
import pytest

from paper_1904_06881_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _drop(L, theta, wet):
    from paper_1904_06881_gb300 import tlb

    wl = W.c3_lattice(dict(L=L, theta=theta, wetting=wet))
    return wl, tlb.lattice_from_workload(wl)


def _same(fa, fb):
    return np.array_equal(fa["rho"], fb["rho"]) and np.array_equal(fa["phi"], fb["phi"])


def test_batched_equals_alone():
    from paper_1904_06881_gb300 import tlb

    specs = [(64, 45.0, W.WET_GEOM_INTERP), (128, 120.0, W.WET_GEOM_INTERP), (96, 90.0, W.WET_FORCE),
             (64, 70.0, W.WET_GEOM_EXTRAP)]
    alone, mix = [], []
    for L, th, wet in specs:
        alone.append(_drop(L, th, wet)[1])
        mix.append(_drop(L, th, wet)[1])
    for a in alone:
        a.step(300)
    tlb.tlb_step_batch([m.h for m in mix], 300)
    for a, m in zip(alone, mix):
        assert m.steps_done == 300
        assert _same(a.fields(), m.fields())


def test_server_alone_vs_mix():
    from paper_1904_06881_gb300 import tlb

    reqs = []
    for k, (L, th, wet, n) in enumerate([(64, 50.0, W.WET_GEOM_INTERP, 200), (128, 110.0, W.WET_GEOM_INTERP, 350),
                                         (96, 90.0, W.WET_FORCE, 120), (64, 75.0, W.WET_GEOM_EXTRAP, 260)]):
        reqs.append((W.c3_lattice(dict(L=L, theta=th, wetting=wet)), n))
    srv = tlb.Server(budget_bytes=64 << 20, max_active=3, steps_per_round=40)
    tickets = []
    for wl, n in reqs:
        p = dict(wl["params"])
        tickets.append(srv.submit(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], wl["mask"], wl["rho"], wl["phi"], n,
                                  **p))
    results = {}
    for _ in range(1000):
        srv.pump()
        for t in tickets:
            if t in results:
                continue
            r = srv.poll(t)
            if r["state"] in (tlb.REQ_DONE, tlb.REQ_FAILED):
                results[t] = r
        if len(results) == len(tickets):
            break
    assert len(results) == len(tickets)
    for (wl, n), t in zip(reqs, tickets):
        r = results[t]
        assert r["state"] == tlb.REQ_DONE and r["status"] == 0
        a = tlb.lattice_from_workload(wl)
        a.step(n)
        assert _same(a.fields(), r)


def test_one_wave_and_large_launches_agree():
    """A D2Q9 launch with more tiles than fit on the GPU at 3 CTAs per SM runs
    the 64-register build of the step kernel, a smaller one the 80-register
    build of the same code.  A lattice alone (small launch) and in a mix with a
    512 x 512 lattice (large launch) gives bit-identical fields."""
    from paper_1904_06881_gb300 import tlb

    specs = [(64, 45.0, W.WET_GEOM_INTERP), (96, 90.0, W.WET_FORCE), (64, 120.0, W.WET_GEOM_EXTRAP)]
    alone = [_drop(L, th, wet)[1] for L, th, wet in specs]
    mix = [_drop(L, th, wet)[1] for L, th, wet in specs] + [_drop(512, 60.0, W.WET_GEOM_INTERP)[1]]
    for a in alone:
        a.step(200)
    tlb.tlb_step_batch([m.h for m in mix], 200)
    for a, m in zip(alone, mix):
        assert _same(a.fields(), m.fields())
