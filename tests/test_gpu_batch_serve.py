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


def test_resident_batch_equals_alone():
    """A resident batch (table built once, steps replayed from CUDA graphs of
    8 steps plus direct launches for the remainder) gives the fields of the
    lattices stepped alone, bit for bit, for D2Q9 and D3Q27."""
    from paper_1904_06881_gb300 import tlb

    specs = [(64, 45.0, W.WET_GEOM_INTERP), (128, 120.0, W.WET_GEOM_INTERP), (96, 90.0, W.WET_FORCE)]
    alone = [_drop(L, th, wet)[1] for L, th, wet in specs]
    mix = [_drop(L, th, wet)[1] for L, th, wet in specs]
    b = tlb.Batch(mix, graph_depth=8)
    for a in alone:
        a.step(43)
    b.step(43)
    for a, m in zip(alone, mix):
        assert m.steps_done == 43
        assert _same(a.fields(), m.fields())
    b.close()
    w3 = [W.c2_lubricated(nx=n, ny=n, nz=16, R=4.0, lub=2, gap=2, kw_rho=0.02) for n in (16, 24)]
    alone3 = [tlb.lattice_from_workload(w) for w in w3]
    mix3 = [tlb.lattice_from_workload(w) for w in w3]
    b3 = tlb.Batch(mix3, graph_depth=4)
    for a in alone3:
        a.step(11)
    b3.step(11)
    for a, m in zip(alone3, mix3):
        assert _same(a.fields(), m.fields())
    b3.close()


def test_batch_tuning_keeps_the_state_and_the_results():
    """The autotuner times candidate configurations with launches that
    recompute the current step: the lattices' fields are unchanged by it,
    the chosen configuration is one of the candidates, and stepping with it
    still gives the lattices' results alone (every variant and tile order
    runs the same arithmetic per node)."""
    from paper_1904_06881_gb300 import tlb

    specs = [(64, 60.0, W.WET_GEOM_INTERP), (256, 100.0, W.WET_GEOM_EXTRAP), (128, 90.0, W.WET_FORCE)]
    alone = [_drop(L, th, wet)[1] for L, th, wet in specs]
    mix = [_drop(L, th, wet)[1] for L, th, wet in specs]
    b = tlb.Batch(mix)
    b.step(5)
    before = [m.fields() for m in mix]
    cfg = b.tune(reps=2)
    after = [m.fields() for m in mix]
    assert all(_same(x, y) for x, y in zip(before, after))
    assert cfg["variant"] in (0, 1) and cfg["tile_order"] in (0, 1, 2) and cfg["graph_depth"] in (2, 8, 32)
    assert cfg["us_per_step"] > 0 and b.config == cfg
    b.step(40)
    for a in alone:
        a.step(45)
    for a, m in zip(alone, mix):
        assert _same(a.fields(), m.fields())


def test_batch_follows_lattices_stepped_alone():
    """Stepping one lattice of a batch on its own shifts its buffer parity
    against the others; the batch rewrites its table and stays exact."""
    from paper_1904_06881_gb300 import tlb

    specs = [(64, 60.0, W.WET_GEOM_INTERP), (96, 90.0, W.WET_FORCE)]
    alone = [_drop(L, th, wet)[1] for L, th, wet in specs]
    mix = [_drop(L, th, wet)[1] for L, th, wet in specs]
    b = tlb.Batch(mix, graph_depth=2)
    b.step(6)
    mix[0].step(3)
    b.step(7)
    alone[0].step(16)
    alone[1].step(13)
    for a, m in zip(alone, mix):
        assert _same(a.fields(), m.fields())


@pytest.mark.parametrize("policy,max_wait", [("fifo", 0.0), ("shortest", 0.0), ("shortest", 1e-9)])
def test_server_admission_order(policy, max_wait):
    """One lattice at a time (max_active = 1): FIFO admits in submission
    order; TLB_SCHED_SHORTEST admits the least work (nodes x steps) first,
    unless every request has waited past max_wait_s (then arrival order).
    Either way each result equals the lattice stepped alone."""
    from paper_1904_06881_gb300 import tlb

    specs = [(96, 60.0, 200), (48, 80.0, 100), (128, 100.0, 60), (64, 90.0, 300)]
    reqs = [(W.c3_lattice(dict(L=L, theta=th, wetting=W.WET_GEOM_INTERP)), n) for L, th, n in specs]
    pol = tlb.SCHED_FIFO if policy == "fifo" else tlb.SCHED_SHORTEST
    srv = tlb.Server(budget_bytes=256 << 20, max_active=1, steps_per_round=50, policy=pol, max_wait_s=max_wait)
    tickets = [srv.submit(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], wl["mask"], wl["rho"], wl["phi"], n,
                          **wl["params"]) for wl, n in reqs]
    results = {}
    for _ in range(200):
        srv.pump()
        for t in tickets:
            if t not in results:
                r = srv.poll(t)
                if r["state"] in (tlb.REQ_DONE, tlb.REQ_FAILED):
                    results[t] = r
        if len(results) == len(tickets):
            break
    srv.close()
    assert len(results) == len(tickets)
    starts = [results[t]["start_s"] for t in tickets]
    order = list(np.argsort(starts, kind="stable"))
    work = [wl["nx"] * wl["ny"] * wl["nz"] * n for wl, n in reqs]
    if policy == "fifo" or max_wait > 0:
        assert order == [0, 1, 2, 3]
    else:
        assert order == list(np.argsort(work, kind="stable"))
    for (wl, n), t in zip(reqs, tickets):
        assert results[t]["state"] == tlb.REQ_DONE
        a = tlb.lattice_from_workload(wl)
        a.step(n)
        assert _same(a.fields(), results[t])
        a.close()
