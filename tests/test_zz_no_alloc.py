"""The allocation-free entry point tlb_step_noalloc, for callers that cannot
allocate device memory while they run, gives the same populations as the
regular context API (tlb_step) on two calls in a row.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1904_06881_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_step_noalloc_matches_context_steps():
    import torch

    from paper_1904_06881_gb300 import tlb

    wl = W.c1_capillary(wetting=W.WET_GEOM_INTERP)
    ref = tlb.lattice_from_workload(wl)
    c, w = tlb.tlb_lattice_directions(wl["lattice"])
    f0, g0 = ref.populations()                      # FP64, library direction order
    dev = torch.device("cuda")
    f = torch.tensor((f0 - w[:, None]).astype(np.float32), device=dev)
    g = torch.tensor(g0.astype(np.float32), device=dev)
    f_tmp, g_tmp = torch.empty_like(f), torch.empty_like(g)
    p = tlb.make_params(wl["lattice"], wl["nx"], wl["ny"], wl["nz"], **wl["params"])
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                           # two calls in a row: the scratch is reused
        tlb.tlb_step_noalloc(p, wl["mask"], f.data_ptr(), f_tmp.data_ptr(), g.data_ptr(), g_tmp.data_ptr(), 7,
                             stream)
        ref.step(7)
        torch.cuda.synchronize()
        fr, gr = ref.populations()
        fn = f.double().cpu().numpy() + w[:, None]
        gn = g.double().cpu().numpy()
        fl = wl["mask"].reshape(-1) == 0
        # same kernels on the same inputs; the parity tests' one-step bound applies
        assert np.abs(fn[:, fl] - fr[:, fl]).max() <= 3e-6 * np.abs(fr[:, fl]).max(), call
        assert np.abs(gn[:, fl] - gr[:, fl]).max() <= 3e-6 * np.abs(gr[:, fl]).max(), call


def test_step_noalloc_rejects_oversize_lattice():
    from paper_1904_06881_gb300 import tlb

    p = tlb.make_params(tlb.D2Q9, 2048, 1024, 1)
    with pytest.raises(tlb.TlbError) as e:
        tlb.tlb_step_noalloc(p, None, 1, 1, 1, 1, 1)
    assert e.value.code == -1
