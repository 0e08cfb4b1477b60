"""The bounded wait of the D3Q27 step's tensor copies, made to run out on
purpose without a GPU fault: a test build (-DTLB_TEST_TMA_TIMEOUT) has every
tile's barrier expect 16 bytes more than its copies send (the copies
themselves complete).  In a child process that loads it, a D3Q27 step
returns after the bound (two seconds per tile at most), tlb_sync reports
TLB_E_TIMEOUT (-7) and keeps reporting it (sticky, also from tlb_step), and a
D2Q9 lattice of the same process (no tensor copies) steps normally: the
context stays usable."""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def child():
    from paper_1904_06881_gb300 import tlb
    from paper_1904_06881_gb300 import workloads as W

    n = 32
    z, y, x = np.mgrid[0:16, 0:n, 0:n].astype(np.float64)
    C2 = 0.5 * (1.0 - np.tanh((np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - 8) ** 2) - 6.0) / 2.0))
    rho, phi = W.phase_fields(C2, np.zeros_like(C2))
    wl = dict(lattice=W.D3Q27, nx=n, ny=n, nz=16, params=W.base_params(), mask=np.zeros((16, n, n), np.uint8),
              rho=rho, phi=phi)
    lat = tlb.lattice_from_workload(wl)
    lib = tlb.lib()
    step1 = lib.tlb_step(lat.h, 1)              # runs; nothing flagged yet
    first = lib.tlb_sync(lat.h)                 # the tiles' waits ran out
    step2 = lib.tlb_step(lat.h, 1)              # runs and returns the sticky error
    second = lib.tlb_sync(lat.h)
    d2 = tlb.lattice_from_workload(W.c0_sessile_drop())
    d2.step(20)
    ok2 = lib.tlb_sync(d2.h)
    finite = bool(np.isfinite(d2.fields()["rho"]).all())
    print("RESULT", step1, first, step2, second, ok2, finite)


@pytest.mark.gpu
def test_tensor_copy_wait_runs_out_and_is_reported():
    from paper_1904_06881_gb300 import build as B

    lib = B.build(timeout_test=True)
    out = subprocess.run([sys.executable, os.path.abspath(__file__)], env=dict(os.environ, TLB_LIBRARY=lib),
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("RESULT")][-1].split()
    assert line[1:] == ["0", "-7", "-7", "-7", "0", "True"], line


if __name__ == "__main__":
    child()
