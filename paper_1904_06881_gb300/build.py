"""Build libtlb.so (CUDA kernels + C ABI) for sm_103a with nvcc, in-tree.

The library lands in paper_1904_06881_gb300/_build/libtlb.so.  Three
translation units (host ABI, D2Q9 kernels, D3Q27 kernels) compile in
parallel; only files newer than their object are rebuilt.

Test builds (the normal library is the product), loaded with
TLB_LIBRARY=<path> in the environment:

  * build(check=True), in _build_check/: the bounds-checked variant: every
    node index a kernel computes is tested against the lattice size, a bad
    one is recorded and its access skipped, and tlb_sync reports
    TLB_E_BOUNDS;
  * build(timeout_test=True), in _build_timeout/: the D3Q27 step's tensor
    copies are awaited for 16 bytes more than they send, so every such wait
    runs out after its one-second bound and tlb_sync reports TLB_E_TIMEOUT.

    python -m paper_1904_06881_gb300.build [--force] [--check | --timeout-test]
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtlb.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libtlb.so")
BUILD_TIMEOUT = os.path.join(HERE, "_build_timeout")
LIB_TIMEOUT = os.path.join(BUILD_TIMEOUT, "libtlb.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--use_fast_math", "-diag-suppress", "177"]
SOURCES = ["tlb_api.cu", "tlb_d2q9.cu", "tlb_d3q27.cu"]
HEADERS = ["tlb_device.cuh", "tlb_kernels.cuh", "tlb_internal.h"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def build(verbose=False, force=False, check=False, timeout_test=False):
    if check:
        bdir, lib, extra = BUILD_CHECK, LIB_CHECK, ["-DTLB_BOUNDS_CHECK"]
    elif timeout_test:
        bdir, lib, extra = BUILD_TIMEOUT, LIB_TIMEOUT, ["-DTLB_TEST_TMA_TIMEOUT"]
    else:
        bdir, lib, extra = BUILD, LIB, []
    os.makedirs(bdir, exist_ok=True)
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "tlb.h")]
    dep_time = _newest(deps)
    nvcc = _nvcc()

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        if not force and os.path.exists(o) and os.path.getmtime(o) >= max(dep_time, os.path.getmtime(s)):
            return o
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-I", os.path.join(ROOT, "include"), "-c", s, "-o", o + ".tmp"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(o + ".tmp", o)
        return o

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < _newest(objs):
        tmp = lib + ".%d.tmp" % os.getpid()
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, check="--check" in sys.argv,
                timeout_test="--timeout-test" in sys.argv))
