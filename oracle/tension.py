"""Oracle of the surface-tension measurements of Sec. III (bubble test,
Eq. QFdef, Eqs. theta1fromtension-theta3fromtension).

TEST INFRASTRUCTURE ONLY: used by the test-suite to check the library's
surface-tension sweep; written separately from it (it shares no code with
the package) and pinned in tests/test_tension_cpu.py.

  * bubble(pair, L, R, steps, **params): an FP64 oracle lattice of the bubble
    of workloads.bubble_2d, stepped;
  * laplace(o, pair): gamma = dP R with dP the bulk pressure p0 at the disc
    centre minus p0 at the box corner (Sec. III bubble test), R the radius of
    the disc whose area is the inner phase's total concentration;
  * deformation(C, inner, third): Eq. QFdef, max - min of the third phase's
    concentration over the interface band 0.05 < C_inner < 0.95 (the band is
    this project's reading of the paper's region Omega);
  * neumann(g12, g13, g23): the three cosine relations, in degrees.
"""
import math

from . import from_workload

# inner and third component (0 = C1 gas, 1 = C2, 2 = C3) of each bubble
_ROLES = {"12": (1, 2), "13": (2, 1), "23": (2, 0)}


def bubble(pair, L, R, steps, **params):
    from paper_1904_06881_gb300 import workloads as W

    o = from_workload(W.bubble_2d(pair, L, R, **params))
    o.step(steps)
    return o


def laplace(o, pair):
    inner = _ROLES[pair][0]
    C = o.fields()["C"]
    p0 = o.aux("p0")
    ny, nx = p0.shape[1], p0.shape[2]
    area = 0.0
    for y in range(ny):
        for x in range(nx):
            area += C[inner, 0, y, x]
    radius = math.sqrt(area / math.pi)
    return (p0[0, ny // 2, nx // 2] - p0[0, 0, 0]) * radius


def deformation(C, inner, third):
    """C: (3, ny, nx) concentrations of one 2D lattice."""
    lo, hi = None, None
    for y in range(C.shape[1]):
        for x in range(C.shape[2]):
            if 0.05 < C[inner, y, x] < 0.95:
                v = C[third, y, x]
                lo = v if lo is None or v < lo else lo
                hi = v if hi is None or v > hi else hi
    return float("nan") if lo is None else hi - lo


def neumann(g12, g13, g23):
    def angle(num, den):
        c = num / den
        return math.degrees(math.acos(c)) if abs(c) <= 1.0 else float("nan")
    t1 = angle(g23 ** 2 - g12 ** 2 - g13 ** 2, 2.0 * g12 * g13)
    t2 = angle(g13 ** 2 - g12 ** 2 - g23 ** 2, 2.0 * g12 * g23)
    t3 = angle(g12 ** 2 - g13 ** 2 - g23 ** 2, 2.0 * g13 * g23)
    return t1, t2, t3
