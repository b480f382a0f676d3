"""The oracle's block loops run under OpenMP (the CPU-baseline leg times it
on every host core).  Within a colour the red-black updates are
order-independent and every other loop writes disjoint cells, so the solve
must give the same phi, bit for bit, and the same cycle count for any
thread count; the residual norm sums per-block partials in block order."""
import numpy as np

import oracle
from oracle import Oracle
from synth import workloads as W


def test_threads_give_identical_solutions():
    p = W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05)
    out = []
    for nt in (1, 4):
        oracle.set_threads(nt)
        o = Oracle.from_problem(p)
        cyc, hist = o.solve(1e-10, 30)
        out.append((cyc, hist, o.get_phi()))
    oracle.set_threads(0)
    (c1, h1, x1), (c4, h4, x4) = out
    assert c1 == c4 and h1 == h4
    assert np.array_equal(x1, x4)


def test_threads_give_identical_cylindrical_jacobi_cycles():
    p = W.cyl_ring_tree(11, force_k=4)
    out = []
    for nt in (1, 3):
        oracle.set_threads(nt)
        o = Oracle.from_problem(p)
        o.set_smoother(jacobi=True)
        o.fmg()
        o.vcycle(2)
        out.append((o.get_phi(), o.residual_norm()))
    oracle.set_threads(0)
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
