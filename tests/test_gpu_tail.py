"""The tail kernel (an option, off by default): the small levels at the
bottom of a V-cycle (Sec. 2.4) run as one cooperative launch per cycle leg,
with a grid barrier between the steps.  Each step is the flat one-thread-per-item form of the same cycle
step, so a cycle through the tail equals the launch-by-launch cycle up to
rounding order.  Checked with the tail covering every group it may (bound
2^40 cells) and off (bound 0): FMG + V-cycles against the FP64 oracle at
1e-12, the two GPU paths against each other, fewer launches with the tail,
mixed-precision solves to tolerance, and a batch tree by tree."""
import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
ALL = 1 << 40


@pytest.fixture(scope="module")
def mg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11370_gb300 import build as B
    B.build()
    import paper_1901_11370_gb300 as m
    return m


CASES = {
    "gauss3d_b8": lambda: W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05),
    "uniform3d_b8": lambda: W.cfg2_gauss3d(base=64, N=8, radii=(), sigma=0.05),
    "poisson2d_b8": lambda: W.cfg1_poisson2d(n=64, N=8),
    "cyl_k5_b16": lambda: W.cyl_ring_tree(24, force_k=5),
    "varcoef3d_periodic_b8": lambda: W.cfg3_varcoef3d(n=32, N=8, contrast=10.0),
    "varcoef3d_periodic_b16": lambda: W.cfg3_varcoef3d(n=32, N=16, seed=2, contrast=10.0),
}


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tail_cycles_match_oracle_and_the_launch_by_launch_cycle(mg, name):
    p = CASES[name]()
    out, launches = {}, {}
    for bound in (0, ALL):
        t = mg.Tree.from_problem(p)
        t.set_tail(bound)
        t.fmg()
        n0 = t.launch_count()
        t.vcycle(2)
        launches[bound] = t.launch_count() - n0
        out[bound] = t.get_phi().cpu().numpy()
    o = Oracle.from_problem(p)
    o.fmg()
    o.vcycle(2)
    ref = o.get_phi()
    assert rel(out[ALL], ref) <= TOL
    assert rel(out[0], ref) <= TOL
    assert rel(out[ALL], out[0]) <= TOL
    assert launches[ALL] < launches[0], launches


@pytest.mark.parametrize("name", ["gauss3d_b8", "cyl_k5_b16", "varcoef3d_periodic_b16"])
def test_tail_mixed_precision_solve_reaches_tolerance(mg, name):
    p = CASES[name]()
    t = mg.Tree.from_problem(p)
    t.set_tail(ALL)
    cyc, r = t.solve(1e-10, 40, precision=mg.MG_FP32_DC)
    assert r <= 1e-10
    o = Oracle.from_problem(p)
    r0, _ = o.residual_norm()
    o.set_phi(t.get_phi().cpu().numpy())
    r1, _ = o.residual_norm()
    assert r1 <= 1.05e-10 * r0, (cyc, r1 / r0)


def test_tail_is_off_by_default_and_a_bound_selects_groups(mg):
    """Off unless a bound is set; a bound takes the groups up to it."""
    p = CASES["uniform3d_b8"]()
    t = mg.Tree.from_problem(p)
    t.fmg()

    def launches():
        n0 = t.launch_count()
        t.vcycle(1)
        return t.launch_count() - n0
    n_default = launches()
    t.set_tail(0)
    n_off = launches()
    t.set_tail(4096)  # the 16^3 level only
    n_small = launches()
    t.set_tail(ALL)
    n_all = launches()
    assert n_default == n_off and n_all < n_small < n_off, (n_default, n_off, n_small, n_all)


def test_tail_batch_matches_oracle_per_tree(mg):
    import torch
    probs = [W.cyl_ring_tree(s, force_k=k) for s, k in ((21, 2), (22, 3), (23, 4), (24, 5), (25, 6), (26, 3))]
    res = {}
    for bound in (0, ALL):
        trees = [mg.Tree.from_problem(q, finalize=False) for q in probs]
        b = mg.Batch(trees)
        b.set_eps(torch.from_numpy(np.concatenate([W.leaf_field(q, "eps") for q in probs])).cuda())
        b.set_rhs(torch.from_numpy(np.concatenate([W.leaf_field(q, "rhs") for q in probs])).cuda())
        b.set_tail(bound)
        b.fmg()
        b.vcycle(2)
        res[bound] = (b.get_phi().cpu().numpy(), list(b.offsets))
    phi, off = res[ALL]
    for i, q in enumerate(probs):
        o = Oracle.from_problem(q)
        o.fmg()
        o.vcycle(2)
        ref = o.get_phi()
        assert rel(phi[off[i]:off[i + 1]], ref) <= TOL, i
        assert rel(res[0][0][off[i]:off[i + 1]], ref) <= TOL, i
