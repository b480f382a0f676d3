"""mg_tree_adapt (Sec. 2.5, "Adapting the grid structure") against the
oracle: the carried phi of every leaf equals the oracle's transfer
(reading R15) to rounding, the adapted tree then cycles like a tree built
from scratch, the old tree is left as it was, and bad requests fail with
their error codes.  The larger case checks a property that holds at any
size: a linear phi is carried exactly."""
import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W
from test_oracle_adapt import LINEAR_CASES, changed, lin2, lin3, problem

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(scope="module")
def mg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11370_gb300 import build as B
    B.build()
    import paper_1901_11370_gb300 as m
    return m


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def with_rhs(p, seed):
    """the same mesh with a seeded smooth right-hand side"""
    c = np.random.default_rng(seed).uniform(0.3, 0.7, 3)
    p.rhs = lambda X, Y, Z: np.exp(-30 * ((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)) - 0.2
    return p


@pytest.mark.parametrize("name", sorted(LINEAR_CASES))
def test_adapt_matches_oracle_transfer_and_cycles(mg, name):
    dim, N, n0, ref0, add, rem = LINEAR_CASES[name]
    phi = lin2 if dim == 2 else lin3
    p0 = with_rhs(problem(dim, N, n0, ref0, phi), 1)
    p1 = with_rhs(problem(dim, N, n0, changed(ref0, add, rem), phi), 2)
    x = np.random.default_rng(5).standard_normal(W.n_leaf_cells(p0))
    t0 = mg.Tree.from_problem(p0)
    t0.set_phi(cuda(x))
    t1 = t0.adapt(add, rem)
    o0 = Oracle.from_problem(p0)
    o0.set_phi(x)
    o1 = Oracle.from_problem(p1)
    o1.transfer_from(o0)
    assert t1.n_leaf == o1.n_leaf
    assert rel(t1.get_phi().cpu().numpy(), o1.get_phi()) < TOL
    assert np.array_equal(t0.get_phi().cpu().numpy(), x)  # the old tree keeps its leaves
    # the adapted tree cycles from the carried phi like the oracle
    f1 = W.leaf_field(p1, "rhs")
    t1.set_rhs(cuda(f1))
    o1.set_rhs(f1)
    t1.vcycle(2)
    o1.vcycle(2)
    assert rel(t1.get_phi().cpu().numpy(), o1.get_phi()) < 1e-12


@pytest.mark.parametrize("name", ["2d_coarsen_full", "3d_coarsen_full"])
def test_adapt_after_cycles_carries_fresh_covered_cells(mg, name):
    """The old tree is cycled first, so its covered cells below the leaf
    stencils hold stale V-cycle values; a removed refinement must still take
    the mean of its former children (R15)."""
    dim, N, n0, ref0, add, rem = LINEAR_CASES[name]
    p0 = with_rhs(problem(dim, N, n0, ref0, None), 3)
    p1 = with_rhs(problem(dim, N, n0, changed(ref0, add, rem), None), 4)
    x = np.random.default_rng(6).standard_normal(W.n_leaf_cells(p0))
    t0 = mg.Tree.from_problem(p0)
    o0 = Oracle.from_problem(p0)
    t0.set_phi(cuda(x))
    o0.set_phi(x)
    t0.vcycle(2)
    o0.vcycle(2)
    assert rel(t0.get_phi().cpu().numpy(), o0.get_phi()) < 1e-12
    t1 = t0.adapt(add, rem)
    o1 = Oracle.from_problem(p1)
    o1.transfer_from(o0)
    assert rel(t1.get_phi().cpu().numpy(), o1.get_phi()) < 1e-12


def test_adapt_cylindrical_matches_oracle(mg):
    bct = (W.BC_AXIS, W.BC_DIRICHLET, W.BC_DIRICHLET, W.BC_DIRICHLET, W.BC_DIRICHLET, W.BC_DIRICHLET)
    ref0 = [(0, 0, 1, 0), (0, 1, 1, 0), (0, 2, 1, 0)]
    add, rem = [(0, 0, 2, 0), (1, 1, 3, 0)], [(0, 2, 1, 0)]
    p0 = problem(2, 8, 32, ref0, lin2, geom=W.GEOM_CYL, bc_type=bct)
    p1 = problem(2, 8, 32, changed(ref0, add, rem), lin2, geom=W.GEOM_CYL, bc_type=bct)
    x = np.random.default_rng(9).standard_normal(W.n_leaf_cells(p0))
    t0 = mg.Tree.from_problem(p0)
    t0.set_phi(cuda(x))
    t1 = t0.adapt(add, rem)
    o0 = Oracle.from_problem(p0)
    o0.set_phi(x)
    o1 = Oracle.from_problem(p1)
    o1.transfer_from(o0)
    assert rel(t1.get_phi().cpu().numpy(), o1.get_phi()) < TOL


def test_adapt_without_changes_is_the_identity(mg):
    dim, N, n0, ref0, _, _ = LINEAR_CASES["3d_coarsen"]
    p = problem(dim, N, n0, ref0, lin3)
    x = np.random.default_rng(2).standard_normal(W.n_leaf_cells(p))
    t0 = mg.Tree.from_problem(p)
    t0.set_phi(cuda(x))
    t1 = t0.adapt()
    assert np.array_equal(t1.get_phi().cpu().numpy(), x)
    bt = t1.build_times()
    assert all(v >= 0 for v in bt) and bt[0] > 0 and bt[3] > 0
    # the sweep kernels are taken over level by level, not tuned again
    for l in range(len(t0.levels())):
        assert t1.sweep_variant(l, mg.MG_FP64) == t0.sweep_variant(l, mg.MG_FP64)


def test_adapt_larger_mesh_carries_linear_phi_exactly(mg):
    """Base 64^3 in 8^3 blocks, one refinement level inside r < 0.3 of the
    centre; the adapted mesh refines the shell 0.3 <= r < 0.4 and coarsens
    r < 0.15 (one level each, so both meshes stay balanced)."""
    N, n0 = 8, 64
    nb = n0 // N
    c = (np.arange(nb) + 0.5) / nb - 0.5
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)  # [k, j, i]
    rows = lambda m: [(0, i, j, k) for k, j, i in zip(*np.nonzero(m))]  # noqa: E731
    ref0 = rows(r < 0.3)
    add, rem = rows((r >= 0.3) & (r < 0.4)), rows(r < 0.15)
    assert add and rem
    p0 = problem(3, N, n0, ref0, lin3)
    p1 = problem(3, N, n0, changed(ref0, add, rem), lin3)
    X0, Y0, Z0, _ = W.leaf_cell_centres(p0)
    X1, Y1, Z1, _ = W.leaf_cell_centres(p1)
    t0 = mg.Tree.from_problem(p0)
    t0.set_phi(cuda(lin3(X0, Y0, Z0)))
    t1 = t0.adapt(add, rem)
    want = lin3(X1, Y1, Z1)
    assert t1.n_leaf == len(want)
    assert rel(t1.get_phi().cpu().numpy(), want) < TOL


def test_adapt_rejects_bad_requests(mg):
    dim, N, n0, ref0, _, _ = LINEAR_CASES["2d_coarsen"]
    t0 = mg.Tree.from_problem(problem(dim, N, n0, ref0, lin2))
    codes = []
    for add, rem in (([(0, 1, 1, 0)], []),          # refined already: not a leaf
                     ([(0, 9, 9, 0)], []),          # no such block
                     ([], [(0, 1, 1, 0)]),          # has a refined child (1, 3, 3)
                     ([], [(0, 3, 3, 0)]),          # not refined
                     ([(2, 6, 6, 0)], [])):         # depth-2 child of (1, 3, 3): breaks 2:1 balance
        with pytest.raises(mg.MGError) as e:
            t0.adapt(add, rem)
        codes.append(e.value.code)
    assert codes == [-1, -1, -1, -1, -2]
    t0.vcycle(1)  # the old tree is still usable


def test_adapt_periodic_3d_matches_oracle(mg):
    """Periodic in x and y, Dirichlet in z, 3D: parent ghosts across the
    periodic faces feed the prolongation of blocks at the domain edge."""
    bct = (W.BC_PERIODIC,) * 4 + (W.BC_DIRICHLET,) * 2
    ref0 = [(0, 0, 1, 1), (0, 3, 1, 1), (0, 1, 1, 1), (0, 2, 3, 0)]
    add, rem = [(0, 0, 0, 1), (0, 0, 1, 0), (1, 0, 2, 2)], [(0, 2, 3, 0)]  # (1, 0, 2, 2) wraps to (0, 3, 1, 1)
    p0 = problem(3, 4, 16, ref0, lin3, bc_type=bct)
    p1 = problem(3, 4, 16, changed(ref0, add, rem), lin3, bc_type=bct)
    x = np.random.default_rng(13).standard_normal(W.n_leaf_cells(p0))
    t0 = mg.Tree.from_problem(p0)
    t0.set_phi(cuda(x))
    t1 = t0.adapt(add, rem)
    o0 = Oracle.from_problem(p0)
    o0.set_phi(x)
    o1 = Oracle.from_problem(p1)
    o1.transfer_from(o0)
    assert rel(t1.get_phi().cpu().numpy(), o1.get_phi()) < TOL

