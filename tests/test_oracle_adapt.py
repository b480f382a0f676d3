"""Pins of the oracle's transfer of phi to an adapted mesh (Sec. 2.5,
"Adapting the grid structure"; reading R15: a block that exists in both
meshes keeps its values, a block whose refinement was removed takes the
restriction of its former children, a new child takes the prolongation of
Sec. 2.3 of its parent).  Pinned by what the operators fix, not by the
oracle itself:
  - an unchanged mesh carries phi bit for bit;
  - prolongation and restriction are exact on linear functions, and so are
    the Dirichlet and refinement ghosts the prolongation reads, so on a
    linear phi the carried field equals phi at the new cell centres;
  - refining a block and coarsening it again gives R P = I + (H^2/8) Delta_H
    on that block (each child mean picks up every face neighbour twice in
    2D and four times in 3D) and leaves every other cell unchanged."""
import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W


def lin2(X, Y, Z):
    return 1.0 + 2.0 * X - 3.0 * Y


def lin3(X, Y, Z):
    return 0.5 - X + 2.0 * Y + 1.5 * Z


def problem(dim, N, n0, refine, phi=None, geom=W.GEOM_CART, bc_type=None):
    base = (n0,) * dim + (1,) * (3 - dim)
    ref = np.asarray(refine, np.int32).reshape(-1, 4)
    bct = bc_type or (W.BC_DIRICHLET,) * 6
    return W.Problem("adapt", dim, N, geom, base, (0.0,) * 3, (1.0,) * 3, bct, (0.0,) * 6, ref, 64,
                     rhs=lambda X, Y, Z: 0.0 * X,
                     bc=None if phi is None else (lambda face, X, Y, Z: phi(X, Y, Z)))


def carried(p_old, p_new, phi_old):
    o = Oracle.from_problem(p_old)
    o.set_phi(phi_old)
    n = Oracle.from_problem(p_new)
    n.transfer_from(o)
    return n.get_phi()


def changed(refine, add=(), remove=()):
    rows = {tuple(int(x) for x in r) for r in np.asarray(refine, np.int32).reshape(-1, 4)}
    rows -= {tuple(r) for r in remove}
    rows |= {tuple(r) for r in add}
    return np.array(sorted(rows), np.int32).reshape(-1, 4)


# (dim, N, base cells, refinement of the old mesh, added, removed)
LINEAR_CASES = {
    "2d_refine": (2, 8, 32, [(0, 1, 1, 0), (0, 2, 1, 0)], [(0, 1, 2, 0), (1, 3, 3, 0), (0, 0, 0, 0)], []),
    "2d_coarsen": (2, 8, 32, [(0, 1, 1, 0), (0, 2, 1, 0), (0, 1, 2, 0), (0, 2, 2, 0), (1, 3, 3, 0)],
                   [(0, 3, 3, 0)], [(1, 3, 3, 0), (0, 2, 2, 0)]),
    "3d_refine": (3, 4, 16, [(0, 1, 1, 1)],
                  [(0, 2, 1, 1), (0, 1, 2, 1), (0, 1, 1, 2), (1, 3, 3, 3), (0, 0, 0, 0)], []),
    "3d_coarsen": (3, 4, 16, [(0, 1, 1, 1), (0, 2, 1, 1), (0, 1, 2, 1), (0, 1, 1, 2), (1, 3, 3, 3)],
                   [(0, 2, 2, 2)], [(1, 3, 3, 3), (0, 2, 1, 1)]),
    # every base block refined (the base level has no leaves, the refined
    # level no refinement faces), then one refinement removed: the coarsened
    # block's values are covered cells below every leaf stencil of the old mesh
    "2d_coarsen_full": (2, 8, 32, [(0, i, j, 0) for j in range(4) for i in range(4)], [], [(0, 1, 2, 0)]),
    "3d_coarsen_full": (3, 4, 16, [(0, i, j, k) for k in range(4) for j in range(4) for i in range(4)], [],
                        [(0, 2, 1, 1)]),
}


@pytest.mark.parametrize("name", sorted(LINEAR_CASES))
def test_linear_phi_is_carried_exactly(name):
    dim, N, n0, ref0, add, rem = LINEAR_CASES[name]
    phi = lin2 if dim == 2 else lin3
    p0 = problem(dim, N, n0, ref0, phi)
    p1 = problem(dim, N, n0, changed(ref0, add, rem), phi)
    X0, Y0, Z0, _ = W.leaf_cell_centres(p0)
    X1, Y1, Z1, _ = W.leaf_cell_centres(p1)
    got = carried(p0, p1, phi(X0, Y0, Z0))
    want = phi(X1, Y1, Z1)
    assert len(got) == len(want) != len(X0)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_cylindrical_field_linear_in_z_is_carried_exactly():
    """(r, z) mesh with the axis at r = 0: the axis ghost mirrors the first
    cell, which is exact for a field that does not depend on r."""
    fz = lambda X, Y, Z: 2.0 - 3.0 * Y  # noqa: E731
    bct = (W.BC_AXIS, W.BC_DIRICHLET, W.BC_DIRICHLET, W.BC_DIRICHLET, W.BC_DIRICHLET, W.BC_DIRICHLET)
    ref0 = [(0, 0, 1, 0), (0, 1, 1, 0), (0, 2, 1, 0)]
    p0 = problem(2, 8, 32, ref0, fz, geom=W.GEOM_CYL, bc_type=bct)
    p1 = problem(2, 8, 32, changed(ref0, [(0, 0, 2, 0), (1, 1, 3, 0)], [(0, 2, 1, 0)]), fz, geom=W.GEOM_CYL,
                 bc_type=bct)
    X0, Y0, Z0, _ = W.leaf_cell_centres(p0)
    X1, Y1, Z1, _ = W.leaf_cell_centres(p1)
    got = carried(p0, p1, fz(X0, Y0, Z0))
    assert np.abs(got - fz(X1, Y1, Z1)).max() <= 1e-13 * 5.0


def test_unchanged_mesh_carries_phi_bit_for_bit():
    p = problem(3, 4, 16, LINEAR_CASES["3d_coarsen"][3], lin3)
    x = np.random.default_rng(7).standard_normal(W.n_leaf_cells(p))
    assert np.array_equal(carried(p, p, x), x)


@pytest.mark.parametrize("dim", [2, 3])
def test_refine_then_coarsen_is_restriction_of_prolongation(dim):
    """Uniform mesh, random phi: refine one interior block, coarsen it back.
    On that block the result is c0 + (sum of the 2D face neighbours
    - 2D c0)/8; everywhere else phi is unchanged."""
    N, n0 = (8, 32) if dim == 2 else (4, 16)
    blk = (1, 2, 0) if dim == 2 else (1, 2, 1)
    p0 = problem(dim, N, n0, [])
    p1 = problem(dim, N, n0, [(0,) + blk])
    x = np.random.default_rng(3).standard_normal(W.n_leaf_cells(p0))
    o0 = Oracle.from_problem(p0)
    o0.set_phi(x)
    o1 = Oracle.from_problem(p1)
    o1.transfer_from(o0)
    o2 = Oracle.from_problem(p0)
    o2.transfer_from(o1)
    back = o2.get_phi()
    # the uniform grid as an array indexed [k][j][i] (x fastest)
    X, Y, Z, H = W.leaf_cell_centres(p0)
    ii = np.floor(X / H[:, 0]).astype(int)
    jj = np.floor(Y / H[:, 1]).astype(int)
    kk = np.floor(Z / H[:, 2]).astype(int) if dim == 3 else np.zeros_like(ii)
    g = np.zeros((n0 if dim == 3 else 1, n0, n0))
    g[kk, jj, ii] = x
    inside = (ii // N == blk[0]) & (jj // N == blk[1]) & ((kk // N == blk[2]) if dim == 3 else True)
    want = x.copy()
    for m in np.nonzero(inside)[0]:
        i, j, k = ii[m], jj[m], kk[m]
        nb = g[k, j, i - 1] + g[k, j, i + 1] + g[k, j - 1, i] + g[k, j + 1, i]
        if dim == 3:
            nb += g[k - 1, j, i] + g[k + 1, j, i]
        want[m] = x[m] + (nb - 2 * dim * x[m]) / 8.0
    assert np.array_equal(back[~inside], x[~inside])
    assert np.abs(back[inside] - want[inside]).max() <= 1e-14 * np.abs(x).max()
    assert np.abs(back[inside] - x[inside]).max() > 1e-3  # R P is not the identity


def test_periodic_round_trip_wraps_the_neighbours():
    """Uniform periodic 2D mesh: refine and coarsen back a block at the
    domain edge.  Its cells take c0 + (sum of face neighbours - 4 c0)/8 with
    the neighbours across the periodic faces taken from the other side."""
    N, n0 = 8, 32
    bct = (W.BC_PERIODIC,) * 4 + (W.BC_DIRICHLET,) * 2
    p0 = problem(2, N, n0, [], bc_type=bct)
    p1 = problem(2, N, n0, [(0, 0, 3, 0)], bc_type=bct)
    x = np.random.default_rng(4).standard_normal(W.n_leaf_cells(p0))
    x -= x.mean()
    o0 = Oracle.from_problem(p0)
    o0.set_phi(x)
    o1 = Oracle.from_problem(p1)
    o1.transfer_from(o0)
    o2 = Oracle.from_problem(p0)
    o2.transfer_from(o1)
    back = o2.get_phi()
    X, Y, Z, H = W.leaf_cell_centres(p0)
    ii = np.floor(X / H[:, 0]).astype(int)
    jj = np.floor(Y / H[:, 1]).astype(int)
    g = np.zeros((n0, n0))
    g[jj, ii] = x
    inside = (ii // N == 0) & (jj // N == 3)
    want = x.copy()
    for m in np.nonzero(inside)[0]:
        i, j = ii[m], jj[m]
        nb = g[j, (i - 1) % n0] + g[j, (i + 1) % n0] + g[(j - 1) % n0, i] + g[(j + 1) % n0, i]
        want[m] = x[m] + (nb - 4 * x[m]) / 8.0
    assert np.array_equal(back[~inside], x[~inside])
    assert np.abs(back[inside] - want[inside]).max() <= 1e-14 * np.abs(x).max()

