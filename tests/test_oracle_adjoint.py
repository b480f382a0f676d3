"""Pins of the oracle's transposed operators and adjoint solve (reading R16).

On refined meshes the composite operator A is not symmetric (Sec. 2.6: a
fine row reads the coarse cell B through its refinement ghost with weight
1/2, the coarse row reads the fine cells through the mean of the covered
cell), so the adjoint needs A^T.  The oracle forms it as the exact reverse
of its forward steps.  Pinned here by:
  * the dense transpose of the column-assembled A (several meshes, each far
    from symmetric, so apply_T = apply would fail);
  * the identity <A x, y> = <x, A^T y> on meshes too large to assemble;
  * the adjoint solve against a dense solve of A^T lambda = g;
  * central finite differences of L = 1/2 sum V (phi - t)^2 through dense
    forward solves, for dL/df and dL/deps;
  * on meshes without refinement faces, the closed-form eps gradient of
    or_eps_grad;
  * the transposes of the divergence and gradient of Sec. 4.1 by the same
    identity, and the cleaning map's adjoint by finite differences.
"""
import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W


def dense(o, fn):
    n = o.n_leaf
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = fn(e)
    return M


def mesh(name, rng=None):
    rng = rng or np.random.default_rng(1)
    if name == "2d_dirichlet_amr":
        ref = W.refine_spheres(2, 4, (16, 16, 1), (0,) * 3, (1,) * 3, (0.4, 0.55, 0), (0.3, 0.15))
        return Oracle(2, 4, 0, (0, 1, 0, 0, 0, 0), (0,) * 6, (16, 16), (0, 0), (1, 1), ref, 16)
    if name == "2d_periodic_amr_eps":
        ref = W.refine_spheres(2, 4, (16, 16, 1), (0,) * 3, (1,) * 3, (0.1, 0.55, 0), (0.3, 0.15), (True,) * 3)
        o = Oracle(2, 4, 0, (2,) * 6, (0,) * 6, (16, 16), (0, 0), (1, 1), ref, 16)
        o.set_eps(np.exp(0.5 * rng.standard_normal(o.n_leaf)))
        return o
    if name == "2d_periodic_amr":
        ref = W.refine_spheres(2, 4, (16, 16, 1), (0,) * 3, (1,) * 3, (0.1, 0.55, 0), (0.3, 0.15), (True,) * 3)
        return Oracle(2, 4, 0, (2,) * 6, (0,) * 6, (16, 16), (0, 0), (1, 1), ref, 16)
    if name == "3d_mixed_amr_eps":
        ref = W.refine_spheres(3, 4, (8,) * 3, (0,) * 3, (1,) * 3, (0.3, 0.3, 0.3), (0.3, 0.2))
        o = Oracle(3, 4, 0, (0, 1, 2, 2, 1, 0), (0,) * 6, (8,) * 3, (0,) * 3, (1,) * 3, ref, 8)
        o.set_eps(np.exp(0.5 * rng.standard_normal(o.n_leaf)))
        return o
    if name == "3d_small_amr":
        ref = W.refine_spheres(3, 4, (8,) * 3, (0,) * 3, (1,) * 3, (0.3, 0.3, 0.3), (0.25,))
        return Oracle(3, 4, 0, (0, 1, 2, 2, 1, 0), (0,) * 6, (8,) * 3, (0,) * 3, (1,) * 3, ref, 8)
    if name == "cyl_amr":
        ref = W.refine_spheres(2, 4, (16, 16, 1), (0,) * 3, (1,) * 3, (0.3, 0.5, 0), (0.25, 0.12))
        return Oracle(2, 4, 1, (3, 0, 0, 0, 0, 0), (0,) * 6, (16, 16), (0, 0), (1, 1), ref, 16)
    if name == "2d_helmholtz_neumann_amr":
        ref = W.refine_spheres(2, 4, (16, 16, 1), (0,) * 3, (1,) * 3, (0.4, 0.55, 0), (0.3, 0.15))
        return Oracle(2, 4, 0, (1, 1, 1, 1, 0, 0), (0,) * 6, (16, 16), (0, 0), (1, 1), ref, 16, helm=20.0)
    raise KeyError(name)


DENSE = ["2d_dirichlet_amr", "2d_periodic_amr_eps", "3d_mixed_amr_eps", "cyl_amr", "2d_helmholtz_neumann_amr"]


@pytest.mark.parametrize("name", DENSE)
def test_transpose_is_the_dense_transpose(name):
    o = mesh(name)
    o.set_homogeneous(True)
    A = dense(o, o.apply)
    AT = dense(o, o.apply_T)
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() > 1e-2 * scale  # refinement faces: far from symmetric
    assert np.abs(AT - A.T).max() <= 1e-14 * scale


@pytest.mark.parametrize("name", ["gauss3d", "periodic3d"])
def test_transpose_identity_on_larger_meshes(name):
    if name == "gauss3d":
        p = W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05)
        o = Oracle(p.dim, p.N, 0, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max)
    else:
        ref = W.refine_spheres(3, 4, (16,) * 3, (0,) * 3, (1,) * 3, (0.5, 0.4, 0.6), (0.3, 0.15), (True,) * 3)
        o = Oracle(3, 4, 0, (2,) * 6, (0,) * 6, (16,) * 3, (0,) * 3, (1,) * 3, ref, 64)
    o.set_homogeneous(True)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(o.n_leaf), rng.standard_normal(o.n_leaf)
    lhs, rhs = np.dot(o.apply(x), y), np.dot(x, o.apply_T(y))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(o.apply(x)).sum() * np.abs(y).max()


@pytest.mark.parametrize("name", ["2d_dirichlet_amr", "3d_mixed_amr_eps", "cyl_amr", "2d_helmholtz_neumann_amr",
                                  "2d_periodic_amr"])
def test_adjoint_solve_reaches_the_dense_solution(name):
    o = mesh(name)
    rng = np.random.default_rng(3)
    o.set_homogeneous(True)
    A = dense(o, o.apply)
    o.set_homogeneous(False)
    vol, _ = o.leaf_geometry()
    g = rng.standard_normal(o.n_leaf)
    lam, _ = o.adjoint(g, 60, 1e-13)
    it, rel = o.last_adjoint
    assert rel <= 1e-13 and it <= 40, (it, rel)
    if o._singular:
        # A^T lambda = g - V sum(g)/sum(V), lambda without its null-space part
        gh = g - vol * g.sum() / vol.sum()
        ref = np.linalg.lstsq(A.T, gh, rcond=None)[0]
        ref -= vol * ref.sum() / vol.sum()
    else:
        ref = np.linalg.solve(A.T, g)
    assert np.abs(lam - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["2d_dirichlet_amr", "3d_small_amr", "cyl_amr"])
def test_adjoint_gradients_match_finite_differences(name):
    """dL/df = lambda and dL/deps, L = 1/2 sum V (phi - t)^2, against central
    differences of dense forward solves (homogeneous boundary values, so
    A phi = f).  L is quadratic in f, so that difference is exact up to
    rounding; for eps the step is 1e-4 eps (O(step^2) truncation).  The
    difference of L is formed from the two solutions directly to avoid the
    cancellation of two nearly equal sums."""
    o = mesh(name)
    rng = np.random.default_rng(4)
    n = o.n_leaf
    vol, _ = o.leaf_geometry()
    eps = np.exp(0.4 * rng.standard_normal(n))
    f, t = rng.standard_normal(n), rng.standard_normal(n)

    def solve(f, eps):
        o.set_eps(eps)
        o.set_homogeneous(True)
        A = dense(o, o.apply)
        o.set_homogeneous(False)
        return np.linalg.solve(A, f)

    def dL(p1, p2, step):
        return 0.5 * np.dot(vol, (p1 - p2) * (p1 + p2 - 2 * t)) / (2 * step)

    phi = solve(f, eps)
    o.set_eps(eps)
    o.set_rhs(f)
    o.set_phi(phi)
    lam, geps = o.adjoint(vol * (phi - t), 80, 1e-14)
    for c in rng.choice(n, 5, replace=False):
        e = np.zeros(n)
        e[c] = 1e-3
        fd_f = dL(solve(f + e, eps), solve(f - e, eps), 1e-3)
        h = 1e-4 * eps[c]
        e = np.zeros(n)
        e[c] = h
        fd_e = dL(solve(f, eps + e), solve(f, eps - e), h)
        assert abs(fd_f - lam[c]) <= 1e-8 * abs(lam[c]), (c, fd_f, lam[c])
        assert abs(fd_e - geps[c]) <= 1e-6 * abs(geps[c]), (c, fd_e, geps[c])


@pytest.mark.parametrize("case", ["2d", "3d", "cyl"])
def test_general_eps_gradient_equals_the_uniform_formula(case):
    rng = np.random.default_rng(5)
    if case == "2d":
        o = Oracle(2, 8, 0, (0, 1, 0, 0, 0, 0), (0.2, 0.1, -0.3, 0.0, 0, 0), (32, 32), (0, 0), (1, 1))
    elif case == "3d":
        o = Oracle(3, 8, 0, (1, 1, 2, 2, 0, 0), (0.1, 0.0, 0, 0, 0.5, 0.0), (16, 16, 16), (0,) * 3, (1,) * 3)
    else:
        o = Oracle(2, 8, 1, (3, 0, 0, 0, 0, 0), (0, 0.4, 0, 0.1, 0, 0), (32, 32), (0, 0), (1, 1))
    o.set_eps(np.exp(0.4 * rng.standard_normal(o.n_leaf)))
    o.set_rhs(rng.standard_normal(o.n_leaf))
    o.fmg()
    o.vcycle(3)
    lam = rng.standard_normal(o.n_leaf)
    a, b = o.eps_grad_T(lam), o.eps_grad(lam)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("name", ["2d_periodic_amr", "2d_dirichlet_amr", "periodic3d"])
def test_divergence_and_gradient_transposes(name):
    if name == "periodic3d":
        ref = W.refine_spheres(3, 4, (16,) * 3, (0,) * 3, (1,) * 3, (0.5, 0.4, 0.6), (0.3, 0.15), (True,) * 3)
        o = Oracle(3, 4, 0, (2,) * 6, (0,) * 6, (16,) * 3, (0,) * 3, (1,) * 3, ref, 64)
    else:
        o = mesh(name)
    rng = np.random.default_rng(6)
    n, D = o.n_leaf, o.dim
    B, v = rng.standard_normal((D, n)), rng.standard_normal(n)
    lhs, rhs = np.dot(o.divergence(B), v), np.sum(B * o.divergence_T(v))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(o.divergence(B)).sum() * np.abs(v).max()
    # the projection is B - G phi: its phi-derivative is -G (homogeneous values)
    o.set_homogeneous(True)
    phi, u = rng.standard_normal(n), rng.standard_normal((D, n))
    o.set_phi(phi)
    Gphi = -o.project(np.zeros((D, n)))
    lhs, rhs = np.sum(Gphi * u), np.dot(phi, o.gradient_T(u))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(Gphi).sum() * np.abs(u).max()


def test_cleaning_adjoint_matches_finite_differences():
    """Divergence cleaning on a periodic refined mesh (Sec. 4.1): B_new =
    B - G phi, phi the zero-mean solution of A phi = P D B; the gradient of
    L = 1/2 sum V |B_new - B_t|^2 by the composed adjoint against central
    differences of dense solves (the map is linear, so they agree to
    rounding)."""
    o = mesh("2d_periodic_amr")
    rng = np.random.default_rng(7)
    n = o.n_leaf
    vol, _ = o.leaf_geometry()
    o.set_homogeneous(True)
    A = dense(o, o.apply)
    o.set_homogeneous(False)
    B, Bt = rng.standard_normal((2, n)), rng.standard_normal((2, n))

    def clean(B):
        f = o.divergence(B)
        f = f - np.dot(vol, f) / vol.sum()
        phi = np.linalg.lstsq(A, f, rcond=None)[0]
        o.set_phi(phi - np.dot(vol, phi) / vol.sum())
        return o.project(B)

    Bn = clean(B)
    gB = o.clean_adjoint(vol * (Bn - Bt), 80, 1e-14)
    for idx in [(0, 5), (1, 100), (0, 400), (1, 700)]:
        e = np.zeros((2, n))
        e[idx] = 1e-3
        B1, B2 = clean(B + e), clean(B - e)
        fd = 0.5 * np.sum(vol * (B1 - B2) * (B1 + B2 - 2 * Bt)) / 2e-3
        assert abs(fd - gB[idx]) <= 1e-8 * abs(fd), (idx, fd, gB[idx])
