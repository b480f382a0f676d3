"""The adjoint on refined meshes through the C ABI against the oracle
(reading R16): the transposed composite operator, the adjoint solve and
dL/deps at equal iteration counts, the cleaning map's adjoint, and the
autograd wrappers.  Refinement faces make A non-symmetric (Sec. 2.6), so
these cases fail if A^T were taken as A.  Tolerance: the transpose matches
to 1e-13 (rounding of sums in a different order, FP64 atomics); the
iterations to 1e-11 relative."""
import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11370_gb300 import build as B
    B.build()
    import paper_1901_11370_gb300 as m
    return m


def rel_diff(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def cases():
    per = (True,) * 3
    return {
        "gauss3d_amr": W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05),
        "mixed3d_amr_eps_b4": W.Problem("mx", 3, 4, 0, (16,) * 3, (0,) * 3, (1,) * 3, (0, 1, 2, 2, 1, 0),
                                        (0.2, 0.1, 0, 0, -0.3, 0.0),
                                        W.refine_spheres(3, 4, (16,) * 3, (0,) * 3, (1,) * 3, (0.3, 0.4, 0.5),
                                                         (0.35, 0.2), (False, True, False)),
                                        512, rhs=lambda X, Y, Z: np.sin(3 * X) * np.cos(2 * Y) + Z,
                                        eps=lambda X, Y, Z: 1 + 0.5 * np.sin(5 * X * Y + Z)),
        "periodic3d_amr_b4": W.Problem("p3", 3, 4, 0, (16,) * 3, (0,) * 3, (1,) * 3, (2,) * 6, (0,) * 6,
                                       W.refine_spheres(3, 4, (16,) * 3, (0,) * 3, (1,) * 3, (0.5, 0.4, 0.6),
                                                        (0.3, 0.15), per), 64,
                                       rhs=lambda X, Y, Z: np.sin(2 * np.pi * X) * np.cos(2 * np.pi * (Y + Z))),
        "dirichlet2d_amr_eps_b8": W.Problem("d2", 2, 8, 0, (64, 64, 1), (0,) * 3, (1,) * 3, (0, 0, 0, 1, 0, 0),
                                            (0.1, -0.2, 0.0, 0.3, 0, 0),
                                            W.refine_spheres(2, 8, (64, 64, 1), (0,) * 3, (1,) * 3, (0.3, 0.6, 0),
                                                             (0.3, 0.15)), 64,
                                            rhs=lambda X, Y, Z: np.exp(-20 * ((X - 0.3) ** 2 + (Y - 0.6) ** 2)),
                                            eps=lambda X, Y, Z: np.exp(np.sin(4 * X) * np.cos(3 * Y))),
        "cyl_amr": W.cyl_ring_tree(11, force_k=4),
        "block2_3d": W.Problem("b2", 3, 2, 0, (8, 8, 8), (0,) * 3, (1,) * 3, (0, 1, 0, 0, 0, 0),
                               (0.1, 0.2, 0, 0, 0, 0),
                               W.refine_spheres(3, 2, (8,) * 3, (0,) * 3, (1,) * 3, (0.5, 0.5, 0.5), (0.3,)), 8,
                               rhs=lambda X, Y, Z: X * Y - Z),
    }


CASES = cases()


def both(mg, p):
    return mg.Tree.from_problem(p), Oracle.from_problem(p)


@pytest.mark.parametrize("name", sorted(CASES))
def test_transpose_matches_oracle(mg, name):
    t, o = both(mg, CASES[name])
    y = np.random.default_rng(1).standard_normal(o.n_leaf)
    a = t.apply_transpose(cuda(y)).cpu().numpy()
    b = o.apply_T(y)
    assert rel_diff(a, b) < 1e-13


@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_matches_oracle_at_equal_iterations(mg, name):
    p = CASES[name]
    t, o = both(mg, p)
    t.fmg(); o.fmg()
    t.vcycle(4); o.vcycle(4)
    g = np.random.default_rng(2).standard_normal(o.n_leaf)
    lam, ge = t.adjoint(cuda(g), n_cycles=8)
    lam_o, ge_o = o.adjoint(g, 8)
    assert rel_diff(lam.cpu().numpy(), lam_o) < 1e-11
    assert rel_diff(ge.cpu().numpy(), ge_o) < 1e-10


@pytest.mark.parametrize("name", ["gauss3d_amr", "periodic3d_amr_b4", "cyl_amr"])
def test_adjoint_solve_reaches_tolerance(mg, name):
    p = CASES[name]
    t, o = both(mg, p)
    t.fmg(); t.vcycle(2)
    g = np.random.default_rng(3).standard_normal(o.n_leaf)
    lam, _ = t.adjoint(cuda(g), want_eps=False, rel_tol=1e-12, max_cycles=60)
    it, rel = t.last_adjoint
    assert rel <= 1e-12 and it <= 40
    lam_o, _ = o.adjoint(g, 60, 1e-13)
    assert rel_diff(lam.cpu().numpy(), lam_o) < 1e-9
    # the returned lambda solves A^T lambda = g (after the compatibility
    # projection on a singular mesh), as the oracle's transpose measures it
    vol, _ = o.leaf_geometry()
    gh = g - vol * g.sum() / vol.sum() if o._singular else g
    r = gh - o.apply_T(lam.cpu().numpy())
    assert np.sqrt(np.dot(vol, (r / vol) ** 2) / vol.sum()) <= 2e-12 * np.sqrt(np.dot(vol, (gh / vol) ** 2) / vol.sum())


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_precision_adjoint_solve_matches_oracle(mg, name):
    """FP32 V-cycles as the approximate inverse inside the FP64 defect
    correction of the adjoint: the same fixed point, checked like the FP64
    form (against the oracle's lambda and by the oracle's transpose)."""
    p = CASES[name]
    t, o = both(mg, p)
    t.fmg(); t.vcycle(2)
    g = np.random.default_rng(3).standard_normal(o.n_leaf)
    lam, geps = t.adjoint(cuda(g), rel_tol=1e-12, max_cycles=60, precision=mg.MG_FP32_DC)
    it, rel = t.last_adjoint
    assert rel <= 1e-12 and it <= 40
    lam_o, _ = o.adjoint(g, 60, 1e-13)
    assert rel_diff(lam.cpu().numpy(), lam_o) < 1e-9
    lam64, geps64 = t.adjoint(cuda(g), rel_tol=1e-12, max_cycles=60)
    assert rel_diff(lam.cpu().numpy(), lam64.cpu().numpy()) < 1e-9
    assert rel_diff(geps.cpu().numpy(), geps64.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("name", ["periodic3d_amr_b4", "dirichlet2d_amr"])
def test_clean_adjoint_matches_oracle(mg, name):
    if name == "dirichlet2d_amr":
        ref = W.refine_spheres(2, 8, (64, 64, 1), (0,) * 3, (1,) * 3, (0.3, 0.6, 0), (0.3, 0.15))
        p = W.Problem("cl2", 2, 8, 0, (64, 64, 1), (0,) * 3, (1,) * 3, (0,) * 6, (0,) * 6, ref, 64)
    else:
        p = CASES[name]
    t, o = both(mg, p)
    gB = np.random.default_rng(4).standard_normal((p.dim, o.n_leaf))
    a = t.clean_adjoint(cuda(gB), rel_tol=1e-12, max_cycles=60).cpu().numpy()
    b = o.clean_adjoint(gB, 60, 1e-13)
    assert rel_diff(a, b) < 1e-9


def test_autograd_on_refined_mesh_matches_oracle(mg):
    """MGSolve backward on a refined 3D mesh with variable eps and mixed
    boundaries equals the oracle's adjoint of the same loss."""
    import torch
    from paper_1901_11370_gb300 import MGSolve
    p = CASES["mixed3d_amr_eps_b4"]
    t, o = both(mg, p)
    rng = np.random.default_rng(5)
    n = o.n_leaf
    f = cuda(W.leaf_field(p, "rhs")).requires_grad_()
    eps = cuda(W.leaf_field(p, "eps")).requires_grad_()
    tgt = cuda(rng.standard_normal(n))
    phi = MGSolve.apply(t, f, eps)
    loss = 0.5 * ((phi - tgt) ** 2).sum()
    loss.backward()
    o.solve(1e-13, 80)
    lam_o, ge_o = o.adjoint(o.get_phi() - tgt.cpu().numpy(), 80, 1e-13)
    assert rel_diff(f.grad.cpu().numpy(), lam_o) < 1e-9
    assert rel_diff(eps.grad.cpu().numpy(), ge_o) < 1e-8


def test_clean_autograd_on_refined_periodic_mesh(mg):
    import torch
    from paper_1901_11370_gb300 import CleanB
    p = CASES["periodic3d_amr_b4"]
    t, o = both(mg, p)
    rng = np.random.default_rng(6)
    B, Bt = rng.standard_normal((3, o.n_leaf)), rng.standard_normal((3, o.n_leaf))
    Bg = cuda(B).requires_grad_()
    Bn = CleanB.apply(t, Bg)
    vol = cuda(o.leaf_geometry()[0])
    loss = 0.5 * (vol * (Bn - cuda(Bt)) ** 2).sum()
    loss.backward()
    Bn_o, _, _ = o.clean(B, rel_tol=1e-13, max_cycles=80)
    g_o = o.clean_adjoint(o.leaf_geometry()[0] * (Bn_o - Bt), 80, 1e-13)
    assert rel_diff(Bn.detach().cpu().numpy(), Bn_o) < 1e-9
    assert rel_diff(Bg.grad.cpu().numpy(), g_o) < 1e-9


def test_unconverged_forward_raises(mg):
    import torch
    from paper_1901_11370_gb300 import MGError, MGSolve
    p = CASES["gauss3d_amr"]
    t = mg.Tree.from_problem(p)
    f = cuda(W.leaf_field(p, "rhs")).requires_grad_()
    with pytest.raises(MGError) as e:
        MGSolve.apply(t, f, None, 1e-12, 2)
    assert e.value.code == -4


def test_cleaning_workload_variant_matches_oracle(mg):
    """The cleaning workload's generator at a 64^3 base (8^3 blocks): the
    cleaning step and its adjoint pass against the oracle."""
    W_ = W
    ci = W_.CleanInputs(n=64, N=8)
    p = ci.problem
    B, Bt = ci.leaf_fields(), ci.target()
    t, o = mg.Tree.from_problem(p), Oracle.from_problem(p)
    Bn, f, cyc, rel = t.clean(cuda(B), 1e-12, 80)
    Bn_o, f_o, _ = o.clean(B, rel_tol=1e-13, max_cycles=80)
    assert rel_diff(f.cpu().numpy(), f_o) < 1e-12
    assert rel_diff(Bn.cpu().numpy(), Bn_o) < 1e-9
    vol, _ = o.leaf_geometry()
    g = vol * (Bn_o - Bt)
    a = t.clean_adjoint(cuda(g), 1e-12, 80).cpu().numpy()
    b = o.clean_adjoint(g, 80, 1e-13)
    a32 = t.clean_adjoint(cuda(g), 1e-12, 80, precision=mg.MG_FP32_DC).cpu().numpy()
    assert rel_diff(a32, b) < 1e-9
    assert rel_diff(a, b) < 1e-9
