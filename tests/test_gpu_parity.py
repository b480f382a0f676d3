"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs at the same cycle counts.  Tolerance: max |phi_gpu - phi_oracle| <=
1e-12 max |phi_oracle| (FP64; red-black updates are order-independent within
a colour, so only rounding order differs)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from synth import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def mg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11370_gb300 import build as B
    B.build()
    import paper_1901_11370_gb300 as m
    return m


def both(mg, p, helm=0.0):
    import torch
    from paper_1901_11370_gb300 import Tree
    t = Tree.from_problem(p) if helm == 0 else None
    if helm:
        t = Tree(p.dim, p.N, p.geom, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max, helm=helm)
        t.set_rhs(torch.from_numpy(W.leaf_field(p, "rhs")).cuda())
        o = Oracle(p.dim, p.N, p.geom, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max, helm=helm)
        o.set_rhs(W.leaf_field(p, "rhs"))
    else:
        o = Oracle.from_problem(p)
    return t, o


def rel_diff(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def small_cases():
    per2 = (True, False, False)
    return {
        "cfg1_2d": W.cfg1_poisson2d(),
        "gauss3d_amr": W.cfg2_gauss3d(base=32, N=8, radii=(0.3, 0.15), sigma=0.05),
        "corner3d_amr_b4": W.Problem("corner", 3, 4, 0, (16, 16, 16), (0,) * 3, (1,) * 3, (0,) * 6,
                                     (0.3, -0.1, 0.2, 0.0, 0.5, 0.1),
                                     W.refine_spheres(3, 4, (16,) * 3, (0,) * 3, (1,) * 3, (0.05, 0.1, 0.0), (0.45, 0.25)),
                                     512, rhs=lambda X, Y, Z: np.sin(3 * X) * np.cos(2 * Y) + Z,
                                     eps=lambda X, Y, Z: 1 + 0.5 * np.sin(5 * X * Y + Z)),
        "periodic2d_amr_eps": W.Problem("per", 2, 4, 0, (32, 32, 1), (0, 0, 0), (1, 1, 1), (2, 2, 0, 1, 0, 0),
                                        (0, 0, 0.2, -0.5, 0, 0),
                                        W.refine_spheres(2, 4, (32, 32, 1), (0, 0, 0), (1, 1, 1), (0.02, 0.5, 0),
                                                         (0.3, 0.15), per2),
                                        512, rhs=lambda X, Y, Z: np.exp(-30 * ((X - 0.1) ** 2 + (Y - 0.5) ** 2)),
                                        eps=lambda X, Y, Z: np.exp(np.sin(2 * math.pi * X))),
        "cyl_amr": W.cyl_ring_tree(11, force_k=4),
        "cyl_odd_k3": W.cyl_ring_tree(12, force_k=3),
        "varcoef3d_singular": W.cfg3_varcoef3d(n=32, N=8, contrast=10.0),
        "varcoef3d_b16": W.cfg3_varcoef3d(n=64, N=16, contrast=10.0, seed=3),
        "block2_3d": W.Problem("b2", 3, 2, 0, (8, 8, 8), (0,) * 3, (1,) * 3, (0, 1, 0, 0, 0, 0), (0.1, 0.2, 0, 0, 0, 0),
                               W.refine_spheres(3, 2, (8,) * 3, (0,) * 3, (1,) * 3, (0.5, 0.5, 0.5), (0.3,)), 8,
                               rhs=lambda X, Y, Z: X * Y - Z),
    }


CASES = small_cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_fmg_and_vcycles_match_oracle(mg, name):
    p = CASES[name]
    t, o = both(mg, p)
    t.fmg()
    o.fmg()
    d1 = rel_diff(t.get_phi().cpu().numpy(), o.get_phi())
    t.vcycle(3)
    o.vcycle(3)
    d2 = rel_diff(t.get_phi().cpu().numpy(), o.get_phi())
    assert d1 < TOL and d2 < TOL, (d1, d2)
    l2, li, r = t.residual_norm(want_res=True)
    l2o, lio, ro = o.residual_norm(want_res=True)
    # residuals differ by at most |A| |dphi| (|A| <= 4 D eps_max / h_min^2) plus rounding of f - A phi
    X, Y, Z, H = W.leaf_cell_centres(p)
    emax = np.abs(W.leaf_field(p, "eps")).max()
    dphi = np.abs(t.get_phi().cpu().numpy() - o.get_phi()).max()
    bound = 2 * (4 * p.dim * emax / H[:, :p.dim].min() ** 2) * (dphi + 1e-15 * np.abs(o.get_phi()).max()) \
        + 1e-13 * (np.abs(W.leaf_field(p, "rhs")).max() + 1.0)
    assert np.abs(r.cpu().numpy() - ro).max() <= bound
    assert abs(l2 - l2o) <= bound + 1e-12 * l2o and abs(li - lio) <= bound + 1e-12 * lio


def test_helmholtz_matches_oracle(mg):
    p = W.cfg1_poisson2d(n=32, N=8)
    t, o = both(mg, p, helm=50.0)
    t.fmg(); o.fmg()
    t.vcycle(2); o.vcycle(2)
    assert rel_diff(t.get_phi().cpu().numpy(), o.get_phi()) < TOL


def test_set_phi_then_vcycle_matches(mg):
    """Warm start: set_phi restricts covered cells and refills ghosts on both sides."""
    import torch
    p = CASES["gauss3d_amr"]
    t, o = both(mg, p)
    x0 = np.random.default_rng(0).standard_normal(o.n_leaf)
    t.set_phi(torch.from_numpy(x0).cuda())
    o.set_phi(x0)
    t.vcycle(2, n_down=1, n_up=3)
    o.set_cycle(1, 3)
    o.vcycle(2)
    assert rel_diff(t.get_phi().cpu().numpy(), o.get_phi()) < TOL


def test_solve_reaches_tolerance_fp64(mg):
    p = W.cfg1_poisson2d()
    t, o = both(mg, p)
    cyc, rel = t.solve(1e-10, 30, fmg_first=True)
    oc, hist = o.solve(1e-10, 30, fmg_first=True)
    assert rel <= 1e-10 and cyc == oc, (cyc, oc, rel, hist)
    assert rel_diff(t.get_phi().cpu().numpy(), o.get_phi()) < 1e-11


@pytest.mark.parametrize("name", ["gauss3d_amr", "cyl_amr", "corner3d_amr_b4", "varcoef3d_singular"])
def test_mixed_precision_defect_correction(mg, name):
    """FP32 cycles inside FP64 defect correction reach 1e-10 relative residual
    as judged by the oracle's own FP64 residual of the GPU solution."""
    p = CASES[name]
    t, o = both(mg, p)
    cyc, rel = t.solve(1e-10, 40, fmg_first=True, precision=mg.MG_FP32_DC)
    assert rel <= 1e-10
    # the FP32 cycles converge like the FP64 ones (a wrong FP32 transfer
    # kernel would cost cycles)
    c64, _ = mg.Tree.from_problem(p).solve(1e-10, 40, fmg_first=True)
    assert cyc <= c64 + 1, (cyc, c64)
    r0 = o.residual_norm()[0]  # oracle phi = 0
    o.set_phi(t.get_phi().cpu().numpy())
    r = o.residual_norm()[0]
    assert r <= 1.5e-10 * r0, (r, r0)
    o2 = Oracle.from_problem(p)
    o2.solve(1e-13, 60)
    x, xr = t.get_phi().cpu().numpy(), o2.get_phi()
    if W.BC_DIRICHLET not in p.bc_type[:2 * p.dim]:  # solution defined up to a constant
        vol, _ = o2.leaf_geometry()
        x, xr = x - np.dot(vol, x) / vol.sum(), xr - np.dot(vol, xr) / vol.sum()
    err = np.linalg.norm(x - xr) / np.linalg.norm(xr)
    assert err < 1e-8, err


@pytest.mark.parametrize("case", ["2d", "3d", "cyl"])
def test_adjoint_matches_oracle(mg, case):
    import torch
    from paper_1901_11370_gb300 import Tree
    rng = np.random.default_rng(23)
    if case == "2d":
        args = (2, 8, 0, (0, 1, 0, 0, 0, 0), (0.2, 0.1, -0.3, 0.0, 0, 0), (32, 32), (0, 0), (1, 1))
    elif case == "3d":
        args = (3, 8, 0, (1, 1, 2, 2, 0, 0), (0.1, 0.0, 0, 0, 0.5, 0.0), (16, 16, 16), (0,) * 3, (1,) * 3)
    else:
        args = (2, 8, 1, (3, 0, 0, 0, 0, 0), (0, 0.4, 0, 0.1, 0, 0), (32, 32), (0, 0), (1, 1))
    o = Oracle(*args)
    t = Tree(*args)
    eps = np.exp(0.4 * rng.standard_normal(o.n_leaf))
    f = rng.standard_normal(o.n_leaf)
    g = rng.standard_normal(o.n_leaf)
    o.set_eps(eps); o.set_rhs(f)
    t.set_eps(torch.from_numpy(eps).cuda()); t.set_rhs(torch.from_numpy(f).cuda())
    for x in (o, t):
        x.fmg()
        x.vcycle(10)
    lam_o, ge_o = o.adjoint(g, n_vcycles=10)
    lam, ge = t.adjoint(torch.from_numpy(g).cuda(), n_cycles=10)
    assert rel_diff(lam.cpu().numpy(), lam_o) < 1e-11
    assert rel_diff(ge.cpu().numpy(), ge_o) < 1e-10


def test_adjoint_rejects_singular_variable_eps_on_refined_mesh(mg):
    """Without Dirichlet faces the compatibility condition sum V f = 0 needs
    conserved fluxes, which variable eps at refinement faces breaks: the
    adjoint says so (MG_ERR_UNSUPPORTED) instead of returning a gradient."""
    import torch
    from paper_1901_11370_gb300 import MGError
    q = CASES["periodic2d_amr_eps"]
    p = W.Problem("per_neu", 2, 4, 0, q.base, q.lo, q.hi, (2, 2, 1, 1, 0, 0), (0,) * 6, q.refine, 512,
                  rhs=q.rhs, eps=q.eps)
    t, _ = both(mg, p)
    with pytest.raises(MGError) as e:
        t.adjoint(torch.zeros(t.n_leaf, dtype=torch.float64, device="cuda"))
    assert e.value.code == -9


def test_autograd_function_gradients(mg):
    """MGSolve backward equals the oracle's dL/df and dL/deps."""
    import torch
    from paper_1901_11370_gb300 import MGSolve, Tree
    args = (2, 8, 0, (0, 0, 0, 0, 0, 0), (0,) * 6, (32, 32), (0, 0), (1, 1))
    rng = np.random.default_rng(4)
    t = Tree(*args)
    n = t.n_leaf
    f = torch.from_numpy(rng.standard_normal(n)).cuda().requires_grad_()
    eps = torch.from_numpy(np.exp(0.3 * rng.standard_normal(n))).cuda().requires_grad_()
    tgt = torch.from_numpy(rng.standard_normal(n)).cuda()
    phi = MGSolve.apply(t, f, eps)
    loss = 0.5 * ((phi - tgt) ** 2).sum()
    loss.backward()
    o = Oracle(*args)
    o.set_eps(eps.detach().cpu().numpy())
    o.set_rhs(f.detach().cpu().numpy())
    o.fmg(); o.vcycle(40)
    lam_o, ge_o = o.adjoint(o.get_phi() - tgt.cpu().numpy(), n_vcycles=30)
    assert rel_diff(f.grad.cpu().numpy(), lam_o) < 1e-9
    assert rel_diff(eps.grad.cpu().numpy(), ge_o) < 1e-8


def _clean_case(name):
    if name == "periodic3d_amr":
        ref = W.refine_spheres(3, 4, (16,) * 3, (0,) * 3, (1,) * 3, (0.5, 0.4, 0.6), (0.3, 0.15), (True,) * 3)
        return W.Problem("cl3", 3, 4, 0, (16,) * 3, (0,) * 3, (1,) * 3, (2,) * 6, (0,) * 6, ref, 64)
    ref = W.refine_spheres(2, 8, (64, 64, 1), (0,) * 3, (1,) * 3, (0.3, 0.6, 0), (0.3, 0.15))
    return W.Problem("cl2", 2, 8, 0, (64, 64, 1), (0,) * 3, (1,) * 3, (0, 0, 0, 0, 0, 0), (0,) * 6, ref, 64)


@pytest.mark.parametrize("name", ["periodic3d_amr", "dirichlet2d_amr"])
def test_divergence_cleaning_matches_oracle(mg, name):
    """div B, the solve and B - grad phi (Sec. 4.1) against the oracle at the
    same cycle counts."""
    import torch
    from paper_1901_11370_gb300 import Tree
    p = _clean_case(name)
    X, Y, Z, _ = W.leaf_cell_centres(p)
    B = np.stack([np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y), np.cos(2 * np.pi * Y + Z),
                  np.sin(2 * np.pi * (X + Z))][:p.dim])
    o = Oracle(p.dim, p.N, 0, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max)
    t = Tree(p.dim, p.N, 0, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max)
    Bg = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    d_o = o.divergence(B)
    d_g = t.divergence(Bg).cpu().numpy()
    assert rel_diff(d_g, d_o) < TOL
    vol, _ = o.leaf_geometry()
    f = d_o - (np.dot(vol, d_o) / vol.sum() if name.startswith("periodic") else 0.0)
    o.set_rhs(f)
    t.set_rhs(torch.from_numpy(f).cuda())
    for x in (o, t):
        x.fmg()
        x.vcycle(4)
    Bn_o = o.project(B)
    Bn_g = t.project(Bg).cpu().numpy()
    assert rel_diff(Bn_g, Bn_o) < TOL
    # cleaning reduces the divergence by a large factor (not to zero: the
    # wide central divergence and the compact Laplacian differ, Sec. 4.1)
    assert np.linalg.norm(o.divergence(Bn_o)) < 0.2 * np.linalg.norm(d_o)


@pytest.mark.parametrize("name", ["periodic3d_amr", "dirichlet2d_amr"])
def test_fourth_order_divergence_matches_oracle(mg, name):
    """The fourth-order divergence (reading R14: second order beside physical
    and refinement faces) and a cleaning step built on it, against the
    oracle."""
    import torch
    from paper_1901_11370_gb300 import Tree
    p = _clean_case(name)
    X, Y, Z, _ = W.leaf_cell_centres(p)
    B = np.stack([np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y), np.cos(2 * np.pi * Y + Z),
                  np.sin(2 * np.pi * (X + Z))][:p.dim])
    o = Oracle(p.dim, p.N, 0, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max)
    t = Tree(p.dim, p.N, 0, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max)
    Bg = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    d_o = o.divergence(B, order=4)
    d_g = t.divergence(Bg, order=4).cpu().numpy()
    assert rel_diff(d_g, d_o) < TOL
    assert np.abs(d_o - o.divergence(B)).max() > 1e-6 * np.abs(d_o).max()  # not the second-order field
    Bn, f, cyc, rel = t.clean(Bg, 1e-10, 60, order=4)
    vol, _ = o.leaf_geometry()
    fo = d_o - (np.dot(vol, d_o) / vol.sum() if name.startswith("periodic") else 0.0)
    assert rel_diff(f.cpu().numpy(), fo) < TOL
    with pytest.raises(mg.MGError):
        t.divergence(Bg, order=3)


@pytest.mark.parametrize("name", ["periodic3d_amr", "dirichlet2d_amr"])
def test_clean_entry_point_matches_oracle(mg, name):
    """mg_clean (div B, zero-mean projection on the periodic problem, solve,
    B - grad phi, all on the device) against the oracle's cleaning solved
    far below the tolerance."""
    import torch
    from paper_1901_11370_gb300 import Tree
    p = _clean_case(name)
    X, Y, Z, _ = W.leaf_cell_centres(p)
    B = np.stack([np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y), np.cos(2 * np.pi * Y + Z),
                  np.sin(2 * np.pi * (X + Z))][:p.dim])
    o = Oracle(p.dim, p.N, 0, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max)
    t = Tree(p.dim, p.N, 0, p.bc_type, p.bc_val, p.base, p.lo, p.hi, p.refine, p.coarse_max)
    Bn, f, cyc, rel = t.clean(torch.from_numpy(np.ascontiguousarray(B)).cuda(), 1e-12, 60)
    assert rel <= 1e-12
    Bn_o, f_o, _ = o.clean(B, rel_tol=1e-13, max_cycles=80)
    assert rel_diff(f.cpu().numpy(), f_o) < TOL
    assert rel_diff(Bn.cpu().numpy(), Bn_o) < 1e-8
    Bj, _, _, relj = t.clean(torch.from_numpy(np.ascontiguousarray(B)).cuda(), 1e-10, 80,
                             smoother=mg.MG_SMOOTH_JACOBI)
    assert relj <= 1e-10 and rel_diff(Bj.cpu().numpy(), Bn_o) < 1e-6


def test_cleaning_autograd_matches_oracle(mg):
    """CleanB backward (uniform periodic mesh) equals the oracle's gradient,
    the cleaning of B_new - B_t (pinned against finite differences)."""
    import torch
    from paper_1901_11370_gb300 import CleanB, Tree
    rng = np.random.default_rng(12)
    args = (3, 8, 0, (2,) * 6, (0.0,) * 6, (16, 16, 16), (0,) * 3, (1,) * 3)
    t = Tree(*args)
    o = Oracle(*args)
    B = rng.standard_normal((3, o.n_leaf))
    Bt = rng.standard_normal((3, o.n_leaf))
    Bg = torch.from_numpy(B).cuda().requires_grad_()
    Bn = CleanB.apply(t, Bg)
    loss = 0.5 * ((Bn - torch.from_numpy(Bt).cuda()) ** 2).sum()
    loss.backward()
    Bn_o, _, _ = o.clean(B, rel_tol=1e-13, max_cycles=80)
    grad_o, _, _ = o.clean(Bn_o - Bt, rel_tol=1e-13, max_cycles=80)
    assert rel_diff(Bn.detach().cpu().numpy(), Bn_o) < 1e-9
    assert rel_diff(Bg.grad.cpu().numpy(), grad_o) < 1e-9


def test_incompatible_rhs_is_reported(mg):
    """A singular problem (periodic and homogeneous Neumann faces) with a
    right-hand side of nonzero mean cannot reach a small residual: mg_solve
    says so (MG_ERR_INCOMPATIBLE_RHS) instead of cycling; the projected
    right-hand side solves."""
    import torch
    p = W.cfg3_varcoef3d(n=16, N=8, seed=4, contrast=5.0)
    t = mg.Tree.from_problem(p)
    f = torch.from_numpy(W.leaf_field(p, "rhs")).cuda() + 0.5
    t.set_rhs(f)
    with pytest.raises(mg.MGError) as e:
        t.solve(1e-10, 20)
    assert e.value.code == -7
    vol = t.leaf_volumes()
    t.set_rhs(f - torch.dot(vol, f) / vol.sum())
    t.set_phi(torch.zeros_like(f))
    cyc, rel = t.solve(1e-10, 40)
    assert rel <= 1e-10


JACOBI_CASES = ["cfg1_2d", "gauss3d_amr", "cyl_amr", "periodic2d_amr_eps", "varcoef3d_b16", "block2_3d"]


@pytest.mark.parametrize("name", JACOBI_CASES)
def test_jacobi_smoother_matches_oracle(mg, name):
    """Weighted-Jacobi smoothing (reading R13: every cell from the values
    before the step, omega = 4/5 in 2D, 6/7 in 3D): FMG and V-cycles match
    the oracle's Jacobi cycles to 1e-12."""
    p = CASES[name]
    t, o = both(mg, p)
    o.set_smoother(jacobi=True)
    t.fmg(smoother=mg.MG_SMOOTH_JACOBI)
    o.fmg()
    t.vcycle(2, smoother=mg.MG_SMOOTH_JACOBI)
    o.vcycle(2)
    assert rel_diff(t.get_phi().cpu().numpy(), o.get_phi()) < TOL


def test_jacobi_mixed_precision_solve(mg):
    """FP32 Jacobi cycles inside FP64 defect correction reach 1e-10 by the
    oracle's own residual; an explicit weight is honoured (and checked)."""
    p = CASES["gauss3d_amr"]
    t, o = both(mg, p)
    cyc, rel = t.solve(1e-10, 60, precision=mg.MG_FP32_DC, smoother=mg.MG_SMOOTH_JACOBI, omega=0.8)
    assert rel <= 1e-10
    r0 = o.residual_norm()[0]
    o.set_phi(t.get_phi().cpu().numpy())
    assert o.residual_norm()[0] <= 1.5e-10 * r0
    with pytest.raises(mg.MGError):
        t.vcycle(1, smoother=mg.MG_SMOOTH_JACOBI, omega=1.5)


@pytest.mark.parametrize("name", ["gauss3d_amr", "cyl_amr", "varcoef3d_b16"])
def test_per_level_schedule_matches_oracle(mg, name):
    """A non-default schedule of smoothing steps per level (mg_set_schedule)
    runs the same cycles as the oracle's per-level schedule."""
    p = CASES[name]
    t, o = both(mg, p)
    nl = len(o.levels())
    down = [(l % 3) + 1 for l in range(nl)]
    up = [3 - (l % 3) for l in range(nl)]
    t.set_schedule(down, up)
    o.set_schedule(down, up)
    assert list(t.schedule()[0]) == down
    t.fmg(); o.fmg()
    t.vcycle(2); o.vcycle(2)
    assert rel_diff(t.get_phi().cpu().numpy(), o.get_phi()) < TOL


def test_schedule_tuner_picks_a_converging_schedule(mg):
    import torch
    p = CASES["varcoef3d_b16"]
    t, o = both(mg, p)
    inner, ms = t.tune_schedule(1e-10, 60, mg.MG_FP32_DC)
    assert inner in (1, 2, 3, 4) and ms > 0
    d, u = t.schedule()
    assert (d >= 0).all() and (u >= 0).all()
    t.set_phi(torch.zeros(t.n_leaf, dtype=torch.float64, device="cuda"))
    cyc, rel = t.solve(1e-10, 60, precision=mg.MG_FP32_DC, inner_cycles=inner)
    o.set_phi(t.get_phi().cpu().numpy())
    r0 = Oracle.from_problem(p).residual_norm()[0]
    assert rel <= 1e-10 and o.residual_norm()[0] <= 1.05e-10 * r0


@pytest.mark.parametrize("name", ["cfg1_2d", "gauss3d_amr", "varcoef3d_singular", "cyl_amr", "periodic2d_amr_eps"])
def test_paper_coarse_solve_matches_oracle(mg, name):
    """The paper's coarse-grid solve (red-black smoothing of the coarsest
    level to 1e-8 absolute / relative, at most 1000 sweeps) on both sides:
    FMG and V-cycles agree to 1e-12, and a mixed-precision solve reaches
    1e-10 by the oracle's residual."""
    import torch
    p = CASES[name]
    t, o = both(mg, p)
    o.set_coarse_mode(True)
    t.fmg(coarse_mode=mg.MG_COARSE_SMOOTH)
    o.fmg()
    t.vcycle(3, coarse_mode=mg.MG_COARSE_SMOOTH)
    o.vcycle(3)
    assert rel_diff(t.get_phi().cpu().numpy(), o.get_phi()) < TOL
    t.set_phi(torch.zeros(t.n_leaf, dtype=torch.float64, device="cuda"))
    cyc, rel = t.solve(1e-10, 60, precision=mg.MG_FP32_DC, coarse_mode=mg.MG_COARSE_SMOOTH)
    assert rel <= 1e-10
    o2 = Oracle.from_problem(p)
    r0 = o2.residual_norm()[0]
    o2.set_phi(t.get_phi().cpu().numpy())
    assert o2.residual_norm()[0] <= 1.5e-10 * r0
